// Admission of the serving loop's requests (host logic only, no CUDA calls, so
// that it is testable without a GPU).
//
// The server keeps its requests in FIFO order.  A free slot starts the head
// request when the device memory it needs fits; the requests queued behind it
// join the same device batch while the batch stays within a job limit and the
// memory that is left.  The memory the server may count on is re-read for
// every decision: the configured budget, but never more than what is free on
// the device right now plus what the server's own workspaces already hold
// (they are reused by the next batch).  So allocations made elsewhere in the
// process, after the server was created, hold requests back instead of making
// their batches fail.
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdint>

namespace sa {

// Bytes the running batches and a new one may take together.
inline uint64_t admission_cap(uint64_t budget, uint64_t free_now, uint64_t held) {
    return std::min(budget, free_now + held);
}

// How many requests at the front of `q` (a sequence of items, `view(item)`
// giving {jobs, est_bytes}) start now as one batch, given the estimates of the
// batches already running (in_use) and the cap above: 0 when the head request
// does not fit; else the head plus each following request while the batch has
// at most max_jobs jobs (the head alone may exceed it) and the memory fits.
// *est receives the bytes of the admitted requests.
template <class Q, class View>
size_t admit_front(const Q& q, View view, uint64_t in_use, uint64_t cap, uint64_t max_jobs,
                   uint64_t* est) {
    *est = 0;
    uint64_t jobs = 0;
    size_t k = 0;
    for (const auto& item : q) {
        const auto v = view(item);
        const uint64_t r_jobs = v.first, r_est = v.second;
        if (in_use + *est + r_est > cap) break;
        if (k > 0 && jobs + r_jobs > max_jobs) break;
        jobs += r_jobs;
        *est += r_est;
        k++;
    }
    return k;
}

}  // namespace sa
