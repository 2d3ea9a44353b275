// Allocation-free score pass: sa_align_batch_noalloc.
//
// Some callers cannot let a library call cudaMalloc: code running inside a
// host framework that owns all device memory through its own allocator (a
// raw cudaMalloc there fragments or double-books the pool), and
// latency-sensitive callers that cannot afford the device-wide
// synchronisation cudaMalloc / cudaFree may imply.  This entry point serves
// them: it computes the same results as sa_align_batch_dev with want_cigar = 0
// (score, ends, second best), on the caller's device buffers, and keeps every
// intermediate array in one fixed, file-scope device array instead of
// allocating.
//
// The array is SA_NOALLOC_SCRATCH_BYTES (32 MiB) on every device that loads the
// library, held until the process exits.  All calls share it and it keeps the
// previous call's contents, so everything that must start at zero is cleared
// at the start of each call, and two calls whose work overlaps on the GPU
// (different streams, or different host threads) race on it.  Batches whose
// intermediate arrays do not fit are rejected with SA_EINVAL and a message
// giving the size needed.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = SA_NOALLOC_SCRATCH_BYTES;

// the scratch itself; host code only ever sees its device address through
// cudaGetSymbolAddress
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

int err(int code, const char* fmt, ...) {
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    return sa::set_error(code, msg);
}

// Device address of g_scratch, looked up once per device with that device
// current (the host-side symbol is only a stand-in, never a device address).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

int scratch_address(int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices) return err(SA_EINVAL, "device %d out of range", device);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return err(SA_ECUDA, "cudaGetSymbolAddress of the no-alloc scratch failed: %s",
                       cudaGetErrorString(e));
        }
        g_addr[device] = p;
    }
    *out = static_cast<unsigned char*>(g_addr[device]);
    return SA_OK;
}

// control block at the start of the scratch (cleared every call)
struct Ctl {
    sa::PlanStats st;
    uint32_t item_counter;
    uint32_t _pad[3];
    uint32_t hist[sa::kNumKeys];
};

inline size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// JobState -> sa_result for a score-only call: the row sa_align_batch_dev's
// finalisation writes with want_cigar = 0 (one helper serves both)
__global__ void k_noalloc_results(const sa_job* __restrict__ jobs, uint32_t n_jobs,
                                  const sa::JobState* __restrict__ state, int32_t min_score,
                                  sa_result* __restrict__ out) {
    const uint32_t job = blockIdx.x * blockDim.x + threadIdx.x;
    if (job >= n_jobs) return;
    out[job] = sa::score_result(jobs[job], state[job], min_score);
}

#define CK(expr)                                                                              \
    do {                                                                                      \
        const cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess) {                                                              \
            cudaGetLastError();                                                               \
            return err(SA_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));              \
        }                                                                                     \
    } while (0)

int run(sa_reference* R, const sa_params* P, const sa_job* d_jobs, uint32_t n_jobs,
        const char* d_reads, uint64_t reads_len, sa_result* d_out, void* stream) {
    if (!R) return err(SA_EINVAL, "reference is NULL");
    // the same limits as every other alignment entry point (a LOCAL best score
    // must fit the 21 bits of the 32-bit score pass's keys: match <= 2047)
    sa::Score sc;
    const int prc = sa::check_scoring(P, &sc);
    if (prc != SA_OK) return prc;
    if (n_jobs == 0) return SA_OK;
    if (!d_jobs || !d_reads || !d_out) return err(SA_EINVAL, "NULL job, read or result buffer");
    const sa::RefView V = sa::ref_view(R);
    CK(cudaSetDevice(V.device));
    unsigned char* base = nullptr;
    const int rc = scratch_address(V.device, &base);
    if (rc != SA_OK) return rc;
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : V.own;

    // fixed part of the layout (known before the read lengths are)
    const size_t off_key = up256(sizeof(Ctl));
    const size_t off_order = up256(off_key + (size_t)n_jobs * 2);
    const size_t off_state = up256(off_order + (size_t)n_jobs * 4);
    const size_t off_rpack = up256(off_state + (size_t)n_jobs * sizeof(sa::JobState));
    if (off_rpack > kScratchBytes)
        return err(SA_EINVAL, "%u jobs need more than the %zu-byte no-alloc scratch; split the batch",
                   n_jobs, kScratchBytes);

    // clear the control block: statistics, error markers, work counter, histogram
    Ctl* ctl = reinterpret_cast<Ctl*>(base);
    CK(cudaMemsetAsync(ctl, 0, sizeof(Ctl), st));
    CK(cudaMemsetAsync(&ctl->st.bad_job, 0xff, 2 * sizeof(uint32_t), st));
    CK(cudaMemsetAsync(&ctl->st.dbg_site, 0xff, sizeof(uint32_t), st));
    sa::launch_plan(d_jobs, n_jobs, reads_len, (int64_t)V.len, nullptr,
                    reinterpret_cast<uint16_t*>(base + off_key), ctl->hist, &ctl->st, st);
    CK(cudaGetLastError());
    sa::PlanStats hs;
    CK(cudaMemcpyAsync(&hs, &ctl->st, sizeof(hs), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (hs.bad_job != 0xffffffffu)
        return err(SA_EINVAL, "job %u is invalid (read length 1..%u, window 1..%u inside the reference, "
                   "read inside the reads buffer)", hs.bad_job, SA_MAX_READ, SA_MAX_WINDOW);

    // the rest of the layout: packed reads, then column-maximum slots
    const uint32_t rw = (hs.max_n + 15) / 16;
    const size_t off_cb = up256(off_rpack + (size_t)n_jobs * rw * 4);
    const int c = sa::cfg_for_rows((int)hs.max_n);
    const int L = sa::cfg_L(c);
    const int G = 32 / L;
    const size_t slot = (size_t)sa::cb_words(hs.max_m) * 4;
    const size_t block_slots = 4 * (size_t)G;        // 128-thread blocks: 4 warps x G groups
    if (off_cb > kScratchBytes || (kScratchBytes - off_cb) / slot < block_slots)
        return err(SA_EINVAL, "this batch needs about %zu bytes of scratch, more than the %zu-byte "
                   "no-alloc scratch; split the batch", off_cb + block_slots * slot, kScratchBytes);
    const size_t blocks_fit = (kScratchBytes - off_cb) / slot / block_slots;

    sa::launch_iota(reinterpret_cast<uint32_t*>(base + off_order), n_jobs, st);
    sa::launch_pack_reads(d_jobs, n_jobs, reinterpret_cast<const uint8_t*>(d_reads),
                          reinterpret_cast<uint32_t*>(base + off_rpack), rw, &ctl->st.bad_read, st);
    CK(cudaGetLastError());

    sa::FillLaunch fl{};
    sa::FillArgs& A = fl.args;
    A.ref = V.d_words;
    A.ref_len = (int64_t)V.len;
    A.jobs = d_jobs;
    A.rpack = reinterpret_cast<const uint32_t*>(base + off_rpack);
    A.rw = rw;
    A.order = reinterpret_cast<const uint32_t*>(base + off_order);
    A.pos_begin = 0;
    A.pos_count = n_jobs;
    A.item_counter = &ctl->item_counter;
    A.sc = sc;
    A.state = reinterpret_cast<sa::JobState*>(base + off_state);
    A.colbest = reinterpret_cast<int32_t*>(base + off_cb);
    A.cb_stride = sa::cb_words(hs.max_m);
    A.n_state = n_jobs;
    A.cb_cap = (kScratchBytes - off_cb) / 4;
    A.dbg = &ctl->st.dbg_site;
    fl.kind = sa::kFillScore;
    fl.block = 128;
    int bps = sa::fill_max_blocks_per_sm(c, sa::kFillScore, P->mode);
    if (bps < 1) bps = 1;
    const size_t warps_needed = ((size_t)n_jobs + G - 1) / G;
    size_t grid = (size_t)V.num_sms * bps;
    grid = std::min(grid, blocks_fit);
    grid = std::min(grid, (warps_needed + 3) / 4);
    fl.grid = (int)std::max<size_t>(grid, 1);
    fl.stream = st;
    sa::launch_fill_cfg(c, fl);
    CK(cudaGetLastError());

    uint32_t bad_read = 0, dbg_site = 0;
    CK(cudaMemcpyAsync(&bad_read, &ctl->st.bad_read, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&dbg_site, &ctl->st.dbg_site, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (bad_read != 0xffffffffu)
        return err(SA_EINVAL, "job %u: read has a base other than A, C, G, T", bad_read);
    if (dbg_site != 0xffffffffu)
        return err(SA_ECUDA, "internal error: a kernel store was out of range (store site %u)", dbg_site);
    k_noalloc_results<<<(n_jobs + 255) / 256, 256, 0, st>>>(
        d_jobs, n_jobs, reinterpret_cast<const sa::JobState*>(base + off_state), P->min_score, d_out);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    return SA_OK;
}

}  // namespace

extern "C" int sa_align_batch_noalloc(sa_reference* ref, const sa_params* params, const sa_job* d_jobs,
                                      uint32_t n_jobs, const char* d_reads, uint64_t reads_len,
                                      sa_result* d_out, void* cuda_stream) {
    try {
        sa::set_error(SA_OK, "");
        return run(ref, params, d_jobs, n_jobs, d_reads, reads_len, d_out, cuda_stream);
    } catch (...) {
        return err(SA_ECUDA, "unexpected host exception");
    }
}
