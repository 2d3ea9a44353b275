// Read-level steps after the alignment of each read's candidate windows:
// sa_effort_limit[_dev] and sa_select[_dev].
//
// The paper aligns a read against several candidate regions (Methods,
// "Effort limit for dynamic programming": candidates ranked by their number of
// supporting seeds, only the best `ceiling` of them aligned) and reports
// paired-end reads as properly paired when their orientation and fragment
// length match the user's expectations, else each end on its own (Methods,
// "Paired-end alignment"), with a mapping quality from the best and the
// second-best hit (Experiments: compatible with BWA's).
//
// Both steps work one warp per read (or per pair): a read's candidates are a
// contiguous range of the batch, read_first[r] .. read_first[r+1]-1, so a warp
// reads them with coalesced loads and reduces with shuffles.
//
// Effort limit: candidates rank by support, then by input order.  The warp
// finds the ceiling-th largest support of the read bit by bit from the top (a
// radix select: keep a bit when at least `ceiling` supports reach the prefix
// with it set), keeps every candidate above it and the earliest ones equal to
// it up to `ceiling` in all, compacted in input order with ballots.
//
// Selection: the best aligned candidate (score, then smallest reference end,
// then earliest job); the second best is the highest hit of the read (every
// aligned candidate's best and its own second) whose reference end lies at
// least n from the chosen one's; MAPQ 60 without a second hit, 0 when it ties,
// else 20 per (match + mismatch) score units of the gap, at most 60.  Paired:
// lanes take the (end 1, end 2) candidate combinations; the proper one with the
// highest summed score wins (ties: earlier end-1 job, then earlier end-2 job;
// lanes hold end-2 candidates in registers and end-1 ones are broadcast);
// the pair's second best is the best proper combination that moves at least
// one end by its read length or more.
#include <algorithm>
#include <cstdarg>
#include <cstdio>

#include "kernels.h"

namespace {

int err(int code, const char* fmt, ...) {
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    return sa::set_error(code, msg);
}

#define SCU(expr)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            cudaGetLastError();                                                             \
            return err(e_ == cudaErrorMemoryAllocation ? SA_ENOMEM : SA_ECUDA, "%s failed: %s", \
                       #expr, cudaGetErrorString(e_));                                      \
        }                                                                                   \
    } while (0)

constexpr int kWarps = 4;                   // warps per block

// ---------------------------------------------------------------------------
// effort limit

__global__ void k_effort_count(const uint32_t* __restrict__ read_first, uint32_t n_reads, uint32_t ceiling,
                               uint32_t* __restrict__ count, unsigned* bad) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_reads) return;
    const uint32_t lo = read_first[r], hi = read_first[r + 1];
    if (hi < lo || (r == 0 && lo != 0)) {
        atomicMin(bad, r);
        count[r] = 0;
        return;
    }
    count[r] = min(hi - lo, ceiling);
}

__global__ void __launch_bounds__(32 * kWarps)
k_effort_select(const sa_job* __restrict__ jobs, const uint32_t* __restrict__ support,
                const uint32_t* __restrict__ read_first, uint32_t n_reads, uint32_t ceiling,
                const uint64_t* __restrict__ kept_off, sa_job* __restrict__ kept,
                uint32_t* __restrict__ kept_from, uint32_t* __restrict__ kept_first) {
    const uint32_t r = blockIdx.x * kWarps + threadIdx.x / 32;
    const uint32_t lane = threadIdx.x & 31u;
    if (r >= n_reads) return;
    const uint32_t lo = read_first[r], hi = read_first[r + 1];
    const uint32_t L = hi >= lo ? hi - lo : 0u;
    const uint64_t base = kept_off[r];
    if (lane == 0) {
        kept_first[r] = (uint32_t)base;
        if (r == n_reads - 1) kept_first[n_reads] = (uint32_t)(base + min(L, ceiling));
    }
    if (L <= ceiling) {
        for (uint32_t c = lane; c < L; c += 32) {
            kept[base + c] = jobs[lo + c];
            kept_from[base + c] = lo + c;
        }
        return;
    }
    // radix select of the ceiling-th largest support (thr); of the candidates
    // with support thr the earliest `quota` are kept
    const bool regs = L <= 64;                           // supports held in two registers
    const uint32_t s0 = (regs && lane < L) ? __ldg(support + lo + lane) : 0u;
    const uint32_t s1 = (regs && 32 + lane < L) ? __ldg(support + lo + 32 + lane) : 0u;
    auto count_ge = [&](uint32_t x) -> uint32_t {        // candidates with support >= x
        uint32_t n = 0;
        if (regs) {
            n = (lane < L && s0 >= x ? 1u : 0u) + (32 + lane < L && s1 >= x ? 1u : 0u);
        } else {
            for (uint32_t c = lane; c < L; c += 32) n += __ldg(support + lo + c) >= x ? 1u : 0u;
        }
        return __reduce_add_sync(0xffffffffu, n);
    };
    uint32_t thr = 0;
    for (int bit = 31; bit >= 0; bit--) {
        const uint32_t cand = thr | (1u << bit);
        if (count_ge(cand) >= ceiling) thr = cand;
    }
    const uint32_t above = thr == 0xffffffffu ? 0u : count_ge(thr + 1u);
    const uint32_t quota = ceiling - above;              // >= 1 candidates with support thr
    // keep support > thr, and the first `quota` with support == thr, in input order
    uint32_t written = 0, eq_seen = 0;
    for (uint32_t c0 = 0; c0 < L; c0 += 32) {
        const uint32_t c = c0 + lane;
        const uint32_t sv = c < L ? (regs ? (c0 == 0 ? s0 : s1) : __ldg(support + lo + c)) : 0u;
        const bool eq = c < L && sv == thr;
        const unsigned me = __ballot_sync(0xffffffffu, eq);
        const uint32_t eq_before = eq_seen + (uint32_t)__popc(me & ((1u << lane) - 1u));
        const bool keep = c < L && (sv > thr || (eq && eq_before < quota));
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const uint64_t at = base + written + (uint32_t)__popc(m & ((1u << lane) - 1u));
            kept[at] = jobs[lo + c];
            kept_from[at] = lo + c;
        }
        written += (uint32_t)__popc(m);
        eq_seen += (uint32_t)__popc(me);
    }
}

// ---------------------------------------------------------------------------
// selection

struct Cand {                      // what the selection reads of one candidate
    int32_t score;
    bool ok;                       // aligned: neither empty nor below min_score
    bool rc;
    int64_t end, begin;
    int32_t second;
    int64_t second_end;
    int32_t n;
};

__device__ __forceinline__ Cand load_cand(const sa_job* jobs, const sa_result* res, uint32_t j) {
    Cand c;
    const sa_result& R = res[j];
    c.score = R.score;
    c.ok = (R.flags & (SA_RES_EMPTY | SA_RES_BELOW_MIN)) == 0u;
    c.rc = (jobs[j].flags & SA_RC) != 0u;
    c.n = (int32_t)jobs[j].read_len;
    c.end = R.ref_end;
    c.begin = R.ref_begin >= 0 ? R.ref_begin : R.ref_end - c.n;   // no traceback: ungapped span
    c.second = R.second;
    c.second_end = R.second_ref_end;
    return c;
}

__device__ __forceinline__ int32_t mapq_of(int32_t best, int32_t second, int32_t a, int32_t b) {
    if (second == SA_NO_SCORE) return SA_MAPQ_MAX;
    const int64_t d = (int64_t)best - second;
    if (d <= 0) return 0;
    if (a + b <= 0) return SA_MAPQ_MAX;
    const int64_t q = (20 * d) / (a + b);
    return q < SA_MAPQ_MAX ? (int32_t)q : SA_MAPQ_MAX;
}

__device__ __forceinline__ int64_t dist(int64_t x, int64_t y) { return x > y ? x - y : y - x; }

// best aligned candidate of [lo, hi): (score desc, end asc, job asc); job kNoJob if none
struct Best {
    int32_t score;
    int64_t end;
    uint32_t job;
};

__device__ __forceinline__ bool better(const Best& x, const Best& y) {   // x ranks above y
    if (x.job == SA_NO_JOB) return false;
    if (y.job == SA_NO_JOB) return true;
    if (x.score != y.score) return x.score > y.score;
    if (x.end != y.end) return x.end < y.end;
    return x.job < y.job;
}

__device__ Best warp_best(const sa_job* jobs, const sa_result* res, uint32_t lo, uint32_t hi, uint32_t lane) {
    Best b{0, 0, SA_NO_JOB};
    for (uint32_t j = lo + lane; j < hi; j += 32) {
        const sa_result& R = res[j];
        if (R.flags & (SA_RES_EMPTY | SA_RES_BELOW_MIN)) continue;
        const Best c{R.score, R.ref_end, j};
        if (better(c, b)) b = c;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Best t;
        t.score = __shfl_xor_sync(0xffffffffu, b.score, o);
        t.end = __shfl_xor_sync(0xffffffffu, b.end, o);
        t.job = __shfl_xor_sync(0xffffffffu, b.job, o);
        if (better(t, b)) b = t;
    }
    return b;
}

// highest hit of [lo, hi) whose reference end is at least n from `end`
__device__ int32_t warp_second(const sa_result* res, uint32_t lo, uint32_t hi, int64_t end, int64_t n,
                               uint32_t lane) {
    int32_t s = SA_NO_SCORE;
    for (uint32_t j = lo + lane; j < hi; j += 32) {
        const sa_result& R = res[j];
        if (R.flags & (SA_RES_EMPTY | SA_RES_BELOW_MIN)) continue;
        if (dist(R.ref_end, end) >= n) s = max(s, R.score);
        if (R.second != SA_NO_SCORE && dist(R.second_ref_end, end) >= n) s = max(s, R.second);
    }
    return __reduce_max_sync(0xffffffffu, s);
}

struct SelArgs {
    const sa_job* jobs;
    const sa_result* res;
    const uint32_t* read_first;
    uint32_t n_reads;
    int32_t a, b;
    int32_t paired, orientation;
    int64_t frag_min, frag_max;
    sa_read_result* out;
};

__device__ void write_single(const SelArgs& A, uint32_t r, uint32_t lo, uint32_t hi, const Best& bst,
                             int32_t second, uint32_t extra, uint32_t lane) {
    if (lane) return;
    sa_read_result o;
    o.n_cand = hi - lo;
    o.frag_len = 0;
    if (bst.job == SA_NO_JOB) {
        o.job = SA_NO_JOB;
        o.score = 0;
        o.second = SA_NO_SCORE;
        o.mapq = 0;
        o.flags = extra & ~(uint32_t)SA_READ_ALIGNED;
    } else {
        o.job = bst.job;
        o.score = bst.score;
        o.second = second;
        o.mapq = mapq_of(bst.score, second, A.a, A.b);
        o.flags = extra | SA_READ_ALIGNED | ((A.jobs[bst.job].flags & SA_RC) ? SA_READ_REVERSE : 0u);
    }
    A.out[r] = o;
}

// fragment length of (j1 end 1, j2 end 2) if properly paired, else -1
__device__ __forceinline__ int64_t frag_of(const Cand& c1, const Cand& c2, int orientation,
                                           int64_t fmin, int64_t fmax) {
    int64_t frag;
    if (orientation == SA_PAIR_FR) {
        if (c1.rc == c2.rc) return -1;
        const Cand& f = c1.rc ? c2 : c1;
        const Cand& r = c1.rc ? c1 : c2;
        frag = r.end - f.begin;
    } else {
        if (c1.rc != c2.rc) return -1;
        const Cand& first = c1.rc ? c2 : c1;
        const Cand& last = c1.rc ? c1 : c2;
        frag = last.end - first.begin;
    }
    return (frag >= fmin && frag <= fmax) ? frag : -1;
}

// Every (end-1 a, end-2 b) combination of aligned candidates, k = a * L2 + b:
// lane t holds end-2 candidate b0 + t of the current chunk in registers and
// end-1 candidate a0 + t of the current chunk; the aligned ones of the end-1
// chunk are broadcast to the whole warp one at a time (no memory access per
// combination; unaligned candidates, e.g. below min_score, cost nothing).
template <typename F>
__device__ __forceinline__ void for_each_combo(const sa_job* jobs, const sa_result* res, uint32_t lo1,
                                               uint32_t L1, uint32_t lo2, uint32_t L2, uint32_t lane, F&& f) {
    for (uint32_t b0 = 0; b0 < L2; b0 += 32) {
        const uint32_t b = b0 + lane;
        Cand cb = {};
        if (b < L2) cb = load_cand(jobs, res, lo2 + b);
        if (!__any_sync(0xffffffffu, cb.ok)) continue;
        for (uint32_t a0 = 0; a0 < L1; a0 += 32) {
            Cand mine = {};
            if (a0 + lane < L1) mine = load_cand(jobs, res, lo1 + a0 + lane);
            // only the aligned end-1 candidates of the chunk are broadcast
            for (unsigned live = __ballot_sync(0xffffffffu, mine.ok); live; live &= live - 1u) {
                const int t = __ffs(live) - 1;
                Cand ca;
                ca.ok = true;
                const int rcn = __shfl_sync(0xffffffffu, (mine.n << 1) | (int)mine.rc, t);
                ca.rc = (rcn & 1) != 0;
                ca.n = rcn >> 1;
                ca.score = __shfl_sync(0xffffffffu, mine.score, t);
                ca.end = __shfl_sync(0xffffffffu, mine.end, t);
                ca.begin = __shfl_sync(0xffffffffu, mine.begin, t);
                if (cb.ok) f(ca, cb, (uint64_t)(a0 + (uint32_t)t) * L2 + b);
            }
        }
    }
}

__global__ void __launch_bounds__(32 * kWarps) k_select(SelArgs A) {
    const uint32_t unit = blockIdx.x * kWarps + threadIdx.x / 32;
    const uint32_t lane = threadIdx.x & 31u;
    if (!A.paired) {
        if (unit >= A.n_reads) return;
        const uint32_t lo = A.read_first[unit], hi = A.read_first[unit + 1];
        const Best b = warp_best(A.jobs, A.res, lo, hi, lane);
        const int32_t s = b.job == SA_NO_JOB ? SA_NO_SCORE
                        : warp_second(A.res, lo, hi, b.end, (int64_t)A.jobs[b.job].read_len, lane);
        write_single(A, unit, lo, hi, b, s, 0u, lane);
        return;
    }
    if (unit >= A.n_reads / 2) return;
    const uint32_t r1 = 2 * unit, r2 = r1 + 1;
    const uint32_t lo1 = A.read_first[r1], hi1 = A.read_first[r1 + 1];
    const uint32_t lo2 = hi1, hi2 = A.read_first[r2 + 1];
    const Best b1 = warp_best(A.jobs, A.res, lo1, hi1, lane);
    const Best b2 = warp_best(A.jobs, A.res, lo2, hi2, lane);
    // proper combinations: lanes over k = a * L2 + b (a end-1 index, b end-2 index)
    const uint32_t L1 = hi1 - lo1, L2 = hi2 - lo2;
    const uint64_t combos = (b1.job != SA_NO_JOB && b2.job != SA_NO_JOB) ? (uint64_t)L1 * L2 : 0ull;
    int32_t best_sum = INT32_MIN;
    uint64_t best_k = UINT64_MAX;
    int64_t best_frag = 0;
    if (combos)
        for_each_combo(A.jobs, A.res, lo1, L1, lo2, L2, lane, [&](const Cand& c1, const Cand& c2, uint64_t k) {
            const int64_t fr = frag_of(c1, c2, A.orientation, A.frag_min, A.frag_max);
            if (fr < 0) return;
            const int32_t sum = c1.score + c2.score;
            if (sum > best_sum || (sum == best_sum && k < best_k)) { best_sum = sum; best_k = k; best_frag = fr; }
        });
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int32_t ts = __shfl_xor_sync(0xffffffffu, best_sum, o);
        const uint64_t tk = __shfl_xor_sync(0xffffffffu, best_k, o);
        const int64_t tf = __shfl_xor_sync(0xffffffffu, best_frag, o);
        if (tk != UINT64_MAX && (ts > best_sum || (ts == best_sum && tk < best_k))) {
            best_sum = ts; best_k = tk; best_frag = tf;
        }
    }
    if (best_k == UINT64_MAX) {
        // no proper pair: each end on its own
        const int32_t s1 = b1.job == SA_NO_JOB ? SA_NO_SCORE
                         : warp_second(A.res, lo1, hi1, b1.end, (int64_t)A.jobs[b1.job].read_len, lane);
        const int32_t s2 = b2.job == SA_NO_JOB ? SA_NO_SCORE
                         : warp_second(A.res, lo2, hi2, b2.end, (int64_t)A.jobs[b2.job].read_len, lane);
        const uint32_t m1 = b2.job != SA_NO_JOB ? (uint32_t)SA_READ_MATE_ALIGNED : 0u;
        const uint32_t m2 = b1.job != SA_NO_JOB ? (uint32_t)SA_READ_MATE_ALIGNED : 0u;
        write_single(A, r1, lo1, hi1, b1, s1, SA_READ_PAIRED | m1, lane);
        write_single(A, r2, lo2, hi2, b2, s2, SA_READ_PAIRED | m2, lane);
        return;
    }
    const uint32_t c1j = lo1 + (uint32_t)(best_k / L2), c2j = lo2 + (uint32_t)(best_k % L2);
    const Cand c1 = load_cand(A.jobs, A.res, c1j), c2 = load_cand(A.jobs, A.res, c2j);
    // the pair's second best: a proper combination moving an end by its read length or more
    int32_t pair_second = SA_NO_SCORE;
    for_each_combo(A.jobs, A.res, lo1, L1, lo2, L2, lane, [&](const Cand& d1, const Cand& d2, uint64_t) {
        if (dist(d1.end, c1.end) < c1.n && dist(d2.end, c2.end) < c2.n) return;
        if (frag_of(d1, d2, A.orientation, A.frag_min, A.frag_max) < 0) return;
        pair_second = max(pair_second, d1.score + d2.score);
    });
    pair_second = __reduce_max_sync(0xffffffffu, pair_second);
    const int32_t pair_mapq = mapq_of(best_sum, pair_second, A.a, A.b);
    const int32_t s1 = warp_second(A.res, lo1, hi1, c1.end, c1.n, lane);
    const int32_t s2 = warp_second(A.res, lo2, hi2, c2.end, c2.n, lane);
    if (lane == 0) {
        const uint32_t both = SA_READ_ALIGNED | SA_READ_PAIRED | SA_READ_PROPER | SA_READ_MATE_ALIGNED;
        sa_read_result o;
        o.job = c1j;
        o.score = c1.score;
        o.second = s1;
        o.mapq = max(pair_mapq, mapq_of(c1.score, s1, A.a, A.b));
        o.flags = both | (c1.rc ? (uint32_t)SA_READ_REVERSE : 0u);
        o.n_cand = L1;
        o.frag_len = best_frag;
        A.out[r1] = o;
        o.job = c2j;
        o.score = c2.score;
        o.second = s2;
        o.mapq = max(pair_mapq, mapq_of(c2.score, s2, A.a, A.b));
        o.flags = both | (c2.rc ? (uint32_t)SA_READ_REVERSE : 0u);
        o.n_cand = L2;
        A.out[r2] = o;
    }
}

__global__ void k_check_first(const uint32_t* __restrict__ read_first, uint32_t n_reads, unsigned* bad) {
    const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_reads) return;
    if (read_first[r + 1] < read_first[r] || (r == 0 && read_first[0] != 0)) atomicMin(bad, r);
}

cudaStream_t stream_of(const sa::RefView& V, void* s) {
    return s ? static_cast<cudaStream_t>(s) : V.own;
}

int check_select_params(const sa_select_params* sp, uint32_t n_reads) {
    if (!sp) return err(SA_EINVAL, "select params is NULL");
    if (sp->sc.match < 0 || sp->sc.mismatch < 0) return err(SA_EINVAL, "scores are magnitudes and must be >= 0");
    if (sp->paired != 0 && sp->paired != 1) return err(SA_EINVAL, "paired must be 0 or 1");
    if (sp->paired && (n_reads & 1u)) return err(SA_EINVAL, "paired selection needs an even number of reads");
    if (sp->orientation != SA_PAIR_FR && sp->orientation != SA_PAIR_FF)
        return err(SA_EINVAL, "orientation must be SA_PAIR_FR or SA_PAIR_FF");
    if (sp->paired && (sp->frag_min < 0 || sp->frag_min > sp->frag_max))
        return err(SA_EINVAL, "fragment range must satisfy 0 <= frag_min <= frag_max");
    return SA_OK;
}

int effort_limit_dev(const sa::RefView& V, const sa_job* d_jobs, const uint32_t* d_support,
                     const uint32_t* d_read_first, uint32_t n_reads, uint32_t ceiling, sa_job* d_kept,
                     uint32_t* d_kept_from, uint32_t* d_kept_first, uint32_t* n_kept, cudaStream_t st) {
    if (ceiling == 0) return err(SA_EINVAL, "ceiling must be >= 1");
    if (n_reads && (!d_jobs || !d_support || !d_read_first || !d_kept || !d_kept_from || !d_kept_first))
        return err(SA_EINVAL, "NULL buffer");
    if (n_reads == 0) {
        if (d_kept_first) SCU(cudaMemsetAsync(d_kept_first, 0, 4, st));
        if (n_kept) *n_kept = 0;
        return SA_OK;
    }
    // scratch: counts, their scan, block sums, the bad-read flag
    const uint64_t nb = sa::scan_bsum_len(n_reads);
    const size_t bytes = (size_t)n_reads * 4 + ((size_t)n_reads + 1) * 8 + nb * 8 + 8 + 16;
    void* tmp = nullptr;
    SCU(cudaMallocAsync(&tmp, bytes, st));
    uint64_t* offs = static_cast<uint64_t*>(tmp);
    uint64_t* bsum = offs + (n_reads + 1);
    uint64_t* total = bsum + nb;
    unsigned* bad = reinterpret_cast<unsigned*>(total + 1);
    uint32_t* count = bad + 4;
    cudaError_t e = cudaMemsetAsync(bad, 0xff, 4, st);
    if (e == cudaSuccess) {
        k_effort_count<<<(n_reads + 255) / 256, 256, 0, st>>>(d_read_first, n_reads, ceiling, count, bad);
        sa::launch_scan_u32(count, n_reads, offs, bsum, total, st);
        k_effort_select<<<(n_reads + kWarps - 1) / kWarps, 32 * kWarps, 0, st>>>(
            d_jobs, d_support, d_read_first, n_reads, ceiling, offs, d_kept, d_kept_from, d_kept_first);
        e = cudaGetLastError();
    }
    unsigned h_bad = 0xffffffffu;
    uint64_t h_total = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, bad, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_total, total, 8, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(tmp, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    SCU(e);
    if (h_bad != 0xffffffffu)
        return err(SA_EINVAL, "read_first is not an ascending offset array from 0 (read %u)", h_bad);
    if (n_kept) *n_kept = (uint32_t)h_total;
    return SA_OK;
}

int select_dev(const sa::RefView& V, const sa_select_params* sp, const sa_job* d_jobs,
               const sa_result* d_res, const uint32_t* d_read_first, uint32_t n_reads,
               sa_read_result* d_out, cudaStream_t st) {
    if (int rc = check_select_params(sp, n_reads)) return rc;
    if (n_reads == 0) return SA_OK;
    if (!d_read_first || !d_out) return err(SA_EINVAL, "NULL buffer");
    unsigned* bad = nullptr;
    SCU(cudaMallocAsync((void**)&bad, 4, st));
    cudaError_t e = cudaMemsetAsync(bad, 0xff, 4, st);
    if (e == cudaSuccess) {
        k_check_first<<<(n_reads + 255) / 256, 256, 0, st>>>(d_read_first, n_reads, bad);
        SelArgs A;
        A.jobs = d_jobs;
        A.res = d_res;
        A.read_first = d_read_first;
        A.n_reads = n_reads;
        A.a = sp->sc.match;
        A.b = sp->sc.mismatch;
        A.paired = sp->paired;
        A.orientation = sp->orientation;
        A.frag_min = sp->frag_min;
        A.frag_max = sp->frag_max;
        A.out = d_out;
        const uint32_t units = sp->paired ? n_reads / 2 : n_reads;
        k_select<<<(units + kWarps - 1) / kWarps, 32 * kWarps, 0, st>>>(A);
        e = cudaGetLastError();
    }
    unsigned h_bad = 0xffffffffu;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, bad, 4, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(bad, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    SCU(e);
    if (h_bad != 0xffffffffu)
        return err(SA_EINVAL, "read_first is not an ascending offset array from 0 (read %u)", h_bad);
    return SA_OK;
}

// host-buffer forms: copy in, run the device form, copy out
template <typename T>
struct DevArr {
    T* p = nullptr;
    cudaStream_t st = nullptr;
    ~DevArr() { if (p) cudaFreeAsync(p, st); }
    cudaError_t get(size_t n, cudaStream_t s) {
        st = s;
        return cudaMallocAsync((void**)&p, std::max<size_t>(n, 1) * sizeof(T), s);
    }
};

bool ascending_from_zero(const uint32_t* first, uint32_t n_reads) {
    if (first[0] != 0) return false;
    for (uint32_t r = 0; r < n_reads; r++)
        if (first[r + 1] < first[r]) return false;
    return true;
}

}  // namespace

extern "C" int sa_effort_limit_dev(sa_reference* ref, const sa_job* jobs, const uint32_t* support,
                                   const uint32_t* read_first, uint32_t n_reads, uint32_t ceiling,
                                   sa_job* kept, uint32_t* kept_from, uint32_t* kept_first,
                                   uint32_t* n_kept, void* stream) {
    try {
        sa::set_error(SA_OK, "");
        if (!ref) return err(SA_EINVAL, "reference is NULL");
        const sa::RefView V = sa::ref_view(ref);
        SCU(cudaSetDevice(V.device));
        return effort_limit_dev(V, jobs, support, read_first, n_reads, ceiling, kept, kept_from, kept_first,
                                n_kept, stream_of(V, stream));
    } catch (...) {
        return err(SA_ENOMEM, "unexpected host exception");
    }
}

extern "C" int sa_effort_limit(sa_reference* ref, const sa_job* jobs, const uint32_t* support,
                               const uint32_t* read_first, uint32_t n_reads, uint32_t ceiling,
                               sa_job* kept, uint32_t* kept_from, uint32_t* kept_first, uint32_t* n_kept) {
    try {
        sa::set_error(SA_OK, "");
        if (!ref) return err(SA_EINVAL, "reference is NULL");
        if (n_reads && (!read_first || !jobs || !support || !kept || !kept_from || !kept_first))
            return err(SA_EINVAL, "NULL buffer");
        if (n_reads && !ascending_from_zero(read_first, n_reads))
            return err(SA_EINVAL, "read_first is not an ascending offset array from 0");
        const sa::RefView V = sa::ref_view(ref);
        SCU(cudaSetDevice(V.device));
        const cudaStream_t st = V.own;
        const uint32_t n_jobs = n_reads ? read_first[n_reads] : 0u;
        DevArr<sa_job> dj, dk;
        DevArr<uint32_t> ds, df, dfrom, dkf;
        SCU(dj.get(n_jobs, st));
        SCU(dk.get(n_jobs, st));
        SCU(ds.get(n_jobs, st));
        SCU(df.get((size_t)n_reads + 1, st));
        SCU(dfrom.get(n_jobs, st));
        SCU(dkf.get((size_t)n_reads + 1, st));
        if (n_jobs) {
            SCU(cudaMemcpyAsync(dj.p, jobs, (size_t)n_jobs * sizeof(sa_job), cudaMemcpyHostToDevice, st));
            SCU(cudaMemcpyAsync(ds.p, support, (size_t)n_jobs * 4, cudaMemcpyHostToDevice, st));
        }
        SCU(cudaMemcpyAsync(df.p, read_first, ((size_t)n_reads + 1) * 4, cudaMemcpyHostToDevice, st));
        uint32_t nk = 0;
        const int rc = effort_limit_dev(V, dj.p, ds.p, df.p, n_reads, ceiling, dk.p, dfrom.p, dkf.p, &nk, st);
        if (rc != SA_OK) return rc;
        if (nk) {
            SCU(cudaMemcpyAsync(kept, dk.p, (size_t)nk * sizeof(sa_job), cudaMemcpyDeviceToHost, st));
            SCU(cudaMemcpyAsync(kept_from, dfrom.p, (size_t)nk * 4, cudaMemcpyDeviceToHost, st));
        }
        if (n_reads) SCU(cudaMemcpyAsync(kept_first, dkf.p, ((size_t)n_reads + 1) * 4, cudaMemcpyDeviceToHost, st));
        SCU(cudaStreamSynchronize(st));
        if (n_kept) *n_kept = nk;
        return SA_OK;
    } catch (...) {
        return err(SA_ENOMEM, "unexpected host exception");
    }
}

extern "C" int sa_select_dev(sa_reference* ref, const sa_select_params* sp, const sa_job* jobs,
                             const sa_result* results, const uint32_t* read_first, uint32_t n_reads,
                             sa_read_result* out, void* stream) {
    try {
        sa::set_error(SA_OK, "");
        if (!ref) return err(SA_EINVAL, "reference is NULL");
        const sa::RefView V = sa::ref_view(ref);
        SCU(cudaSetDevice(V.device));
        return select_dev(V, sp, jobs, results, read_first, n_reads, out, stream_of(V, stream));
    } catch (...) {
        return err(SA_ENOMEM, "unexpected host exception");
    }
}

extern "C" int sa_select(sa_reference* ref, const sa_select_params* sp, const sa_job* jobs,
                         const sa_result* results, const uint32_t* read_first, uint32_t n_reads,
                         sa_read_result* out) {
    try {
        sa::set_error(SA_OK, "");
        if (!ref) return err(SA_EINVAL, "reference is NULL");
        if (int rc = check_select_params(sp, n_reads)) return rc;
        if (n_reads == 0) return SA_OK;
        if (!read_first || !out) return err(SA_EINVAL, "NULL buffer");
        if (!ascending_from_zero(read_first, n_reads))
            return err(SA_EINVAL, "read_first is not an ascending offset array from 0");
        const uint32_t n_jobs = read_first[n_reads];
        if (n_jobs && (!jobs || !results)) return err(SA_EINVAL, "NULL buffer");
        const sa::RefView V = sa::ref_view(ref);
        SCU(cudaSetDevice(V.device));
        const cudaStream_t st = V.own;
        DevArr<sa_job> dj;
        DevArr<sa_result> dr;
        DevArr<uint32_t> df;
        DevArr<sa_read_result> dout;
        SCU(dj.get(n_jobs, st));
        SCU(dr.get(n_jobs, st));
        SCU(df.get((size_t)n_reads + 1, st));
        SCU(dout.get(n_reads, st));
        if (n_jobs) {
            SCU(cudaMemcpyAsync(dj.p, jobs, (size_t)n_jobs * sizeof(sa_job), cudaMemcpyHostToDevice, st));
            SCU(cudaMemcpyAsync(dr.p, results, (size_t)n_jobs * sizeof(sa_result), cudaMemcpyHostToDevice, st));
        }
        SCU(cudaMemcpyAsync(df.p, read_first, ((size_t)n_reads + 1) * 4, cudaMemcpyHostToDevice, st));
        const int rc = select_dev(V, sp, dj.p, dr.p, df.p, n_reads, dout.p, st);
        if (rc != SA_OK) return rc;
        SCU(cudaMemcpyAsync(out, dout.p, (size_t)n_reads * sizeof(sa_read_result), cudaMemcpyDeviceToHost, st));
        SCU(cudaStreamSynchronize(st));
        return SA_OK;
    } catch (...) {
        return err(SA_ENOMEM, "unexpected host exception");
    }
}
