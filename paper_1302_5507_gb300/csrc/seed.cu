// Seeding front end (the paper's step 3): candidate windows of whole reads.
//
// SOAP3-dp aligns reads with neither end placed by taking seeds (substrings of
// the read) at regular intervals along the read and its reverse complement,
// aligning them back to the reference with its GPU BWT index, and enumerating
// the candidate regions they point to, each scored by its number of supporting
// seeds (Methods, "Implementation details of SOAP3-dp", step 3; "Effort limit
// for dynamic programming").  The windows then go to the effort limit and the
// dynamic programming.
//
// Index (built once per reference, on the host, then resident on the device):
//  - the suffix array SA of the reference followed by a terminator smaller
//    than every base (rows = L + 1; row 0 is the empty suffix), ordered by the
//    first 32 bases of each suffix (exact for every pattern of up to 32
//    bases, which is all backward search and the lookup table below need);
//  - the BWT of that order in 64-byte chunks, as the paper lays its index out
//    so that all the data for one base step is one memory access: four 32-bit
//    counts of A, C, G, T before the chunk, then 192 two-bit BWT codes as two bit
//    planes (one match mask per 32 rows);
//  - a lookup table of the row interval of every 12-base pattern, which
//    replaces the first 12 steps of each backward search;
//  - the full suffix array for locating (4 bytes a row: the paper's index
//    samples it to save GPU memory; on a device with hundreds of GB the full
//    array locates each hit with one load instead of a walk).
//
// Per call: one thread per seed runs the backward search (a lookup-table read,
// then two rank queries of one 64-byte chunk each per remaining base), a scan
// turns the occurrence counts into hit slots, one thread per seed locates its
// hits (diagonal = position - offset in the strand's sequence), and each
// (read, strand) sorts its hits by diagonal and cuts them into regions where
// neighbouring diagonals differ by more than `join` (one thread for up to 32
// hits, a block with a shared-memory bitonic sort beyond).  A region's window
// spans its diagonals plus the read length plus `pad` on both sides; its
// support is the number of distinct seeds with a hit in it.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "kernels.h"
#include "seed_index.h"

namespace {

int err(int code, const char* fmt, ...) {
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    return sa::set_error(code, msg);
}

#define ECU(expr)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            cudaGetLastError();                                                             \
            return err(e_ == cudaErrorMemoryAllocation ? SA_ENOMEM : SA_ECUDA, "%s failed: %s", \
                       #expr, cudaGetErrorString(e_));                                      \
        }                                                                                   \
    } while (0)
#define ETRY(expr)                    \
    do {                              \
        int rc_ = (expr);             \
        if (rc_ != SA_OK) return rc_; \
    } while (0)

constexpr int kMaxSeedsPerStrand = 128;            // seeds of one strand (support bit mask)
constexpr uint32_t kMaxHitsPerStrand = 8192;       // hits one (read, strand) may have
constexpr uint32_t kSmallHits = 32;                // up to this many: one thread sorts them
constexpr int64_t kDiagBias = 1 << 20;             // diagonals (>= -1024) stored biased, non-negative

struct Buf {
    void* p = nullptr;
    size_t cap = 0;
    int ensure(size_t bytes, const char* what) {
        if (bytes <= cap && p) return SA_OK;
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        const size_t nb = std::max<size_t>(bytes + bytes / 8, 1 << 16);
        if (cudaMalloc(&p, nb) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return err(SA_ENOMEM, "cudaMalloc of %zu bytes for %s failed", nb, what);
        }
        cap = nb;
        return SA_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// validation and sizes of one call (device, mirrored to the host)
struct SeedStats {
    uint32_t max_n;
    uint32_t bad_read;        // first read out of range or with a base other than A/C/G/T
    uint32_t n_large;         // (read, strand) pairs with more than kSmallHits hits
    uint32_t _pad;
    uint64_t total[2];        // hits, candidates
};

struct TmpCand {              // one region, before compaction
    uint64_t ref_pos;
    uint32_t win_len;
    uint32_t support;
};

}  // namespace

struct sa_seed_index {
    int device = 0;
    uint64_t L = 0;               // reference bases
    uint32_t rows = 0;            // L + 1
    uint32_t dollar_row = 0;      // row of suffix 0 (its BWT entry is the terminator)
    uint32_t C[4] = {};           // rows before the first suffix starting with A, C, G, T
    uint32_t* d_sa = nullptr;     // rows
    uint4* d_occ = nullptr;       // 4 uint4 (64 bytes) per chunk
    uint2* d_lut = nullptr;       // [lo, hi) row interval of each 12-base pattern
    cudaStream_t own = nullptr;   // the reference's stream
    std::mutex mu;
    Buf stats, seeds, cnt, hoff, bsum, hits, large, tmp, ncand, coff;
    SeedStats* h_stats = nullptr;
};

namespace {

// ---------------------------------------------------------------------------
// device

__device__ __forceinline__ int base_code(uint8_t ch) {
    switch (ch | 0x20) {          // lower case
        case 'a': return 0;
        case 'c': return 1;
        case 'g': return 2;
        case 't': return 3;
        default: return -1;
    }
}

// rows r < i whose BWT entry is base c (the terminator's row never counts)
__device__ __forceinline__ uint32_t occ_rank(const uint4* __restrict__ occ, uint32_t i, uint32_t c,
                                             uint32_t dollar_row) {
    const uint32_t chunk = i / sa::kChunkRows, in = i - chunk * sa::kChunkRows;
    const uint4* q = occ + (size_t)chunk * 4;
    const uint4 h = __ldg(q), a = __ldg(q + 1), b = __ldg(q + 2), d = __ldg(q + 3);
    const uint32_t lo[6] = {a.x, a.y, a.z, a.w, b.x, b.y};      // low bit of each row's entry
    const uint32_t hi[6] = {b.z, b.w, d.x, d.y, d.z, d.w};      // high bit
    uint32_t r = c == 0 ? h.x : (c == 1 ? h.y : (c == 2 ? h.z : h.w));
    const uint32_t flip_lo = (c & 1u) ? 0u : ~0u, flip_hi = (c & 2u) ? 0u : ~0u;
#pragma unroll
    for (int k = 0; k < 6; k++) {
        const int first = 32 * k;
        if (first < (int)in) {
            uint32_t m = (lo[k] ^ flip_lo) & (hi[k] ^ flip_hi);      // rows of this word holding c
            const int left = (int)in - first;
            if (left < 32) m &= (1u << left) - 1u;
            r += __popc(m);
        }
    }
    if (c == 0 && dollar_row >= chunk * sa::kChunkRows && dollar_row < i) r--;
    return r;
}

struct SearchArgs {
    const uint8_t* reads;
    const uint64_t* read_off;
    const uint32_t* read_len;
    uint32_t n_reads;
    uint32_t S;                  // seed slots per strand
    int lam, step;
    uint32_t max_occ;
    const uint2* lut;
    const uint4* occ;
    uint32_t dollar_row;
    uint32_t C0, C1, C2, C3;
    uint2* seed;                 // per slot: (first row, occurrences kept)
    uint32_t* cnt;               // per slot: occurrences kept (for the scan)
};

__global__ void k_seed_validate(const uint8_t* __restrict__ reads, uint64_t reads_len,
                                const uint64_t* __restrict__ off, const uint32_t* __restrict__ len,
                                uint32_t n_reads, SeedStats* st) {
    const uint32_t r = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (r >= n_reads) return;
    const uint64_t o = off[r];
    const uint32_t n = len[r];
    bool bad = n == 0 || n > SA_MAX_READ || o > reads_len || reads_len - o < n;
    if (!bad)
        for (uint32_t t = lane; t < n; t += 32) bad |= base_code(reads[o + t]) < 0;
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
        if (bad) atomicMin(&st->bad_read, r);
        else atomicMax(&st->max_n, n);
    }
}

// one thread per seed slot: backward search of the seed's bases from its end
__global__ void k_seed_search(SearchArgs A) {
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (uint64_t)A.n_reads * 2 * A.S) return;
    const uint32_t r = (uint32_t)(g / (2ull * A.S));
    const uint32_t s = (uint32_t)(g / A.S) & 1u;
    const uint32_t k = (uint32_t)(g % A.S);
    const uint32_t n = A.read_len[r];
    const int o = (int)k * A.step;
    uint2 out = make_uint2(0, 0);
    if (o + A.lam <= (int)n) {
        const uint8_t* rd = A.reads + A.read_off[r];
        // base j of the seed: the read at o + j, or on the reverse strand the
        // complement of the read at n - 1 - (o + j)
        auto seed_base = [&](int j) -> uint32_t {
            const int c = s ? 3 - base_code(rd[n - 1 - (o + j)]) : base_code(rd[o + j]);
            return (uint32_t)c;
        };
        uint32_t P = 0;
        for (int j = A.lam - sa::kLutK; j < A.lam; j++) P = (P << 2) | seed_base(j);
        const uint2 iv = __ldg(A.lut + P);
        uint32_t lo = iv.x, hi = iv.y;
        for (int j = A.lam - sa::kLutK - 1; j >= 0 && lo < hi; j--) {
            const uint32_t c = seed_base(j);
            const uint32_t Cc = c == 0 ? A.C0 : (c == 1 ? A.C1 : (c == 2 ? A.C2 : A.C3));
            lo = Cc + occ_rank(A.occ, lo, c, A.dollar_row);
            hi = Cc + occ_rank(A.occ, hi, c, A.dollar_row);
        }
        const uint32_t found = hi > lo ? hi - lo : 0u;
        if (found && found <= A.max_occ) out = make_uint2(lo, found);
    }
    A.seed[g] = out;
    A.cnt[g] = out.y;
}

// one thread per seed slot: its hits, keyed (biased diagonal << 8 | seed index)
__global__ void k_seed_locate(const uint2* __restrict__ seed, const uint64_t* __restrict__ hoff, uint64_t n_slots,
                              uint32_t S, int step, const uint32_t* __restrict__ sa, uint64_t* __restrict__ hits) {
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_slots) return;
    const uint2 sd = seed[g];
    if (!sd.y) return;
    const uint32_t k = (uint32_t)(g % S);
    const int64_t o = (int64_t)k * step;
    uint64_t* dst = hits + hoff[g];
    for (uint32_t t = 0; t < sd.y; t++) {
        const int64_t d = (int64_t)__ldg(sa + sd.x + t) - o;
        dst[t] = ((uint64_t)(d + kDiagBias) << 8) | k;
    }
}

struct ClusterArgs {
    const uint64_t* hits;
    const uint64_t* hoff;         // per seed slot; (read, strand) rs owns slots rs*S .. rs*S+S-1
    uint64_t n_slots;
    uint32_t S;
    uint32_t n_rs;                // 2 * n_reads
    const uint32_t* read_len;
    int64_t L;
    int64_t pad, join;
    TmpCand* tmp;                 // per hit slot (a region never outnumbers its hits)
    uint32_t* ncand;              // regions per (read, strand)
    uint32_t* large;              // (read, strand) pairs with more than kSmallHits hits
    SeedStats* st;
};

__device__ __forceinline__ void hit_range(const ClusterArgs& A, uint32_t rs, uint64_t* b, uint64_t* e) {
    *b = A.hoff[(uint64_t)rs * A.S];
    *e = A.hoff[(uint64_t)rs * A.S + A.S];     // hoff has n_slots + 1 entries
}

__device__ __forceinline__ TmpCand make_region(const ClusterArgs& A, int64_t dmin, int64_t dmax, int n,
                                               uint32_t support) {
    int64_t start = dmin - A.pad;
    if (start < 0) start = 0;
    int64_t end = dmax + n + A.pad;
    if (end > A.L) end = A.L;
    if (end > start + (int64_t)SA_MAX_WINDOW) end = start + SA_MAX_WINDOW;
    TmpCand c;
    c.ref_pos = (uint64_t)start;
    c.win_len = (uint32_t)(end - start);
    c.support = support;
    return c;
}

// one thread per (read, strand) with at most kSmallHits hits: insertion sort,
// then the regions in diagonal order
__global__ void k_seed_cluster_small(ClusterArgs A) {
    const uint32_t rs = blockIdx.x * blockDim.x + threadIdx.x;
    if (rs >= A.n_rs) return;
    uint64_t b, e;
    hit_range(A, rs, &b, &e);
    const uint32_t h = (uint32_t)(e - b);
    if (h > kSmallHits) {
        A.large[atomicAdd(&A.st->n_large, 1u)] = rs;
        return;
    }
    uint64_t key[kSmallHits];
    for (uint32_t t = 0; t < h; t++) {
        const uint64_t v = A.hits[b + t];
        uint32_t q = t;
        while (q > 0 && key[q - 1] > v) {
            key[q] = key[q - 1];
            q--;
        }
        key[q] = v;
    }
    const int n = (int)A.read_len[rs >> 1];
    uint32_t nreg = 0;
    uint32_t t = 0;
    while (t < h) {
        uint32_t m[4] = {0, 0, 0, 0};
        const int64_t dmin = (int64_t)(key[t] >> 8) - kDiagBias;
        int64_t dlast = dmin;
        uint32_t u = t;
        for (; u < h; u++) {
            const int64_t d = (int64_t)(key[u] >> 8) - kDiagBias;
            if (u > t && d - dlast > A.join) break;
            const uint32_t sk = (uint32_t)(key[u] & 0xFFu);
            m[sk >> 5] |= 1u << (sk & 31);
            dlast = d;
        }
        const uint32_t sup = __popc(m[0]) + __popc(m[1]) + __popc(m[2]) + __popc(m[3]);
        A.tmp[b + nreg] = make_region(A, dmin, dlast, n, sup);
        nreg++;
        t = u;
    }
    A.ncand[rs] = nreg;
}

// one block per (read, strand) with more hits: bitonic sort in shared memory,
// region starts by a block scan, one thread per region
constexpr int kLargeThreads = 512;
__global__ void __launch_bounds__(kLargeThreads) k_seed_cluster_large(ClusterArgs A) {
    extern __shared__ __align__(16) uint64_t s_key[];           // kMaxHitsPerStrand
    __shared__ uint32_t s_scan[kLargeThreads];
    uint32_t* s_start = reinterpret_cast<uint32_t*>(s_key + kMaxHitsPerStrand);   // region starts
    const uint32_t rs = A.large[blockIdx.x];
    uint64_t b, e;
    hit_range(A, rs, &b, &e);
    const uint32_t h = (uint32_t)(e - b);
    uint32_t P = 1;
    while (P < h) P <<= 1;
    for (uint32_t t = threadIdx.x; t < P; t += blockDim.x) s_key[t] = t < h ? A.hits[b + t] : ~0ull;
    __syncthreads();
    for (uint32_t size = 2; size <= P; size <<= 1) {
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (uint32_t t = threadIdx.x; t < P / 2; t += blockDim.x) {
                const uint32_t i = 2 * t - (t & (stride - 1));      // lower index of the pair
                const uint32_t j = i + stride;
                const bool up = (i & size) == 0;
                const uint64_t x = s_key[i], y = s_key[j];
                if ((x > y) == up) {
                    s_key[i] = y;
                    s_key[j] = x;
                }
            }
            __syncthreads();
        }
    }
    // region starts: hits whose diagonal exceeds the previous one by more than join
    const uint32_t per = (h + blockDim.x - 1) / blockDim.x;     // consecutive hits per thread
    const uint32_t t0 = threadIdx.x * per, t1 = min(h, t0 + per);
    auto is_start = [&](uint32_t i) {
        return i == 0 || (int64_t)(s_key[i] >> 8) - (int64_t)(s_key[i - 1] >> 8) > A.join;
    };
    uint32_t mine = 0;
    for (uint32_t i = t0; i < t1; i++) mine += is_start(i) ? 1u : 0u;
    s_scan[threadIdx.x] = mine;
    __syncthreads();
    for (uint32_t o = 1; o < blockDim.x; o <<= 1) {
        const uint32_t v = threadIdx.x >= o ? s_scan[threadIdx.x - o] : 0u;
        __syncthreads();
        s_scan[threadIdx.x] += v;
        __syncthreads();
    }
    const uint32_t nreg = s_scan[blockDim.x - 1];
    uint32_t q = s_scan[threadIdx.x] - mine;
    for (uint32_t i = t0; i < t1; i++)
        if (is_start(i)) s_start[q++] = i;
    __syncthreads();
    const int n = (int)A.read_len[rs >> 1];
    for (uint32_t g = threadIdx.x; g < nreg; g += blockDim.x) {
        const uint32_t i0 = s_start[g], i1 = g + 1 < nreg ? s_start[g + 1] : h;
        uint32_t m[4] = {0, 0, 0, 0};
        for (uint32_t i = i0; i < i1; i++) {
            const uint32_t sk = (uint32_t)(s_key[i] & 0xFFu);
            m[sk >> 5] |= 1u << (sk & 31);
        }
        const uint32_t sup = __popc(m[0]) + __popc(m[1]) + __popc(m[2]) + __popc(m[3]);
        const int64_t dmin = (int64_t)(s_key[i0] >> 8) - kDiagBias;
        const int64_t dmax = (int64_t)(s_key[i1 - 1] >> 8) - kDiagBias;
        A.tmp[b + g] = make_region(A, dmin, dmax, n, sup);
    }
    if (threadIdx.x == 0) A.ncand[rs] = nreg;
}

// one thread per (read, strand): its regions to the caller's arrays (forward
// strand first, each in diagonal order)
__global__ void k_seed_emit(const TmpCand* __restrict__ tmp, const uint64_t* __restrict__ hoff, uint32_t S,
                            const uint32_t* __restrict__ ncand, const uint64_t* __restrict__ coff, uint32_t n_rs,
                            const uint64_t* __restrict__ read_off, const uint32_t* __restrict__ read_len,
                            sa_job* __restrict__ out, uint32_t* __restrict__ support,
                            uint32_t* __restrict__ read_first, uint64_t total) {
    const uint32_t rs = blockIdx.x * blockDim.x + threadIdx.x;
    if (rs >= n_rs) return;
    const uint64_t c0 = coff[rs];
    if ((rs & 1u) == 0) read_first[rs >> 1] = (uint32_t)c0;
    if (rs == n_rs - 1) read_first[n_rs >> 1] = (uint32_t)total;
    const uint32_t nc = ncand[rs];
    const uint64_t b = hoff[(uint64_t)rs * S];
    const uint32_t r = rs >> 1;
    for (uint32_t q = 0; q < nc; q++) {
        const TmpCand c = tmp[b + q];
        sa_job j;
        j.read_off = read_off[r];
        j.read_len = read_len[r];
        j.flags = (rs & 1u) ? SA_RC : 0u;
        j.ref_pos = c.ref_pos;
        j.win_len = c.win_len;
        j._pad = 0;
        out[c0 + q] = j;
        support[c0 + q] = c.support;
    }
}

int check_seed_params(const sa_seed_params* p) {
    if (!p) return err(SA_EINVAL, "seed params is NULL");
    if (p->seed_len < (uint32_t)sa::kLutK || p->seed_len > (uint32_t)sa::kKeyBases)
        return err(SA_EINVAL, "seed_len must be %d..%d", sa::kLutK, sa::kKeyBases);
    if (p->seed_step < 1) return err(SA_EINVAL, "seed_step must be >= 1");
    if (p->max_occ < 1) return err(SA_EINVAL, "max_occ must be >= 1");
    if (p->pad > (1u << 16) || p->join > (1u << 16)) return err(SA_EINVAL, "pad and join must be <= 65536");
    return SA_OK;
}

int run_candidates(sa_seed_index* I, const sa_seed_params* P, const char* d_reads, uint64_t reads_len,
                   const uint64_t* d_off, const uint32_t* d_len, uint32_t n_reads, sa_job* d_out,
                   uint32_t* d_support, uint32_t* d_first, uint64_t cap, uint64_t* n_cand, cudaStream_t st) {
    ETRY(I->stats.ensure(sizeof(SeedStats), "seed statistics"));
    if (!I->h_stats) ECU(cudaMallocHost((void**)&I->h_stats, sizeof(SeedStats)));
    SeedStats* ds = I->stats.as<SeedStats>();
    ECU(cudaMemsetAsync(ds, 0, sizeof(SeedStats), st));
    ECU(cudaMemsetAsync(&ds->bad_read, 0xff, 4, st));
    const uint8_t* reads = reinterpret_cast<const uint8_t*>(d_reads);
    k_seed_validate<<<(n_reads + 7) / 8, 256, 0, st>>>(reads, reads_len, d_off, d_len, n_reads, ds);
    ECU(cudaGetLastError());
    ECU(cudaMemcpyAsync(I->h_stats, ds, sizeof(SeedStats), cudaMemcpyDeviceToHost, st));
    ECU(cudaStreamSynchronize(st));
    if (I->h_stats->bad_read != 0xffffffffu)
        return err(SA_EINVAL, "read %u is invalid (length 1..%u inside the reads buffer, bases A, C, G, T)",
                   I->h_stats->bad_read, SA_MAX_READ);
    const uint32_t max_n = I->h_stats->max_n;
    const uint32_t S = max_n >= P->seed_len ? (max_n - P->seed_len) / P->seed_step + 1 : 1;
    if (S > (uint32_t)kMaxSeedsPerStrand)
        return err(SA_EINVAL, "reads of %u bases have %u seeds per strand, more than %d: raise seed_step",
                   max_n, S, kMaxSeedsPerStrand);
    if ((uint64_t)S * P->max_occ > kMaxHitsPerStrand)
        return err(SA_EINVAL, "%u seeds per strand x max_occ %u may exceed %u hits per read strand: lower "
                   "max_occ or raise seed_step", S, P->max_occ, kMaxHitsPerStrand);
    const uint32_t n_rs = 2 * n_reads;
    const uint64_t n_slots = (uint64_t)n_rs * S;
    ETRY(I->seeds.ensure(n_slots * sizeof(uint2), "seeds"));
    ETRY(I->cnt.ensure(n_slots * 4 + 4, "seed counts"));
    ETRY(I->hoff.ensure((n_slots + 1) * 8, "hit offsets"));
    ETRY(I->bsum.ensure(sa::scan_bsum_len(n_slots + 1) * 8, "scan"));
    ETRY(I->ncand.ensure((size_t)n_rs * 4 + 4, "region counts"));
    ETRY(I->coff.ensure(((size_t)n_rs + 1) * 8, "candidate offsets"));
    ETRY(I->large.ensure((size_t)n_rs * 4, "large list"));
    SearchArgs A{};
    A.reads = reads;
    A.read_off = d_off;
    A.read_len = d_len;
    A.n_reads = n_reads;
    A.S = S;
    A.lam = (int)P->seed_len;
    A.step = (int)P->seed_step;
    A.max_occ = P->max_occ;
    A.lut = I->d_lut;
    A.occ = I->d_occ;
    A.dollar_row = I->dollar_row;
    A.C0 = I->C[0];
    A.C1 = I->C[1];
    A.C2 = I->C[2];
    A.C3 = I->C[3];
    A.seed = I->seeds.as<uint2>();
    A.cnt = I->cnt.as<uint32_t>();
    k_seed_search<<<(unsigned)((n_slots + 255) / 256), 256, 0, st>>>(A);
    ECU(cudaGetLastError());
    // hit offsets: exclusive scan over the slots plus one closing entry
    ECU(cudaMemsetAsync(I->cnt.as<uint32_t>() + n_slots, 0, 4, st));
    sa::launch_scan_u32(I->cnt.as<uint32_t>(), n_slots + 1, I->hoff.as<uint64_t>(), I->bsum.as<uint64_t>(),
                        &ds->total[0], st);
    ECU(cudaGetLastError());
    ECU(cudaMemcpyAsync(&I->h_stats->total[0], &ds->total[0], 8, cudaMemcpyDeviceToHost, st));
    ECU(cudaStreamSynchronize(st));
    const uint64_t n_hits = I->h_stats->total[0];
    ETRY(I->hits.ensure(std::max<uint64_t>(n_hits, 1) * 8, "hits"));
    ETRY(I->tmp.ensure(std::max<uint64_t>(n_hits, 1) * sizeof(TmpCand), "regions"));
    k_seed_locate<<<(unsigned)((n_slots + 255) / 256), 256, 0, st>>>(
        I->seeds.as<uint2>(), I->hoff.as<uint64_t>(), n_slots, S, (int)P->seed_step, I->d_sa,
        I->hits.as<uint64_t>());
    ECU(cudaGetLastError());
    ClusterArgs C{};
    C.hits = I->hits.as<uint64_t>();
    C.hoff = I->hoff.as<uint64_t>();
    C.n_slots = n_slots;
    C.S = S;
    C.n_rs = n_rs;
    C.read_len = d_len;
    C.L = (int64_t)I->L;
    C.pad = P->pad;
    C.join = P->join;
    C.tmp = I->tmp.as<TmpCand>();
    C.ncand = I->ncand.as<uint32_t>();
    C.large = I->large.as<uint32_t>();
    C.st = ds;
    k_seed_cluster_small<<<(n_rs + 127) / 128, 128, 0, st>>>(C);
    ECU(cudaGetLastError());
    ECU(cudaMemcpyAsync(&I->h_stats->n_large, &ds->n_large, 4, cudaMemcpyDeviceToHost, st));
    ECU(cudaStreamSynchronize(st));
    if (I->h_stats->n_large) {
        const size_t smem = kMaxHitsPerStrand * (8 + 4);
        ECU(cudaFuncSetAttribute(k_seed_cluster_large, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_seed_cluster_large<<<I->h_stats->n_large, kLargeThreads, smem, st>>>(C);
        ECU(cudaGetLastError());
    }
    ECU(cudaMemsetAsync(I->ncand.as<uint32_t>() + n_rs, 0, 4, st));
    sa::launch_scan_u32(I->ncand.as<uint32_t>(), (uint64_t)n_rs + 1, I->coff.as<uint64_t>(), I->bsum.as<uint64_t>(),
                        &ds->total[1], st);
    ECU(cudaGetLastError());
    ECU(cudaMemcpyAsync(&I->h_stats->total[1], &ds->total[1], 8, cudaMemcpyDeviceToHost, st));
    ECU(cudaStreamSynchronize(st));
    const uint64_t total = I->h_stats->total[1];
    *n_cand = total;
    if (total > cap)
        return err(SA_EOVERFLOW, "%llu candidate windows, room for %llu", (unsigned long long)total,
                   (unsigned long long)cap);
    if (total > 0xffffffffull) return err(SA_EOVERFLOW, "more than 2^32 candidate windows; split the batch");
    k_seed_emit<<<(n_rs + 127) / 128, 128, 0, st>>>(I->tmp.as<TmpCand>(), I->hoff.as<uint64_t>(), S,
                                                    I->ncand.as<uint32_t>(), I->coff.as<uint64_t>(), n_rs, d_off,
                                                    d_len, d_out, d_support, d_first, total);
    ECU(cudaGetLastError());
    ECU(cudaStreamSynchronize(st));
    return SA_OK;
}

}  // namespace

extern "C" {

void sa_default_seed_params(sa_seed_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->seed_len = 20;
    p->seed_step = 10;
    p->max_occ = 256;
    p->pad = 24;
    p->join = 16;
}

int sa_seed_index_create(sa_reference* ref, sa_seed_index** out) {
    try {
        sa::set_error(SA_OK, "");
        if (!ref || !out) return err(SA_EINVAL, "NULL argument");
        *out = nullptr;
        const sa::RefView V = sa::ref_view(ref);
        if (V.len + sa::kKeyBases >= 0xffffffffull)
            return err(SA_EINVAL, "the seed index holds references of up to 2^32 - 33 bases");
        ECU(cudaSetDevice(V.device));
        // the packed reference back from the device (the same bases the alignment reads)
        const uint64_t words = (V.len + 15) / 16;
        std::vector<uint32_t> w(words + 4, 0);
        ECU(cudaMemcpy(w.data(), V.d_words + sa::kRefFrontPad, words * 4, cudaMemcpyDeviceToHost));
        sa::SeedHostIndex H;
        sa::build_seed_index(w.data(), V.len, H);
        std::unique_ptr<sa_seed_index> I(new (std::nothrow) sa_seed_index());
        if (!I) return err(SA_ENOMEM, "host allocation failed");
        I->device = V.device;
        I->L = V.len;
        I->rows = (uint32_t)(V.len + 1);
        I->dollar_row = H.dollar_row;
        for (int c = 0; c < 4; c++) I->C[c] = H.C[c];
        I->own = V.own;
        auto up = [&](void** dst, const void* src, size_t bytes) -> int {
            if (cudaMalloc(dst, bytes) != cudaSuccess) {
                cudaGetLastError();
                return err(SA_ENOMEM, "cudaMalloc of %zu bytes for the seed index failed", bytes);
            }
            ECU(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
            return SA_OK;
        };
        int rc = up((void**)&I->d_sa, H.sa.data(), H.sa.size() * 4);
        if (rc == SA_OK) rc = up((void**)&I->d_occ, H.occ.data(), H.occ.size() * 4);
        static_assert(sizeof(sa::RowInterval) == sizeof(uint2), "lookup table entries are two uint32");
        if (rc == SA_OK) rc = up((void**)&I->d_lut, H.lut.data(), H.lut.size() * sizeof(uint2));
        if (rc != SA_OK) {
            cudaFree(I->d_sa);
            cudaFree(I->d_occ);
            cudaFree(I->d_lut);
            return rc;
        }
        *out = I.release();
        return SA_OK;
    } catch (const std::bad_alloc&) {
        return err(SA_ENOMEM, "host memory exhausted while building the seed index");
    } catch (...) {
        return err(SA_ECUDA, "unexpected host exception");
    }
}

int sa_seed_index_destroy(sa_seed_index* I) {
    if (!I) return err(SA_EINVAL, "seed index is NULL");
    try {
        cudaSetDevice(I->device);
        {
            std::lock_guard<std::mutex> lk(I->mu);
            Buf* all[] = {&I->stats, &I->seeds, &I->cnt, &I->hoff, &I->bsum, &I->hits, &I->large, &I->tmp,
                          &I->ncand, &I->coff};
            for (Buf* b : all) b->release();
            if (I->h_stats) cudaFreeHost(I->h_stats);
            cudaFree(I->d_sa);
            cudaFree(I->d_occ);
            cudaFree(I->d_lut);
        }
        delete I;
        return SA_OK;
    } catch (...) {
        return err(SA_ECUDA, "unexpected host exception");
    }
}

int sa_seed_index_info(const sa_seed_index* I, uint64_t* ref_len, uint64_t* device_bytes) {
    if (!I) return err(SA_EINVAL, "seed index is NULL");
    if (ref_len) *ref_len = I->L;
    if (device_bytes)
        *device_bytes = (uint64_t)I->rows * 4 + ((uint64_t)I->rows / sa::kChunkRows + 1) * 64 + (uint64_t)sa::kLutSize * 8;
    return SA_OK;
}

int sa_seed_candidates_dev(sa_seed_index* I, const sa_seed_params* P, const char* d_reads, uint64_t reads_len,
                           const uint64_t* d_read_off, const uint32_t* d_read_len, uint32_t n_reads,
                           sa_job* d_cand, uint32_t* d_support, uint32_t* d_read_first, uint64_t cand_cap,
                           uint64_t* n_cand, void* cuda_stream) {
    try {
        sa::set_error(SA_OK, "");
        if (!I || !n_cand) return err(SA_EINVAL, "NULL seed index or n_cand");
        ETRY(check_seed_params(P));
        *n_cand = 0;
        if (!d_read_first) return err(SA_EINVAL, "read_first is NULL");
        if (n_reads && (!d_reads || !d_read_off || !d_read_len)) return err(SA_EINVAL, "NULL read buffer");
        if (n_reads >= (1u << 30)) return err(SA_EINVAL, "at most 2^30 - 1 reads per call");
        std::lock_guard<std::mutex> lk(I->mu);
        ECU(cudaSetDevice(I->device));
        cudaStream_t st = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : I->own;
        if (n_reads == 0) {
            ECU(cudaMemsetAsync(d_read_first, 0, 4, st));
            ECU(cudaStreamSynchronize(st));
            return SA_OK;
        }
        if (cand_cap && (!d_cand || !d_support)) return err(SA_EINVAL, "NULL candidate buffer");
        return run_candidates(I, P, d_reads, reads_len, d_read_off, d_read_len, n_reads, d_cand, d_support,
                              d_read_first, cand_cap, n_cand, st);
    } catch (...) {
        return err(SA_ECUDA, "unexpected host exception");
    }
}

int sa_seed_candidates(sa_seed_index* I, const sa_seed_params* P, const char* reads, uint64_t reads_len,
                       const uint64_t* read_off, const uint32_t* read_len, uint32_t n_reads, sa_job* cand,
                       uint32_t* support, uint32_t* read_first, uint64_t cand_cap, uint64_t* n_cand) {
    try {
        sa::set_error(SA_OK, "");
        if (!I || !n_cand) return err(SA_EINVAL, "NULL seed index or n_cand");
        ETRY(check_seed_params(P));
        *n_cand = 0;
        if (!read_first) return err(SA_EINVAL, "read_first is NULL");
        if (n_reads && (!reads || !read_off || !read_len)) return err(SA_EINVAL, "NULL read buffer");
        if (cand_cap && (!cand || !support)) return err(SA_EINVAL, "NULL candidate buffer");
        ECU(cudaSetDevice(I->device));
        Buf dr, doff, dlen, dc, dsup, dfirst;
        struct Free {
            Buf* b[6];
            ~Free() {
                for (Buf* x : b) x->release();
            }
        } guard{{&dr, &doff, &dlen, &dc, &dsup, &dfirst}};
        ETRY(dr.ensure(reads_len + 16, "reads"));
        ETRY(doff.ensure((size_t)n_reads * 8 + 8, "read offsets"));
        ETRY(dlen.ensure((size_t)n_reads * 4 + 4, "read lengths"));
        ETRY(dfirst.ensure(((size_t)n_reads + 1) * 4, "read_first"));
        if (reads_len) ECU(cudaMemcpy(dr.p, reads, reads_len, cudaMemcpyHostToDevice));
        if (n_reads) {
            ECU(cudaMemcpy(doff.p, read_off, (size_t)n_reads * 8, cudaMemcpyHostToDevice));
            ECU(cudaMemcpy(dlen.p, read_len, (size_t)n_reads * 4, cudaMemcpyHostToDevice));
        }
        // device output as large as the caller's buffers
        const uint64_t dev_cap = std::max<uint64_t>(cand_cap, 1);
        ETRY(dc.ensure(dev_cap * sizeof(sa_job), "candidates"));
        ETRY(dsup.ensure(dev_cap * 4, "support"));
        const int rc = sa_seed_candidates_dev(I, P, dr.as<char>(), reads_len, doff.as<uint64_t>(),
                                              dlen.as<uint32_t>(), n_reads, dc.as<sa_job>(), dsup.as<uint32_t>(),
                                              dfirst.as<uint32_t>(), cand_cap, n_cand, nullptr);
        if (rc != SA_OK) return rc;
        ECU(cudaMemcpy(read_first, dfirst.p, ((size_t)n_reads + 1) * 4, cudaMemcpyDeviceToHost));
        if (*n_cand) {
            ECU(cudaMemcpy(cand, dc.p, *n_cand * sizeof(sa_job), cudaMemcpyDeviceToHost));
            ECU(cudaMemcpy(support, dsup.p, *n_cand * 4, cudaMemcpyDeviceToHost));
        }
        return SA_OK;
    } catch (...) {
        return err(SA_ECUDA, "unexpected host exception");
    }
}

}  // extern "C"
