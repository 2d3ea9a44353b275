// Staging, planning, traceback and result kernels of libsa.
//
//  pack_ref       ASCII reference -> 2-bit words (validation included)
//  plan           per job: validation, length bucket + size class, statistics
//  plan_scan      bucket histogram -> offsets (one block)
//  plan_scatter   job ids into bucket order
//  pack_reads     ASCII reads -> 2-bit words, reverse complement for SA_RC jobs
//  rect_plan      per job: the sub-rectangle that holds every optimal path
//  scan_u64       exclusive prefix sums (3-phase)
//  traceback      walk the direction bits from the best cell (one thread per job)
//  finalize       sa_result + compacted CIGAR in job order
#include <cstdio>

#include "kernels.h"
#include "walk.cuh"

namespace sa {

__device__ __forceinline__ int base_code(uint8_t c) {
    switch (c) {
    case 'A': case 'a': return 0;
    case 'C': case 'c': return 1;
    case 'G': case 'g': return 2;
    case 'T': case 't': return 3;
    }
    return -1;
}

// ---------------------------------------------------------------------------
// reference packing: one thread per output word (16 bases)

__global__ void k_pack_ref(const uint8_t* __restrict__ ascii, uint64_t len, uint64_t base_off,
                           uint32_t* __restrict__ words, unsigned long long* bad_pos) {
    const uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint64_t p0 = w * 16;
    if (p0 >= len) return;
    uint32_t v = 0;
    for (int k = 0; k < 16; k++) {
        const uint64_t p = p0 + k;
        if (p >= len) break;
        const int c = base_code(ascii[p]);
        if (c < 0) { atomicMin(bad_pos, (unsigned long long)(base_off + p)); continue; }
        v |= (uint32_t)c << (2 * k);
    }
    words[(base_off / 16) + w] = v;
}

void launch_pack_ref(const uint8_t* ascii, uint64_t len, uint64_t base_off, uint32_t* words,
                     unsigned long long* bad_pos, cudaStream_t st) {
    const uint64_t nw = (len + 15) / 16;
    if (!nw) return;
    k_pack_ref<<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(ascii, len, base_off, words, bad_pos);
}

// ---------------------------------------------------------------------------
// planning

__global__ void k_plan(const sa_job* __restrict__ jobs, uint32_t n_jobs, uint64_t reads_len,
                       int64_t ref_len, const uint8_t* __restrict__ plan_cfg, uint16_t* __restrict__ key,
                       uint32_t* __restrict__ hist, PlanStats* stats) {
    __shared__ uint32_t sh[kNumKeys];
    for (int k = threadIdx.x; k < kNumKeys; k += blockDim.x) sh[k] = 0;
    __syncthreads();
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t maxn = 0, maxm = 0;
    unsigned long long cells = 0;
    if (j < n_jobs) {
        const sa_job J = jobs[j];
        const uint32_t n = J.read_len, m = J.win_len;
        bool ok = n >= 1 && n <= SA_MAX_READ && m >= 1 && m <= SA_MAX_WINDOW &&
                  J.ref_pos <= (uint64_t)ref_len && (uint64_t)m <= (uint64_t)ref_len - J.ref_pos &&
                  J.read_off <= reads_len && (uint64_t)n <= reads_len - J.read_off &&
                  (J.flags & ~SA_RC) == 0u;
        if (!ok) {
            atomicMin(&stats->bad_job, j);
            key[j] = 0;
        } else {
            const int c = plan_cfg ? (int)plan_cfg[n] : cfg_for_rows((int)n);
            const int k = c * kNumSizeCls + (kNumSizeCls - 1 - size_class(m));
            key[j] = (uint16_t)k;
            atomicAdd(&sh[k], 1u);
            maxn = n;
            maxm = m;
            cells = (unsigned long long)n * m;
        }
    }
    // warp-aggregate the statistics
    for (int o = 16; o >= 1; o >>= 1) {
        maxn = max(maxn, __shfl_xor_sync(0xffffffffu, maxn, o));
        maxm = max(maxm, __shfl_xor_sync(0xffffffffu, maxm, o));
        cells += __shfl_xor_sync(0xffffffffu, cells, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&stats->max_n, maxn);
        atomicMax(&stats->max_m, maxm);
        atomicAdd(&stats->cells, cells);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kNumKeys; k += blockDim.x)
        if (sh[k]) atomicAdd(&hist[k], sh[k]);
}

constexpr int kScanKeysThreads = 1024;
__global__ void __launch_bounds__(kScanKeysThreads)
k_plan_scan(const uint32_t* __restrict__ hist, uint32_t* __restrict__ key_off, uint32_t* __restrict__ cursor) {
    // one block: exclusive scan of the kNumKeys counts, kPer consecutive keys a thread
    constexpr int kPer = (kNumKeys + kScanKeysThreads - 1) / kScanKeysThreads;
    __shared__ uint32_t warp_tot[32];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    uint32_t v[kPer], sum = 0;
#pragma unroll
    for (int q = 0; q < kPer; q++) {
        const int k = t * kPer + q;
        v[q] = k < kNumKeys ? hist[k] : 0u;
        sum += v[q];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += x;
        }
        warp_tot[lane] = w;                    // inclusive over warps
    }
    __syncthreads();
    uint32_t acc = incl - sum + (wid ? warp_tot[wid - 1] : 0u);
#pragma unroll
    for (int q = 0; q < kPer; q++) {
        const int k = t * kPer + q;
        if (k < kNumKeys) key_off[k] = acc;
        acc += v[q];
    }
    if (t == kScanKeysThreads - 1) key_off[kNumKeys] = warp_tot[31];
    for (int k = t; k < kNumKeys; k += kScanKeysThreads) cursor[k] = 0;
}

__global__ void k_plan_scatter(const uint16_t* __restrict__ key, uint32_t n_jobs,
                               const uint32_t* __restrict__ key_off, uint32_t* __restrict__ cursor,
                               uint32_t* __restrict__ order) {
    // lanes with the same key take their slots with one atomic per key and warp
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int k = j < n_jobs ? (int)key[j] : -1;
    const unsigned same = __match_any_sync(0xffffffffu, k);
    const int leader = __ffs(same) - 1;
    uint32_t base = 0;
    if (lane == leader && k >= 0) base = atomicAdd(&cursor[k], (uint32_t)__popc(same));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (k >= 0) order[key_off[k] + base + (uint32_t)__popc(same & ((1u << lane) - 1u))] = j;
}

void launch_plan(const sa_job* jobs, uint32_t n_jobs, uint64_t reads_len, int64_t ref_len,
                 const uint8_t* plan_cfg, uint16_t* key, uint32_t* hist, PlanStats* stats, cudaStream_t st) {
    if (!n_jobs) return;
    k_plan<<<(n_jobs + 255) / 256, 256, 0, st>>>(jobs, n_jobs, reads_len, ref_len, plan_cfg, key, hist, stats);
}

void launch_plan_order(const uint16_t* key, uint32_t n_jobs, const uint32_t* hist,
                       uint32_t* key_off, uint32_t* cursor, uint32_t* order, cudaStream_t st) {
    k_plan_scan<<<1, kScanKeysThreads, 0, st>>>(hist, key_off, cursor);
    if (n_jobs)
        k_plan_scatter<<<(n_jobs + 255) / 256, 256, 0, st>>>(key, n_jobs, key_off, cursor, order);
}

// ---------------------------------------------------------------------------
// jobs the 16-bit pass flagged: per length bucket, compacted into that bucket's
// range of `list` (list[cfg_begin[c] + k]), counts in cnt[c]

__global__ void k_collect_overflow(const uint32_t* __restrict__ order, uint32_t n_pos,
                                   const JobState* __restrict__ state,
                                   const uint32_t* __restrict__ cfg_begin, uint32_t* __restrict__ list,
                                   uint32_t* __restrict__ cnt) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pos) return;
    const uint32_t job = order[p];
    if (!(state[job].flags & kStOverflow)) return;
    int c = 0;
    while (c + 1 < kNumCfg && cfg_begin[c + 1] <= p) c++;
    list[cfg_begin[c] + atomicAdd(&cnt[c], 1u)] = job;
}

void launch_collect_overflow(const uint32_t* order, uint32_t n_pos, const JobState* state,
                             const uint32_t* cfg_begin, uint32_t* list, uint32_t* cnt,
                             cudaStream_t st) {
    if (!n_pos) return;
    k_collect_overflow<<<(n_pos + 255) / 256, 256, 0, st>>>(order, n_pos, state, cfg_begin, list, cnt);
}

// ---------------------------------------------------------------------------
// read packing: one thread per 16-base output word.  The thread loads the (at
// most five) aligned 32-bit words that hold its 16 source bytes, lines them up
// with funnel shifts, and converts four bytes at a time: the 2-bit code of an
// A/C/G/T byte (either case) is ((x >> 1) ^ (x >> 2)) & 3, and the byte is valid
// when it equals the character its code names ("acgt", looked up with a byte
// permute) once lower-cased.  A reverse-complemented job's word is the forward
// packing of the mirrored source bytes with its 2-bit fields reversed and
// complemented.

__device__ __forceinline__ uint32_t pack4_codes(uint32_t x, uint32_t* bad_bytes) {
    const uint32_t c = ((x >> 1) ^ (x >> 2)) & 0x03030303u;          // code of each byte
    // the selector c0 | c1<<4 | c2<<8 | c3<<12 from the code bytes, then "acgt"[code]
    const uint32_t sel = __byte_perm(c | (c >> 4), 0u, 0x4420);
    const uint32_t want = __byte_perm(0x74676361u, 0u, sel);
    *bad_bytes = (x | 0x20202020u) ^ want;                          // nonzero bytes: not ACGTacgt
    // the four codes side by side in the top byte (the other products stay below it)
    return c * 0x01041040u;
}

__global__ void k_pack_reads(const sa_job* __restrict__ jobs, uint32_t n_jobs,
                             const uint8_t* __restrict__ reads, uint32_t* __restrict__ rpack,
                             uint32_t rw, unsigned* bad_job) {
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t job = (uint32_t)(t / rw), w = (uint32_t)(t % rw);
    if (job >= n_jobs) return;
    const sa_job J = jobs[job];
    const int n = (int)J.read_len;
    if (16 * (int)w >= n) return;                    // past the read: never read by the passes
    const bool rc = (J.flags & SA_RC) != 0u;
    // the source bytes of this word: forward [16w, 16w + cnt), reverse-complemented
    // the mirror image [n - 16w - cnt, n - 16w)
    const int cnt = min(16, n - 16 * (int)w);
    const int lo = rc ? n - 16 * (int)w - cnt : 16 * (int)w;
    const uint8_t* src = reads + J.read_off + lo;
    const uint32_t mis = (uint32_t)((uintptr_t)src & 3u);
    const uint32_t* wp = reinterpret_cast<const uint32_t*>((uintptr_t)src - mis);
    const int nw = (int)((mis + (uint32_t)cnt + 3u) >> 2);       // aligned words holding the bytes
    uint32_t q[5];
#pragma unroll
    for (int k = 0; k < 5; k++) q[k] = k < nw ? __ldg(wp + k) : 0u;
    uint32_t top[4], badw = 0u;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const uint32_t x = __funnelshift_r(q[k], q[k + 1], 8u * mis);   // bytes 4k .. 4k+3
        uint32_t bb;
        top[k] = pack4_codes(x, &bb);
        // only bytes j < cnt are the read's
        const int left = cnt - 4 * k;
        const uint32_t keep = left >= 4 ? 0xFFFFFFFFu : (left <= 0 ? 0u : (1u << (8 * left)) - 1u);
        badw |= bb & keep;
    }
    // codes of bytes 0..15 at bits 2j
    uint32_t v = __byte_perm(__byte_perm(top[0], top[1], 0x0073), __byte_perm(top[2], top[3], 0x0073), 0x5410);
    if (cnt < 16) v &= (1u << (2 * cnt)) - 1u;
    if (rc) {
        // field j -> field cnt-1-j, complemented: reverse all 32 bits, swap each
        // field's two bits back, drop the fields past cnt, flip the codes (3 - c)
        uint32_t r = __brev(v);
        r = ((r >> 1) & 0x55555555u) | ((r & 0x55555555u) << 1);
        r >>= 2 * (16 - cnt);
        v = r ^ (cnt < 16 ? (1u << (2 * cnt)) - 1u : 0xFFFFFFFFu);
    }
    rpack[(size_t)job * rw + w] = v;
    if (badw) atomicMin(bad_job, job);
}

void launch_pack_reads(const sa_job* jobs, uint32_t n_jobs, const uint8_t* reads, uint32_t* rpack,
                       uint32_t rw, unsigned* bad_job, cudaStream_t st) {
    if (!n_jobs) return;
    const uint64_t threads = (uint64_t)n_jobs * rw;
    k_pack_reads<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(jobs, n_jobs, reads, rpack, rw, bad_job);
}

struct BandLists { uint32_t* p[kNumBand]; };

// ---------------------------------------------------------------------------
// reduced traceback rectangle.
//
// Every alignment path that ends at the best cell (i*, j*) with the best score
// uses at most j* read bases (#M + #I <= j*) and, because each deleted window
// base costs at least e, at most (a*j* - best)/e deletions (#D).  Its first
// cell is therefore at column >= i* - j* - (a*j* - best)/e.  The DP restricted
// to columns [i_lo, i*] and rows [1, j*] (with the border of a fresh DP on its
// left) reproduces every value on such a path and every comparison the
// traceback makes, so the walk from its corner gives the same CIGAR.
// With e = 0 the bound does not exist and the whole window is used.
// Before any of that, a job whose traceback is a gapless diagonal run (below)
// takes the diagonal class and no direction pass at all.

// Steps of a gapless traceback from the best cell, or 0.  Let c_m be the score
// of the m diagonal cells ending at (i*, j*).  If c_k = best (LOCAL: the first
// such k; GLOCAL: k = j*, the run starting on row 0), then along the run
// H(i*-m, j*-m) = best - c_m: each H is at least the run's prefix score (a path
// to it) and at most H(i, j) - delta (the recurrence).  The traceback takes the
// diagonal first on ties (SOAP3-dp Methods section 3 backtracks from the end
// cell through the recurrence's sources), so it walks exactly that run: down to
// the first zero, where LOCAL stops, or to row 0.  Its CIGAR is k matches /
// mismatches and it needs no direction pass.
// 16 bases p0 .. p0 + 15 of a packed sequence (base p at bits 2 (p & 15) of
// word p >> 4), base p0 + t at bits 2t; the second word is read only when the
// bases straddle it (so p0 + 15 is the last base the caller may touch)
__device__ __forceinline__ uint32_t bases16_from(const uint32_t* __restrict__ w, uint64_t p0) {
    const uint64_t wi = p0 >> 4;
    const uint32_t sh = (uint32_t)(p0 & 15) * 2u;
    const uint32_t lo = __ldg(w + wi);
    return sh ? (uint32_t)((((uint64_t)__ldg(w + wi + 1) << 32) | lo) >> sh) : lo;
}

__device__ int gapless_steps(const uint32_t* __restrict__ refw, uint64_t ref_pos, const uint32_t* __restrict__ rp,
                             int istar, int jstar, int32_t best, const Score& sc) {
    const bool local = sc.mode == SA_LOCAL;
    if (!local && jstar > istar) return 0;            // the run would leave the window before row 0
    const int mmax = min(istar, jstar);
    int32_t c = 0;
    int m = 0;
    // 16 steps at a time: the window and read bases of steps m+1 .. m+16 compared
    // as two words (base t of both at bits 2t is step m + 16 - t)
    while (mmax - m >= 16) {
        const uint32_t x = bases16_from(refw, ref_pos + (uint64_t)(istar - m - 16)) ^
                           bases16_from(rp, (uint64_t)(jstar - m - 16));
        const uint32_t eq = ~(x | (x >> 1)) & 0x55555555u;
        if (local && (int64_t)c + 16 * (int64_t)sc.a >= best) {
            // the best can be reached inside these 16 steps: take them one by one
            for (int t = 15; t >= 0; t--) {
                c += ((eq >> (2 * t)) & 1u) ? sc.a : sc.b;
                m++;
                if (c == best) return m;
            }
        } else {
            const int mt = __popc(eq);
            c += sc.a * mt + sc.b * (16 - mt);
            m += 16;
        }
        if ((int64_t)c + (int64_t)sc.a * (mmax - m) < best) return 0;   // best is out of reach
    }
    uint64_t tw_at = ~0ull;
    uint32_t tw = 0, rwd = 0;
    int rw_at = -1;
    while (m < mmax) {
        m++;
        const uint64_t pos = ref_pos + (uint64_t)(istar - m);          // window column i* - m + 1
        const int jr = jstar - m;                                      // read row j* - m + 1, 0-based
        if ((pos >> 4) != tw_at) { tw_at = pos >> 4; tw = __ldg(refw + tw_at); }
        if ((jr >> 4) != rw_at) { rw_at = jr >> 4; rwd = __ldg(rp + rw_at); }
        const uint32_t tb = (tw >> (2 * (pos & 15))) & 3u, rb = (rwd >> (2 * (jr & 15))) & 3u;
        c += tb == rb ? sc.a : sc.b;
        if (local && c == best) return m;
        if ((int64_t)c + (int64_t)sc.a * (mmax - m) < best) return 0;
    }
    return (!local && c == best) ? jstar : 0;
}

__global__ void k_rect_plan(const sa_job* __restrict__ jobs, const uint32_t* __restrict__ order,
                            uint32_t n_pos, const uint32_t* __restrict__ cfg_begin,
                            const JobState* __restrict__ state, Score sc,
                            int32_t min_score, int allow_band, Rect* __restrict__ rect,
                            uint64_t* __restrict__ sizes, BandLists lists, uint32_t* cls_count,
                            uint32_t* __restrict__ rect_flag, int heights, const uint32_t* __restrict__ refw,
                            const uint32_t* __restrict__ rpack, uint32_t rw) {
    // no early return: the class lists are appended with warp-wide ballots
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = p < n_pos;
    const uint32_t job = valid ? order[p] : 0u;
    Rect R;
    R.off = 0;
    R.wave = 0;
    R.i_lo = 1;
    R.w = 0;
    R.rows = 0;
    R.start_i = 0;
    R.start_j = 0;
    R.cls = kClsNone;
    R.d_lo = 0;
    R.lpos = 0;
    int c = 0;
    while (valid && c + 1 < kNumCfg && cfg_begin[c + 1] <= p) c++;   // the position's bucket
    R.cfg = c;
    if (valid) {
        const JobState st = state[job];
        if (!(st.flags & kStEmpty) && st.best >= min_score) {
            const int istar = st.i_star, jstar = st.j_star;
            const int64_t slack = (int64_t)sc.a * jstar - st.best;     // S = a*j* - best >= 0
            const int32_t e = -sc.GE;
            int64_t span = istar;
            R.cls = kClsRect;
            if (allow_band && slack == 0 && sc.a > 0) {
                // every base of an optimal path is a match: the walk from (i*, j*)
                // takes the diagonal (ties go to M first) down to row 0
                R.cls = kClsDiag;
                R.d_lo = istar - jstar;
            } else if (e > 0) {
                // a path with #D deletions pays at least o + e*#D for them (one
                // opening at least), one with #I insertions o + (a + e)*#I
                const int64_t o = (int64_t)sc.GE - sc.GO;                 // gap open magnitude
                const int64_t dmax = slack >= o + e ? (slack - o) / e : 0;
                const int64_t imax = slack >= o + sc.a + e ? (slack - o) / (sc.a + e) : 0;
                const int64_t width = dmax + imax + 1;
                R.d_lo = (int)((int64_t)(istar - jstar) - dmax);
                if (allow_band)
                    R.cls = width <= 8 ? kClsBand8 : width <= 16 ? kClsBand16
                          : (width <= 32 ? kClsBand32 : (width <= 64 ? kClsBand64 : kClsRect));
                span = (int64_t)jstar + dmax;
            }
            R.rows = jstar;
            if (R.cls != kClsDiag && allow_band) {
                const int k = gapless_steps(refw, jobs[job].ref_pos, rpack + (size_t)job * rw, istar, jstar,
                                            st.best, sc);
                if (k > 0) {
                    R.cls = kClsDiag;
                    R.rows = k;
                }
            }
            if (R.cls == kClsDiag) {
                R.d_lo = istar - jstar;
                R.start_i = istar;
                R.start_j = jstar;
            }
            if (R.cls == kClsRect) {
                int64_t ilo = (int64_t)istar - span + 1;
                if (ilo < 1) ilo = 1;
                R.i_lo = (int)ilo;
                R.w = istar - (int)ilo + 1;
                R.start_i = R.w;
                R.start_j = jstar;
            }
        }
    }
    const unsigned lane = threadIdx.x & 31u;
#pragma unroll
    for (int k = 0; k < kNumBand; k++) {
        const int cls = band_cls(k);
        const unsigned mask = __ballot_sync(0xffffffffu, valid && R.cls == cls);
        if (mask) {
            const int leader = __ffs(mask) - 1;
            uint32_t base = 0;
            if ((int)lane == leader) base = atomicAdd(&cls_count[cls], (uint32_t)__popc(mask));
            base = __shfl_sync(0xffffffffu, base, leader);
            if (valid && R.cls == cls) {
                R.lpos = base + (uint32_t)__popc(mask & ((1u << lane) - 1u));
                lists.p[k][R.lpos] = job;
            }
        }
    }
#pragma unroll
    for (int cls : {(int)kClsRect, (int)kClsDiag}) {
        const unsigned mask = __ballot_sync(0xffffffffu, valid && R.cls == cls);
        if (mask && (int)lane == __ffs(mask) - 1) atomicAdd(&cls_count[cls], (uint32_t)__popc(mask));
    }
    if (valid) {
        rect[job] = R;
        sizes[p] = R.w > 0 ? rect_words(cfg_L(c), cfg_K(c), R.w, heights != 0) : 0;
        rect_flag[p] = R.w > 0 ? 1u : 0u;
    }
}

// the jobs of the wavefront rectangle pass, in the bucketed order (rect_pos is
// the exclusive scan of rect_flag), and where each bucket's run of them begins
// The jobs of the wavefront rectangle pass, by bucket and within a bucket by
// rectangle width, widest first (a counting sort on kRectWidthClasses classes of
// eight columns): the lane groups of a warp then run rectangles of about the same
// width, and a warp runs as many steps as its widest.  The order inside a class is
// the arrival order of the scatter's atomics, which changes no result: each job's
// direction data depends on its own rectangle only.  list_pos[q] is the bucketed
// position of list entry q; rect_begin[c] is where bucket c's run begins.
constexpr int kRectWidthClasses = 128;

__device__ __forceinline__ uint32_t rect_sort_key(const Rect& R) {
    const int cls = min(kRectWidthClasses - 1, (R.w + 7) >> 3);
    return (uint32_t)(R.cfg * kRectWidthClasses + (kRectWidthClasses - 1 - cls));
}

__global__ void k_rect_hist(const uint32_t* __restrict__ order, uint32_t n_pos, const uint32_t* __restrict__ rect_flag,
                            const Rect* __restrict__ rect, uint32_t* __restrict__ hist) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n_pos && rect_flag[p]) atomicAdd(&hist[rect_sort_key(rect[order[p]])], 1u);
}

__global__ void k_rect_scatter(const uint32_t* __restrict__ order, uint32_t n_pos,
                               const uint32_t* __restrict__ rect_flag, const Rect* __restrict__ rect,
                               const uint64_t* __restrict__ start, uint32_t* __restrict__ cursor,
                               uint32_t* __restrict__ list, uint32_t* __restrict__ list_pos) {
    const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n_pos && rect_flag[p]) {
        const uint32_t job = order[p];
        const uint32_t key = rect_sort_key(rect[job]);
        const uint64_t q = start[key] + atomicAdd(&cursor[key], 1u);
        list[q] = job;
        list_pos[q] = p;
    }
}

__global__ void k_rect_bounds(const uint64_t* __restrict__ start, const uint64_t* total,
                              uint32_t* __restrict__ rect_begin) {
    const int c = threadIdx.x;
    if (c < kNumCfg) rect_begin[c] = (uint32_t)start[c * kRectWidthClasses];
    if (c == kNumCfg) rect_begin[c] = (uint32_t)*total;
}

uint64_t rect_sort_bytes() { return (uint64_t)kNumCfg * kRectWidthClasses * 16; }

void launch_rect_list(const uint32_t* order, uint32_t n_pos, const uint32_t* rect_flag, const Rect* rect,
                      void* sort_scratch, uint64_t* bsum, uint64_t* total, uint32_t* list, uint32_t* list_pos,
                      uint32_t* rect_begin, cudaStream_t st) {
    if (!n_pos) return;
    constexpr uint32_t nk = kNumCfg * kRectWidthClasses;
    uint64_t* start = static_cast<uint64_t*>(sort_scratch);
    uint32_t* hist = reinterpret_cast<uint32_t*>(start + nk);
    uint32_t* cursor = hist + nk;
    cudaMemsetAsync(hist, 0, 2 * nk * sizeof(uint32_t), st);
    k_rect_hist<<<(n_pos + 255) / 256, 256, 0, st>>>(order, n_pos, rect_flag, rect, hist);
    launch_scan_u32(hist, nk, start, bsum, total, st);
    k_rect_scatter<<<(n_pos + 255) / 256, 256, 0, st>>>(order, n_pos, rect_flag, rect, start, cursor, list, list_pos);
    k_rect_bounds<<<1, 64, 0, st>>>(start, total, rect_begin);
}

void launch_rect_plan(const sa_job* jobs, const uint32_t* order, uint32_t n_pos, const uint32_t* cfg_begin,
                      const JobState* state, const Score& sc, int32_t min_score, int allow_band,
                      Rect* rect, uint64_t* sizes, uint32_t* const* lists, uint32_t* cls_count,
                      uint32_t* rect_flag, int heights, const uint32_t* ref, const uint32_t* rpack, uint32_t rw,
                      cudaStream_t st) {
    if (!n_pos) return;
    BandLists bl;
    for (int k = 0; k < kNumBand; k++) bl.p[k] = lists[k];
    k_rect_plan<<<(n_pos + 255) / 256, 256, 0, st>>>(jobs, order, n_pos, cfg_begin, state, sc, min_score,
                                                      allow_band, rect, sizes, bl, cls_count, rect_flag,
                                                      heights, ref + kRefFrontPad, rpack, rw);
}

// wave assignment of the rectangle jobs (their positions in the bucketed order,
// list_pos[0 .. n)): a job belongs to the wave of its first direction word, so its
// words fit the arena slack (cap - wave words >= the largest job).
__global__ void k_rect_assign(const uint32_t* __restrict__ order, const uint32_t* __restrict__ list_pos,
                              uint32_t n, const uint64_t* __restrict__ offs, uint64_t wave_words,
                              Rect* __restrict__ rect, uint32_t* max_wave) {
    const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const uint32_t p = list_pos[q];
    const uint32_t job = order[p];
    const uint64_t wv = wave_words ? offs[p] / wave_words : 0;
    Rect R = rect[job];
    R.wave = (int)wv;
    R.off = offs[p] - wv * wave_words;
    rect[job] = R;
    atomicMax(max_wave, (uint32_t)wv);
}

void launch_rect_assign(const uint32_t* order, const uint32_t* list_pos, uint32_t n, const uint64_t* offs,
                        uint64_t wave_words, Rect* rect, uint32_t* max_wave, cudaStream_t st) {
    if (!n) return;
    k_rect_assign<<<(n + 255) / 256, 256, 0, st>>>(order, list_pos, n, offs, wave_words, rect, max_wave);
}

// ---------------------------------------------------------------------------
// exclusive scan of uint64 (or uint32 widened) values: block sums, scan of the
// block sums in one block, then per-block scan with the carried offset

constexpr int kScanBlock = 1024;

template <typename T>
__device__ __forceinline__ uint64_t block_excl_scan(uint64_t v, uint64_t* total) {
    __shared__ uint64_t warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        uint64_t s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) warp_sums[lane] = s;
    }
    __syncthreads();
    const uint64_t before = wid ? warp_sums[wid - 1] : 0;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

template <typename T>
__global__ void k_scan_reduce(const T* __restrict__ in, uint64_t n, uint64_t* __restrict__ bsum) {
    const uint64_t i = blockIdx.x * (uint64_t)kScanBlock + threadIdx.x;
    uint64_t v = i < n ? (uint64_t)in[i] : 0;
    uint64_t tot;
    block_excl_scan<T>(v, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_blocksums(uint64_t* __restrict__ bsum, uint32_t nb, uint64_t* total_out) {
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < nb; base += kScanBlock) {
        const uint32_t i = base + threadIdx.x;
        const uint64_t v = i < nb ? bsum[i] : 0;
        uint64_t tot;
        const uint64_t ex = block_excl_scan<uint64_t>(v, &tot);
        if (i < nb) bsum[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total_out = carry;
}

template <typename T>
__global__ void k_scan_apply(const T* __restrict__ in, uint64_t n, const uint64_t* __restrict__ bsum,
                             uint64_t* __restrict__ out) {
    const uint64_t i = blockIdx.x * (uint64_t)kScanBlock + threadIdx.x;
    uint64_t v = i < n ? (uint64_t)in[i] : 0;
    uint64_t tot;
    const uint64_t ex = block_excl_scan<T>(v, &tot);
    if (i < n) out[i] = bsum[blockIdx.x] + ex;
}

template <typename T>
static void scan_impl(const T* in, uint64_t n, uint64_t* out, uint64_t* bsum, uint64_t* total,
                      cudaStream_t st) {
    if (!n) {
        cudaMemsetAsync(total, 0, sizeof(uint64_t), st);
        return;
    }
    const uint32_t nb = (uint32_t)((n + kScanBlock - 1) / kScanBlock);
    k_scan_reduce<T><<<nb, kScanBlock, 0, st>>>(in, n, bsum);
    k_scan_blocksums<<<1, kScanBlock, 0, st>>>(bsum, nb, total);
    k_scan_apply<T><<<nb, kScanBlock, 0, st>>>(in, n, bsum, out);
}

void launch_scan_u64(const uint64_t* in, uint64_t n, uint64_t* out, uint64_t* bsum, uint64_t* total,
                     cudaStream_t st) {
    scan_impl<uint64_t>(in, n, out, bsum, total, st);
}
void launch_scan_u32(const uint32_t* in, uint64_t n, uint64_t* out, uint64_t* bsum, uint64_t* total,
                     cudaStream_t st) {
    scan_impl<uint32_t>(in, n, out, bsum, total, st);
}

// ---------------------------------------------------------------------------
// traceback: one thread per job, walking the direction nibbles of its rectangle
// (the same priority as the definition: stop > diagonal > D > I, gaps opened on
// ties, which the nibbles encode cell by cell).  Ops are written in reverse
// order, run-length merged, into the job's temporary slot.

__device__ __forceinline__ uint32_t nibble_at(const uint32_t* __restrict__ arena, uint64_t off,
                                              int L, int K, int pad, int i, int j) {
    const int idx = j - 1 + pad;
    const int g = idx / K, r = idx - g * K;
    const int s = i - 1 + g;                 // the step at which lane g computed column i
    const uint32_t word = arena[off + ((uint64_t)s * ((K + 7) / 8) + (r >> 3)) * L + g];
    return (word >> (4 * (r & 7))) & 15u;
}

__device__ __forceinline__ uint32_t band_nibble(const uint32_t* __restrict__ arena, uint64_t base,
                                                int W, int k, int j) {
    const uint32_t word = arena[base + ((uint64_t)(j - 1) * W + (k >> 3)) * 32];
    return (word >> (4 * (k & 7))) & 15u;
}

__global__ void k_traceback(const sa_job* __restrict__ jobs, uint32_t job_begin, uint32_t n_jobs,
                            const JobState* __restrict__ state, const Rect* __restrict__ rect,
                            const uint32_t* __restrict__ arena, BandLayout band, int wave, int mode,
                            int plain,
                            int cfg_force, int32_t min_score, uint32_t* __restrict__ tmp_ops,
                            uint32_t tmp_stride, TbOut* __restrict__ tb, unsigned* err_job,
                            HeightWalk hw, const uint32_t* __restrict__ list, int part) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= n_jobs) return;
    // part 0: every job; part 1: every job but the rectangle jobs' height walks;
    // part 2: only those walks, one thread per entry of the rectangle list (every
    // lane of a warp walks, and neighbouring entries have rectangles of about the
    // same size)
    const uint32_t job = list ? list[job_begin + tid] : job_begin + tid;
    const Rect R = rect[job];
    const int bidx = band_index(R.cls);
    const bool banded = bidx >= 0;
    TbOut out;
    out.n_rev = 0;
    out.read_begin = -1;
    out.ref_begin_rel = -1;
    if (R.cls == kClsDiag && !plain) {
        // gapless path: R.rows diagonal steps from (i*, j*) = (start_i, start_j)
        if (wave != 0 || part == 2) return;
        tmp_ops[(uint64_t)job * tmp_stride] = ((uint32_t)R.rows << 4) | 0u;
        out.n_rev = 1;
        out.read_begin = R.start_j - R.rows;
        out.ref_begin_rel = R.start_i - R.rows;
        tb[job] = out;
        return;
    }
    // banded jobs were walked by their band pass
    if (banded || R.w <= 0 || R.wave != wave) return;
    const JobState st = state[job];
    int si = R.start_i, sj = R.start_j;
    if (plain) {
        // whole-window direction bits: start at the best cell found by the same fill
        if ((st.flags & kStEmpty) || st.best < min_score) { tb[job] = out; return; }
        si = st.i_star;
        sj = st.j_star;
    }
    const int c = cfg_force >= 0 ? cfg_force : R.cfg;
    const int L = cfg_L(c), K = cfg_K(c);
    const int pad = (mode == SA_LOCAL) ? L * K - R.rows : 0;
    // banded jobs walk in window coordinates (start at the best cell, border at
    // column 0); rectangle jobs in rectangle coordinates (border at column 0 of
    // the rectangle, window column i_lo - 1)
    const int bw = banded ? band_width_of(bidx) : 0;
    const uint64_t bbase = banded ? band.base[bidx] + (uint64_t)(R.lpos >> 5) * band.warp_stride[bidx] + (R.lpos & 31u) : 0;
    if (banded) {
        si = st.i_star;
        sj = st.j_star;
    }
    const int imax_walk = banded ? st.i_star : R.w;
    const uint64_t off = R.off;
    if (part == 2 && !(hw.on && !plain)) return;
    if (hw.on && !banded && !plain) {
        if (part == 1) return;                       // walked by the list launch
        // byte heights of the rectangle (LOCAL, every score below 255); column 0 of
        // the rectangle (window column i_lo - 1) and row 0 are borders of value 0
        const sa_job J = jobs[job];
        const uint32_t* refw = hw.ref + kRefFrontPad;
        const uint32_t* rp = hw.rpack + (size_t)job * hw.rw;
        const int64_t col0 = (int64_t)J.ref_pos + R.i_lo - 2;     // reference position of rectangle column 0
        // row jj's lane g and row r in it (idx = jj - 1 + pad = g*K + r), kept for the
        // last row asked: the walk's scans stay on one row or move one row up
        int memo_j = -1, memo_g = 0, memo_r = 0;
        const int KH = (K + 3) / 4;
        auto height = [&](int ii, int jj) -> int32_t {
            if (ii < 0 || jj < 0 || ii > R.w || jj > R.rows) return kNeg32;
            if (ii == 0 || jj == 0) return 0;
            if (jj != memo_j) {
                if (jj == memo_j - 1) {
                    if (--memo_r < 0) { memo_r = K - 1; memo_g--; }
                } else {
                    const int idx = jj - 1 + pad;
                    memo_g = idx / K;
                    memo_r = idx - memo_g * K;
                }
                memo_j = jj;
            }
            const int s = ii - 1 + memo_g;       // the step at which lane g computed column ii
            const uint32_t word = arena[off + ((uint64_t)s * KH + (memo_r >> 2)) * L + memo_g];
            return (int32_t)((word >> (8 * (memo_r & 3))) & 255u);
        };
        auto match = [&](int ii, int jj) -> bool {
            const int64_t p = col0 + ii;
            const uint32_t t = (__ldg(refw + (p >> 4)) >> (2 * (p & 15))) & 3u;
            const uint32_t r = (__ldg(rp + ((jj - 1) >> 4)) >> (2 * ((jj - 1) & 15))) & 3u;
            return t == r;
        };
        const WalkEnd e = walk_heights(si, sj, st.best, R.w, R.rows, st.best, hw.sc.GO, hw.sc.GE, hw.sc.a,
                                       hw.sc.b, height, match, tmp_ops + (uint64_t)job * tmp_stride, tmp_stride);
        if (e.bad) {
            atomicMin(err_job, job);
            out.n_rev = 0;
            out.read_begin = 0;
            out.ref_begin_rel = 0;
        } else {
            out.n_rev = e.n_rev;
            out.read_begin = e.j;
            out.ref_begin_rel = (R.i_lo - 1) + e.i;
        }
        tb[job] = out;
        return;
    }
    auto nib_at = [&](int ii, int jj, bool* out_bad) -> uint32_t {
        if (banded) {
            const int k = ii - jj - R.d_lo;
            if (k < 0 || k >= bw) { *out_bad = true; return 0u; }
            return band_nibble(band.arena, bbase, bw / 8, k, jj);
        }
        return nibble_at(arena, off, L, K, pad, ii, jj);
    };
    const WalkEnd e = walk_nibbles(si, sj, imax_walk, R.rows, mode, nib_at,
                                   tmp_ops + (uint64_t)job * tmp_stride, tmp_stride);
    if (e.bad) {
        atomicMin(err_job, job);
        out.n_rev = 0;
        out.read_begin = 0;
        out.ref_begin_rel = 0;
        tb[job] = out;
        return;
    }
    out.n_rev = e.n_rev;
    out.read_begin = e.j;
    out.ref_begin_rel = banded ? e.i : (R.i_lo - 1) + e.i;
    tb[job] = out;
}

void launch_traceback(const sa_job* jobs, uint32_t job_begin, uint32_t n_jobs, const JobState* state,
                      const Rect* rect, const uint32_t* arena, const BandLayout& band, int wave,
                      int mode, int plain, int cfg_force, int32_t min_score, uint32_t* tmp_ops,
                      uint32_t tmp_stride, TbOut* tb, unsigned* err_job, const HeightWalk& hw,
                      cudaStream_t st, const uint32_t* list, int part) {
    if (!n_jobs) return;
    k_traceback<<<(n_jobs + 127) / 128, 128, 0, st>>>(jobs, job_begin, n_jobs, state, rect, arena,
                                                       band, wave, mode, plain, cfg_force, min_score,
                                                       tmp_ops, tmp_stride, tb, err_job, hw, list, part);
}

__global__ void k_iota(uint32_t* __restrict__ p, uint32_t n) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) p[k] = k;
}

void launch_iota(uint32_t* p, uint32_t n, cudaStream_t st) {
    if (!n) return;
    k_iota<<<(n + 255) / 256, 256, 0, st>>>(p, n);
}

// plain form: the whole window of every job of a batch, fixed stride per job
__global__ void k_plain_rect(const sa_job* __restrict__ jobs, uint32_t j0, uint32_t nb,
                             uint64_t stride, Rect* __restrict__ rect) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    const sa_job J = jobs[j0 + k];
    Rect R;
    R.off = (uint64_t)k * stride;
    R.i_lo = 1;
    R.w = (int)J.win_len;
    R.rows = (int)J.read_len;
    R.start_i = 0;
    R.start_j = 0;
    R.wave = 0;
    R.cls = kClsRect;
    R.d_lo = 0;
    R.lpos = 0;
    R.cfg = -1;
    rect[j0 + k] = R;
}

void launch_plain_rect(const sa_job* jobs, uint32_t j0, uint32_t nb, uint64_t stride, Rect* rect,
                       cudaStream_t st) {
    if (!nb) return;
    k_plain_rect<<<(nb + 255) / 256, 256, 0, st>>>(jobs, j0, nb, stride, rect);
}

// number of CIGAR ops of each job (soft clips included)
__global__ void k_cigar_count(const sa_job* __restrict__ jobs, uint32_t n_jobs,
                              const JobState* __restrict__ state, const TbOut* __restrict__ tb,
                              int mode, int want_cigar, int32_t min_score,
                              uint32_t* __restrict__ count) {
    const uint32_t job = blockIdx.x * blockDim.x + threadIdx.x;
    if (job >= n_jobs) return;
    const JobState st = state[job];
    uint32_t c = 0;
    const bool tb_done = want_cigar && !(st.flags & kStEmpty) && st.best >= min_score;
    if (tb_done) {
        const TbOut t = tb[job];
        c = (uint32_t)t.n_rev;
        if (mode == SA_LOCAL) {
            c += t.read_begin > 0 ? 1u : 0u;
            c += (int)jobs[job].read_len > st.j_star ? 1u : 0u;
        }
    }
    count[job] = c;
}

void launch_cigar_count(const sa_job* jobs, uint32_t n_jobs, const JobState* state, const TbOut* tb,
                        int mode, int want_cigar, int32_t min_score, uint32_t* count,
                        cudaStream_t st) {
    if (!n_jobs) return;
    k_cigar_count<<<(n_jobs + 255) / 256, 256, 0, st>>>(jobs, n_jobs, state, tb, mode, want_cigar,
                                                         min_score, count);
}

__global__ void k_finalize(const sa_job* __restrict__ jobs, uint32_t n_jobs,
                           const JobState* __restrict__ state, const TbOut* __restrict__ tb,
                           const uint32_t* __restrict__ count, const uint64_t* __restrict__ coff,
                           const uint32_t* __restrict__ tmp_ops, uint32_t tmp_stride, int mode,
                           int want_cigar, int32_t min_score, sa_result* __restrict__ out,
                           uint32_t* __restrict__ cigar) {
    const uint32_t job = blockIdx.x * blockDim.x + threadIdx.x;
    if (job >= n_jobs) return;
    const sa_job J = jobs[job];
    const JobState st = state[job];
    sa_result r = score_result(J, st, min_score);
    r.cigar_off = (uint32_t)coff[job];
    r.cigar_len = count[job];
    if (!(st.flags & kStEmpty)) {
        const bool tb_done = want_cigar && st.best >= min_score;
        if (tb_done) {
            const TbOut t = tb[job];
            r.read_begin = t.read_begin;
            r.ref_begin = (int64_t)J.ref_pos + t.ref_begin_rel;
            uint32_t* o = cigar + coff[job];
            int k = 0;
            if (mode == SA_LOCAL && t.read_begin > 0) o[k++] = ((uint32_t)t.read_begin << 4) | 4u;
            const uint32_t* src = tmp_ops + (uint64_t)job * tmp_stride;
            for (int q = t.n_rev - 1; q >= 0; q--) o[k++] = src[q];
            if (mode == SA_LOCAL && (int)J.read_len > st.j_star)
                o[k++] = ((uint32_t)(J.read_len - st.j_star) << 4) | 4u;
        }
    }
    out[job] = r;
}

void launch_finalize(const sa_job* jobs, uint32_t n_jobs, const JobState* state, const TbOut* tb,
                     const uint32_t* count, const uint64_t* coff, const uint32_t* tmp_ops,
                     uint32_t tmp_stride, int mode, int want_cigar, int32_t min_score,
                     sa_result* out, uint32_t* cigar, cudaStream_t st) {
    if (!n_jobs) return;
    k_finalize<<<(n_jobs + 255) / 256, 256, 0, st>>>(jobs, n_jobs, state, tb, count, coff, tmp_ops,
                                                      tmp_stride, mode, want_cigar, min_score, out,
                                                      cigar);
}

}  // namespace sa
