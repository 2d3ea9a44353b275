// Score pass in 16-bit packed pairs (LOCAL): two jobs per lane group, job A in
// the low and job B in the high half of every register, updated together with
// the DPX s16x2 max/add instructions.
//
// Representation: every H, E, F value x is stored as x + beta with beta = -S_GO
// (= o + e), and H additionally carries + S_GO (as in the 32-bit kernel), so the
// recurrence of SOAP3-dp Methods section 3 becomes, per half,
//   G  = max(HG(i-1,j-1) + (delta - S_GO), beta)      zero floor of LOCAL folded in
//   E  = max(E(i,j-1) + S_GE, HG(i,j-1))
//   F  = max(F(i-1,j) + S_GE, HG(i-1,j))
//   H  = max(G, E, F),   HG = H + S_GO
// Every stored H is >= beta, so HG = H + S_GO on both halves is one 32-bit
// multiply-add with a fixed carry compensation (the FMA pipe), the border values
// (H = 0 -> HG = 0, E = F = -inf -> 0) are all zero, and all maxima are signed
// 16-bit DPX operations.
//
// Best cell: each cell's key (H + beta) * 32 + (31 - r) (r the row in the lane)
// is formed with one multiply-add on both halves; a lane keeps the maximum key of
// its rows per column (the largest H and, among equal H, the first row), stores
// it at every step (one 128-byte line per warp and step) and passes it down the
// group, whose last lane stores the group's column maximum.  The epilogue finds
// the first column i* holding the largest H from the group's column maxima and
// the first row from the lanes' stored keys of column i*.  (Storing only where a
// lane's key rises leaves partial sectors that cost the same DRAM traffic as
// whole lines, plus the rise test on the ALU pipe.)
//
// Exact overflow detection: keys are exact while H + beta <= 1023.  A cell's H
// is at most its diagonal predecessor + a, so while every H + beta so far is
// below 1024 - a the next one is at most 1023; the first H that reaches the
// threshold is therefore exact and shows up in the column maxima.  A pair in
// which either job's maximum (over every column the pair computed) reaches it is
// flagged (kStOverflow) and both jobs are recomputed by the 32-bit kernel (past
// the threshold the low half's key can carry into the high half).
#pragma once

#include "fill.cuh"

namespace sa {

// words of the per-lane 16-bit profile (two jobs x 4 bases x rows rounded up to 4)
template <int K>
constexpr int prof16_words_per_warp() { return 2 * 4 * ((K + 3) / 4) * 2 * 32; }

__device__ __forceinline__ uint32_t pack2(int32_t lo, int32_t hi) {
    return ((uint32_t)lo & 0xFFFFu) | ((uint32_t)hi << 16);
}
__device__ __forceinline__ int32_t lo16(uint32_t v) { return (int32_t)(int16_t)(v & 0xFFFFu); }
__device__ __forceinline__ int32_t hi16(uint32_t v) { return (int32_t)(int16_t)(v >> 16); }
__device__ __forceinline__ int32_t half16(uint32_t v, int h) { return h ? hi16(v) : lo16(v); }

template <int L, int K>
__global__ void __launch_bounds__(128) k_fill16(FillArgs A) {
    static_assert(32 % L == 0, "L must divide 32");
    static_assert(K <= 32, "row tags are 5 bits");
    constexpr int G = 32 / L;              // groups per warp, 2 jobs per group
    constexpr int K4 = (K + 3) / 4;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int g = lane % L;
    const int grp = lane / L;
    const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int64_t cb_base = (int64_t)(gwarp * G + grp) * A.cb_stride + kCbFront;   // column 1's slot
    uint32_t* cb = reinterpret_cast<uint32_t*>(A.colbest) + cb_base;
    const uint64_t lk_base = (uint64_t)gwarp * A.lk_stride + lane;
    uint32_t* lk = A.lane_keys + lk_base;
    const Score S = A.sc;
    const uint32_t count = A.count_ptr ? *A.count_ptr : A.pos_count;
    extern __shared__ __align__(16) int32_t s_prof[];
    int32_t* prof = s_prof + (threadIdx.x >> 5) * prof16_words_per_warp<K>();
    const uint32_t one = blockDim.x >> 7;               // 1 at run time
    const uint32_t nf = g != 0 ? one : 0u;              // lane 0 takes the zero border
    const int32_t beta = -S.GO;
    const uint32_t GE2 = pack2(S.GE, S.GE);
    const uint32_t BETA2 = pack2(beta, beta);
    // H + S_GO on both halves as one 32-bit add: with S_GO < 0 the low half always
    // carries (every stored H is >= beta = -S_GO), so the high half's constant is
    // S_GO - 1; with S_GO = 0 there is nothing to add
    const uint32_t GO2C = S.GO == 0 ? 0u : (((uint32_t)S.GO & 0xFFFFu) + ((uint32_t)(S.GO - 1) << 16));
    const int32_t thr = 1024 - S.a;                      // biased overflow threshold

    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(A.item_counter, 1u);
        item = __shfl_sync(FULL, item, 0);
        if (item * (uint32_t)(2 * G) >= count) break;
        uint32_t jobv[2];
        int n[2] = {0, 0}, w[2] = {0, 0};
        int64_t wstart[2] = {0, 0};
        bool has[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const uint32_t p = item * (2 * G) + 2 * grp + h;
            has[h] = p < count;
            jobv[h] = has[h] ? __ldg(A.order + A.pos_begin + p) : 0u;
            if (has[h]) {
                const sa_job J = A.jobs[jobv[h]];
                n[h] = (int)J.read_len;
                w[h] = (int)J.win_len;
                wstart[h] = (int64_t)J.ref_pos;
            }
        }
        const int wmax = max(w[0], w[1]);
        const int nblk = wmax > 0 ? (wmax + L - 1 + 7) >> 3 : 0;
        int nblk_warp = nblk;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) nblk_warp = max(nblk_warp, __shfl_xor_sync(FULL, nblk_warp, o));
        if (nblk_warp == 0) continue;

        // profile: entry ((h*4 + t)*K4 + r/4)*32 + lane (4 x int16 in a uint2) holds
        // (delta - S_GO) of rows r..r+3 of job h against base t; padding rows never
        // match.  Written and read through the same uint2 type, so the reads of the
        // next job cannot be ordered before these stores.
        int pad[2];
        uint2* prof2 = reinterpret_cast<uint2*>(prof);
#pragma unroll
        for (int h = 0; h < 2; h++) {
            pad[h] = L * K - n[h];
            const uint32_t* rp = A.rpack + (size_t)jobv[h] * A.rw;
#pragma unroll
            for (int q = 0; q < K4; q++) {
                int code[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int r = 4 * q + u;
                    const int j = g * K + r + 1 - pad[h];
                    code[u] = -1;
                    if (r < K && w[h] > 0 && j >= 1 && j <= n[h])
                        code[u] = (int)((__ldg(rp + ((j - 1) >> 4)) >> (2 * ((j - 1) & 15))) & 3u);
                }
#pragma unroll
                for (int t = 0; t < 4; t++) {
                    uint2 v;
                    v.x = pack2(code[0] == t ? S.dm : S.dx, code[1] == t ? S.dm : S.dx);
                    v.y = pack2(code[2] == t ? S.dm : S.dx, code[3] == t ? S.dm : S.dx);
                    prof2[((h * 4 + t) * K4 + q) * 32 + lane] = v;
                }
            }
        }

        // order the profile stores before this item's loads (each lane reads only
        // its own entries; with the barrier the result no longer depended on code
        // generation, see the design notes)
        __syncwarp();
        // column 0: H(0,j) = 0 -> HG = 0; F = -inf -> 0
        uint32_t HG[K], F[K];
        auto reset_col0 = [&]() {
#pragma unroll
            for (int r = 0; r < K; r++) { HG[r] = 0u; F[r] = 0u; }
        };
        reset_col0();
        uint32_t h_up_prev = 0u;
        uint32_t hg_bot = 0u, e_bot = 0u, cm_bot = 0u;

        uint32_t wbn[2];
#pragma unroll
        for (int h = 0; h < 2; h++) wbn[h] = load_window16<L, K>(A, wstart[h], 0, g);
        for (int b = 0; b < nblk_warp; b++) {
            uint32_t wb[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                wb[h] = wbn[h];
                wbn[h] = load_window16<L, K>(A, wstart[h], b + 1, g);
            }
#pragma unroll
            for (int u = 0; u < 8; u++) {
                const int s = 8 * b + u;
                const int i = s - g + 1;
                // lane 0: the border (every border value is 0 in this representation)
                const uint32_t hg_up = __shfl_up_sync(FULL, hg_bot, 1, L) * nf;
                const uint32_t e_up = __shfl_up_sync(FULL, e_bot, 1, L) * nf;
                const uint32_t cm_up = __shfl_up_sync(FULL, cm_bot, 1, L) * nf;
                const uint32_t diag = h_up_prev;
                h_up_prev = hg_up;
                const uint32_t tA = (wb[0] >> (2 * u)) & 3u, tB = (wb[1] >> (2 * u)) & 3u;
                const uint2* pa = prof2 + (tA * K4) * 32 + lane;
                const uint2* pb = prof2 + ((4 + tB) * K4) * 32 + lane;
                uint2 qa = pa[0], qb = pb[0];
                uint32_t e = e_up, hga = hg_up;
                uint32_t lm = 0u, kpair = 0u;
                // the diagonal term of row r+1 is formed while row r still holds
                // H(i-1, j) (no copy of the old value is kept)
                uint32_t gcur = __viaddmax_s16x2(diag, __byte_perm(qa.x, qb.x, 0x5410), BETA2);
#pragma unroll
                for (int r = 0; r < K; r++) {
                    const uint32_t gv = gcur;                                  // max(G, 0) + beta
                    if (r + 1 < K) {
                        const int rn = r + 1;
                        if ((rn & 3) == 0) { qa = pa[(rn / 4) * 32]; qb = pb[(rn / 4) * 32]; }
                        const uint32_t xa = (rn & 2) ? qa.y : qa.x, xb = (rn & 2) ? qb.y : qb.x;
                        const uint32_t dn = __byte_perm(xa, xb, (rn & 1) ? 0x7632 : 0x5410);
                        gcur = __viaddmax_s16x2(HG[r], dn, BETA2);
                    }
                    const uint32_t f = __viaddmax_s16x2(F[r], GE2, HG[r]);
                    e = __viaddmax_s16x2(e, GE2, hga);
                    const uint32_t hv = __vimax3_s16x2(gv, e, f);
                    F[r] = f;
                    HG[r] = hv * one + GO2C;
                    hga = HG[r];
                    // key of both halves; no carry while H + beta <= 1023
                    const uint32_t key = hv * (32u * one) + (uint32_t)(31 - r) * 0x10001u;
                    if ((r & 1) == 1) lm = __vimax3_s16x2(lm, kpair, key);
                    else if (r == K - 1) lm = __vimax3_s16x2(lm, key, key);
                    else kpair = key;
                }
                hg_bot = HG[K - 1];
                e_bot = e;
                const uint32_t cm = __vimax3_s16x2(cm_up, lm, lm);
                cm_bot = cm;
                // steps outside the windows land in slack slots / are never read
                if (g == L - 1 && SA_GUARD((uint64_t)(cb_base + i - 1) < A.cb_cap, A.dbg, kSiteCb16)) cb[i - 1] = cm;
                if (SA_GUARD(lk_base + (uint64_t)s * 32 < A.lk_cap, A.dbg, kSiteLaneKeys)) lk[(size_t)s * 32] = lm;
                if (8 * b < L && s < g) {      // before this lane's first column
                    reset_col0();
                    h_up_prev = 0u;
                }
            }
        }

        // per job of the pair: best, second best, overflow flag
        __syncwarp();
        int32_t cmax = 0;
        for (int ii = g + 1; ii <= wmax; ii += L) {
            const uint32_t c2 = cb[ii - 1];
            cmax = max(cmax, max(hi16(c2), lo16(c2)) >> 5);
        }
#pragma unroll
        for (int o = 1; o < L; o <<= 1) cmax = max(cmax, __shfl_xor_sync(FULL, cmax, o, L));
        const bool ovf = cmax >= thr;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            // first column holding the largest H
            int32_t v = -1;
            int vi = 0;
            for (int ii = g + 1; ii <= w[h]; ii += L) {
                const int32_t x = half16(cb[ii - 1], h) >> 5;
                if (x > v) { v = x; vi = ii; }
            }
#pragma unroll
            for (int o = 1; o < L; o <<= 1) {
                const int32_t ov = __shfl_xor_sync(FULL, v, o, L);
                const int oi = __shfl_xor_sync(FULL, vi, o, L);
                if (ov > v || (ov == v && oi < vi)) { v = ov; vi = oi; }
            }
            const bool empty = v <= beta;
            // first row of that column: the lanes' stored keys of column vi
            int vj = 1 << 20;
            if (vi > 0) {
                const int32_t k = half16(lk[(size_t)(vi + g - 1) * 32], h);
                if ((k >> 5) == v) vj = g * K + (31 - (k & 31)) + 1 - pad[h];
            }
#pragma unroll
            for (int o = 1; o < L; o <<= 1) vj = min(vj, __shfl_xor_sync(FULL, vj, o, L));
            // second best: colbest(i) over columns at least n away from the best
            int32_t sv = 0;
            int si = 0;
            const int wsec = empty ? 0 : w[h];
            for (int ii = g + 1; ii <= wsec; ii += L) {
                const int dd = ii > vi ? ii - vi : vi - ii;
                if (dd < n[h]) continue;
                const int32_t x = half16(cb[ii - 1], h) >> 5;
                if (si == 0 || x > sv) { sv = x; si = ii; }
            }
#pragma unroll
            for (int o = 1; o < L; o <<= 1) {
                const int32_t ov = __shfl_xor_sync(FULL, sv, o, L);
                const int oi = __shfl_xor_sync(FULL, si, o, L);
                if (oi != 0 && (si == 0 || ov > sv || (ov == sv && oi < si))) { sv = ov; si = oi; }
            }
            if (g == 0 && has[h]) {
                JobState st;
                st.best = empty ? 0 : v - beta;
                st.i_star = empty ? 0 : vi;
                st.j_star = empty ? 0 : vj;
                st.second = (empty || si == 0) ? SA_NO_SCORE : sv - beta;
                st.second_i = empty ? 0 : si;
                st.flags = (empty ? kStEmpty : 0u) | (ovf ? kStOverflow : 0u);
                if (SA_GUARD(jobv[h] < A.n_state, A.dbg, kSiteState16)) A.state[jobv[h]] = st;
            }
        }
        __syncwarp();
    }
}

}  // namespace sa
