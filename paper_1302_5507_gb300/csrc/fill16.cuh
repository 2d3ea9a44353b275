// Score pass in 16-bit packed pairs (LOCAL): two jobs per lane group, job A in
// the low and job B in the high half of every register, updated together with
// the DPX s16x2 max/add instructions.
//
// Representation: every value is scaled by 32, so its low 5 bits are zero and a
// row tag fits below it in the best-cell keys.  With beta = o + e (= -S_GO),
// B = max(beta, mismatch) and c = 32 (B - beta) (0 unless the mismatch costs
// more than opening a gap), a half holds
//   X = 32 H + c                                  (H >= 0 in LOCAL)
//   E~ = 32 (E + B),  F~ = 32 (F + B),  G~ = 32 (H(i-1,j-1) + delta + B)
// and the recurrence of SOAP3-dp Methods section 3 becomes, per half,
//   G~ = X(i-1,j-1) + 32 (delta - S_GO)
//   E~ = max(E~(i,j-1) + 32 S_GE, X(i,j-1))
//   F~ = max(F~(i-1,j) + 32 S_GE, X(i-1,j))
//   X  = max(G~, E~, F~) + 32 S_GO                 G~ floored at 32 B: the zero floor of LOCAL
// The borders are X = c (H = 0) and E~ = F~ = 0 (E = F = -B, below every
// H + S_GO), and every value is >= 0.
//
// Diagonal term: a byte permute pairs the two jobs' 16-bit profile entries, and
// G~ = max(X(i-1,j-1) + 32 (delta - S_GO), 32 B) takes the zero floor; then
// X = max(G~, E~, F~) + 32 S_GO is one 32-bit multiply-add on both halves with a
// fixed carry compensation (every H~ >= 32 B >= 32 beta, so the low half always
// carries).  (A form that keeps 32-bit profile entries and forms G~ of both halves
// with one three-input add, the floor moved to X, needs twice the shared memory;
// at the resulting occupancy it was slower.)
//
// Best cell: a cell's key is X + (31 - r) (r the row in the lane), formed and
// folded into the lane's running maximum with one DPX add-max a row; a lane keeps
// the maximum key of its rows per column (the largest H and, among equal H, the
// first row), stores it at every step (one 128-byte line per warp and step) and
// passes it down the group, whose last lane stores the group's column maximum.
// The epilogue finds the first column i* holding the largest H from the group's
// column maxima and the first row from the lanes' stored keys of column i*.
// (Storing only where a lane's key rises leaves partial sectors that cost the
// same DRAM traffic as whole lines, plus the rise test on the ALU pipe.)
//
// Exact overflow detection: values are exact while H + B <= 1023 (32 (H + B) <
// 2^15).  A cell's H is at most its diagonal predecessor + a, so while every
// H + B so far is below 1024 - a the next one is at most 1023; the first H that
// reaches the threshold is therefore exact and shows up in the column maxima.  A
// pair in which either job's maximum (over every column the pair computed)
// reaches it is flagged (kStOverflow) and both jobs are recomputed by the 32-bit
// kernel (past the threshold one half can carry into the other).  The host runs
// this pass only for schemes with a + B < 1024.
#pragma once

#include "fill.cuh"


namespace sa {

// words of the per-lane 16-bit profile of a warp (two jobs x 4 bases x rows
// rounded up to 4)
template <int K>
constexpr int prof16_words_per_warp() { return 2 * 4 * ((K + 3) / 4) * 2 * 32; }

__device__ __forceinline__ uint32_t pack2(int32_t lo, int32_t hi) {
    return ((uint32_t)lo & 0xFFFFu) | ((uint32_t)hi << 16);
}
__device__ __forceinline__ int32_t lo16(uint32_t v) { return (int32_t)(int16_t)(v & 0xFFFFu); }
__device__ __forceinline__ int32_t hi16(uint32_t v) { return (int32_t)(int16_t)(v >> 16); }
__device__ __forceinline__ int32_t half16(uint32_t v, int h) { return h ? hi16(v) : lo16(v); }

// resident 128-thread blocks a SM asked of the register allocator: rows 25-28
// then fit four blocks in 128 registers (their profiles take 56 KB a block);
// elsewhere (0: no request) the allocator's own choice reaches the same occupancy
// with a faster schedule
template <int K>
constexpr int fill16_min_blocks() { return (K >= 25 && K <= 28) ? 4 : 0; }

template <int L, int K>
__global__ void __launch_bounds__(128, fill16_min_blocks<K>()) k_fill16(FillArgs A) {
    // steps a loop body and the unrolling of the per-item profile loop: past 16 rows
    // the eight-step body and the per-item code (profile, epilogue) do not fit the
    // instruction cache together (warps that change items often, short windows,
    // stalled on instruction fetch), so the body takes four steps and the profile
    // loop stays rolled
    constexpr int kStepUnroll = K <= 16 ? 8 : 4;
    constexpr int kProfUnroll = K <= 16 ? (K + 3) / 4 : 1;
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
    const uint32_t nf = g != 0 ? one : 0u;              // lane 0 takes the border
    const int32_t beta = -S.GO;
    const int32_t cH = max(0, -S.dx);                   // B - beta
    const uint32_t C2 = pack2(32 * cH, 32 * cH);        // X of H = 0
    const uint32_t x_border = g != 0 ? 0u : C2;
    const uint32_t GE2 = pack2(32 * S.GE, 32 * S.GE);
    const uint32_t FLG2 = pack2(32 * (beta + cH), 32 * (beta + cH));   // G~ of H = 0: the floor
    // X = G~ - 32 beta on both halves as one 32-bit add: the low half always
    // carries (G~ >= 32 B >= 32 beta), so the high half's constant is one less
    const uint32_t GO2C = beta == 0 ? 0u : (((uint32_t)(-32 * beta) & 0xFFFFu) + ((uint32_t)(-32 * beta - 1) << 16));
    const int32_t thr = 1024 - S.a - beta;              // overflow: (key >> 5) = H + B - beta reaches it

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
        // 32 (delta - S_GO) of rows r..r+3 of job h against base t; padding rows
        // never match.  Written and read through the same uint2 type, so the reads
        // of the next job cannot be ordered before these stores.
        int pad[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            pad[h] = L * K - n[h];
            const uint32_t* rp = A.rpack + (size_t)jobv[h] * A.rw;
#pragma unroll kProfUnroll
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
                    const int32_t e0 = 32 * (code[0] == t ? S.dm : S.dx), e1 = 32 * (code[1] == t ? S.dm : S.dx);
                    const int32_t e2 = 32 * (code[2] == t ? S.dm : S.dx), e3 = 32 * (code[3] == t ? S.dm : S.dx);
                    uint2 v;
                    v.x = pack2(e0, e1);
                    v.y = pack2(e2, e3);
                    reinterpret_cast<uint2*>(prof)[((h * 4 + t) * K4 + q) * 32 + lane] = v;
                }
            }
        }

        // order the profile stores before this item's loads (each lane reads only
        // its own entries; with the barrier the result no longer depended on code
        // generation, see the design notes)
        __syncwarp();
        // column 0: X = c (H = 0), F~ = 0
        uint32_t X[K], F[K];
        auto reset_col0 = [&]() {
#pragma unroll
            for (int r = 0; r < K; r++) { X[r] = C2; F[r] = 0u; }
        };
        reset_col0();
        uint32_t x_up_prev = C2;
        uint32_t x_bot = 0u, e_bot = 0u, cm_bot = 0u;

        // one wavefront step: lane g computes column i = s - g + 1 of its K rows
        // against window base tA (job A) and tB (job B)
        auto step = [&](const int s, const uint32_t tA, const uint32_t tB, const bool first_block) {
            const int i = s - g + 1;
            // lane 0: the border (X = c, E~ = 0, no key)
            const uint32_t x_up = __shfl_up_sync(FULL, x_bot, 1, L) * nf + x_border;
            const uint32_t e_up = __shfl_up_sync(FULL, e_bot, 1, L) * nf;
            const uint32_t cm_up = __shfl_up_sync(FULL, cm_bot, 1, L) * nf;
            const uint32_t diag = x_up_prev;
            x_up_prev = x_up;
            uint32_t e = e_up, xa = x_up, lm = 0u;
            // the diagonal term of row r+1 is formed while X[r] still holds X(i-1, j)
            // (no copy of the old value stays live)
            {
                const uint2* pa = reinterpret_cast<const uint2*>(prof) + (tA * K4) * 32 + lane;
                const uint2* pb = reinterpret_cast<const uint2*>(prof) + ((4 + tB) * K4) * 32 + lane;
                uint2 qa = pa[0], qb = pb[0];
                uint32_t gcur = __viaddmax_s16x2(diag, __byte_perm(qa.x, qb.x, 0x5410), FLG2);
#pragma unroll
                for (int r = 0; r < K; r++) {
                    const uint32_t gv = gcur;
                    if (r + 1 < K) {
                        const int rn = r + 1;
                        if ((rn & 3) == 0) { qa = pa[(rn / 4) * 32]; qb = pb[(rn / 4) * 32]; }
                        const uint32_t xa2 = (rn & 2) ? qa.y : qa.x, xb2 = (rn & 2) ? qb.y : qb.x;
                        const uint32_t dn = __byte_perm(xa2, xb2, (rn & 1) ? 0x7632 : 0x5410);
                        gcur = __viaddmax_s16x2(X[r], dn, FLG2);
                    }
                    const uint32_t f = __viaddmax_s16x2(F[r], GE2, X[r]);
                    e = __viaddmax_s16x2(e, GE2, xa);
                    const uint32_t hv = __vimax3_s16x2(gv, e, f);
                    F[r] = f;
                    X[r] = hv * one + GO2C;
                    xa = X[r];
                    lm = __viaddmax_s16x2(X[r], (uint32_t)(31 - r) * 0x10001u, lm);
                }
            }
            x_bot = X[K - 1];
            e_bot = e;
            const uint32_t cm = __vimax3_s16x2(cm_up, lm, lm);
            cm_bot = cm;
            // steps outside the windows land in slack slots / are never read
            if (g == L - 1 && SA_GUARD((uint64_t)(cb_base + i - 1) < A.cb_cap, A.dbg, kSiteCb16)) cb[i - 1] = cm;
            if (SA_GUARD(lk_base + (uint64_t)s * 32 < A.lk_cap, A.dbg, kSiteLaneKeys)) lk[(size_t)s * 32] = lm;
            if (first_block && s < g) {       // before this lane's first column
                reset_col0();
                x_up_prev = C2;
            }
        };

        uint32_t wbn[2];
#pragma unroll
        for (int h = 0; h < 2; h++) wbn[h] = load_window16<L, K>(A, wstart[h], 0, g);
        // the first blocks (steps s < L), where lanes before their first column keep
        // resetting it, run one step a loop body; the rest of the item runs without the
        // reset, so no step of the main loop joins two definitions of X and F (which
        // cost a register move a row)
        int b = 0;
        for (; b < nblk_warp && 8 * b < L; b++) {
            uint32_t wb[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                wb[h] = wbn[h];
                wbn[h] = load_window16<L, K>(A, wstart[h], b + 1, g);
            }
#pragma unroll 1
            for (int u = 0; u < 8; u++) step(8 * b + u, (wb[0] >> (2 * u)) & 3u, (wb[1] >> (2 * u)) & 3u, true);
        }
        for (; b < nblk_warp; b++) {
            uint32_t wb[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                wb[h] = wbn[h];
                wbn[h] = load_window16<L, K>(A, wstart[h], b + 1, g);
            }
#pragma unroll kStepUnroll
            for (int u = 0; u < 8; u++) step(8 * b + u, (wb[0] >> (2 * u)) & 3u, (wb[1] >> (2 * u)) & 3u, false);
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
            const bool empty = v <= cH;        // H = 0 everywhere
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
                st.best = empty ? 0 : v - cH;
                st.i_star = empty ? 0 : vi;
                st.j_star = empty ? 0 : vj;
                st.second = (empty || si == 0) ? SA_NO_SCORE : sv - cH;
                st.second_i = empty ? 0 : si;
                st.flags = (empty ? kStEmpty : 0u) | (ovf ? kStOverflow : 0u);
                if (SA_GUARD(jobv[h] < A.n_state, A.dbg, kSiteState16)) A.state[jobv[h]] = st;
            }
        }
        __syncwarp();
    }
}

}  // namespace sa
