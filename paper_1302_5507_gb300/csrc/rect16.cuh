// Wavefront rectangle pass in 16-bit packed pairs (byte heights); the score
// pass's kernel and helpers are in fill16.cuh.
#pragma once

#include "fill16.cuh"

namespace sa {

// Rectangle pass in 16-bit packed pairs with byte heights (LOCAL, every score
// below 255): the direction data of two wavefront-rectangle jobs per lane group,
// the same wavefront, profile and byte permute as the score pass, without keys
// or column maxima.  Values are not scaled: with B' the smallest multiple of 256
// that is >= max(beta, mismatch), a half holds X = H + B' - beta, E~ = E + B',
// F~ = F + B' and H~ = H + B' (G~ floored at B'), so the low byte of each half of
// H~ is the cell's height, which the walk reads back (every value stays below
// 2^15 for the schemes the API takes).  Each job's heights go to its own arena
// range in the layout of the 32-bit pass (word k of lane g at step s:
// off + (s * KH + k) * L + g, byte r & 3 of word r / 4 for row r), only for the
// blocks of its own rectangle.
template <int L, int K>
__global__ void __launch_bounds__(128) k_fill16h(FillArgs A) {
    static_assert(32 % L == 0, "L must divide 32");
    constexpr int G = 32 / L;
    constexpr int K4 = (K + 3) / 4;
    constexpr int KH = (K + 3) / 4;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int g = lane % L;
    const int grp = lane / L;
    const Score S = A.sc;
    const uint32_t count = A.count_ptr ? *A.count_ptr : A.pos_count;
    extern __shared__ __align__(16) int32_t s_prof[];
    int32_t* prof = s_prof + (threadIdx.x >> 5) * prof16_words_per_warp<K>();
    const uint32_t one = blockDim.x >> 7;               // 1 at run time
    const uint32_t nf = g != 0 ? one : 0u;              // lane 0 takes the border
    const int32_t beta = -S.GO;
    const int32_t Bp = ((max(beta, -S.b) + 255) >> 8) << 8;   // B'
    const uint32_t C2 = pack2(Bp - beta, Bp - beta);    // X of H = 0
    const uint32_t x_border = g != 0 ? 0u : C2;
    const uint32_t GE2 = pack2(S.GE, S.GE);
    const uint32_t FLG2 = pack2(Bp, Bp);                // G~ of H = 0: the floor
    // X = H~ - beta on both halves as one 32-bit add (H~ >= B' >= beta: the low
    // half always carries)
    const uint32_t GO2C = beta == 0 ? 0u : (((uint32_t)(-beta) & 0xFFFFu) + ((uint32_t)(-beta - 1) << 16));

    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(A.item_counter, 1u);
        item = __shfl_sync(FULL, item, 0);
        if (item * (uint32_t)(2 * G) >= count) break;
        uint32_t jobv[2];
        int rows[2] = {0, 0}, w[2] = {0, 0}, nblk[2] = {0, 0};
        int64_t wstart[2] = {0, 0};
        uint64_t aoff[2] = {0, 0};
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const uint32_t p = item * (2 * G) + 2 * grp + h;
            jobv[h] = p < count ? __ldg(A.order + A.pos_begin + p) : 0u;
            if (p < count) {
                const Rect R = A.rect[jobv[h]];
                if (R.w > 0 && R.wave == A.wave) {
                    rows[h] = R.rows;
                    w[h] = R.w;
                    wstart[h] = (int64_t)A.jobs[jobv[h]].ref_pos + R.i_lo - 1;
                    aoff[h] = R.off;
                    nblk[h] = (w[h] + L - 1 + 7) >> 3;
                }
            }
        }
        int nblk_warp = max(nblk[0], nblk[1]);
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) nblk_warp = max(nblk_warp, __shfl_xor_sync(FULL, nblk_warp, o));
        if (nblk_warp == 0) continue;

        // profile of both jobs' rows (rows padded at the top never match), as in the
        // score pass but unscaled
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int pad = L * K - rows[h];
            const uint32_t* rp = A.rpack + (size_t)jobv[h] * A.rw;
#pragma unroll
            for (int q = 0; q < K4; q++) {
                int code[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int r = 4 * q + u;
                    const int j = g * K + r + 1 - pad;
                    code[u] = -1;
                    if (r < K && w[h] > 0 && j >= 1 && j <= rows[h])
                        code[u] = (int)((__ldg(rp + ((j - 1) >> 4)) >> (2 * ((j - 1) & 15))) & 3u);
                }
#pragma unroll
                for (int t = 0; t < 4; t++) {
                    uint2 v;
                    v.x = pack2(code[0] == t ? S.dm : S.dx, code[1] == t ? S.dm : S.dx);
                    v.y = pack2(code[2] == t ? S.dm : S.dx, code[3] == t ? S.dm : S.dx);
                    reinterpret_cast<uint2*>(prof)[((h * 4 + t) * K4 + q) * 32 + lane] = v;
                }
            }
        }
        __syncwarp();
        uint32_t X[K], F[K];
        auto reset_col0 = [&]() {
#pragma unroll
            for (int r = 0; r < K; r++) { X[r] = C2; F[r] = 0u; }
        };
        reset_col0();
        uint32_t x_up_prev = C2;
        uint32_t x_bot = 0u, e_bot = 0u;

        auto step = [&](const int b, const int s, const uint32_t tA, const uint32_t tB, const bool first_block) {
            const uint32_t x_up = __shfl_up_sync(FULL, x_bot, 1, L) * nf + x_border;
            const uint32_t e_up = __shfl_up_sync(FULL, e_bot, 1, L) * nf;
            const uint32_t diag = x_up_prev;
            x_up_prev = x_up;
            uint32_t e = e_up, xa = x_up;
            uint32_t hq[4] = {0u, 0u, 0u, 0u};           // H~ of the current four rows
            uint32_t wa[KH], wbk[KH];
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
                hq[r & 3] = hv;
                if ((r & 3) == 3 || r == K - 1) {
                    // the low bytes of the four rows' halves: job A's and job B's words
                    const uint32_t p01 = __byte_perm(hq[0], hq[1], 0x6240);   // A0 A1 B0 B1
                    const uint32_t p23 = __byte_perm(hq[2], hq[3], 0x6240);   // A2 A3 B2 B3
                    wa[r >> 2] = __byte_perm(p01, p23, 0x5410);
                    wbk[r >> 2] = __byte_perm(p01, p23, 0x7632);
                    hq[0] = hq[1] = hq[2] = hq[3] = 0u;
                }
            }
            x_bot = X[K - 1];
            e_bot = e;
            if (first_block && s < g) {       // before this lane's first column
                reset_col0();
                x_up_prev = C2;
            }
#pragma unroll
            for (int h = 0; h < 2; h++) {
                if (b < nblk[h]) {
#pragma unroll
                    for (int k = 0; k < KH; k++) {
                        const uint64_t at = aoff[h] + ((uint64_t)s * KH + k) * L + g;
                        if (SA_GUARD(at < A.arena_cap, A.dbg, kSiteArena)) A.arena[at] = h ? wbk[k] : wa[k];
                    }
                }
            }
        };

        uint32_t wbn[2];
#pragma unroll
        for (int h = 0; h < 2; h++) wbn[h] = load_window16<L, K>(A, wstart[h], 0, g);
        // the first blocks (steps s < L, column-0 resets) one step a loop body, the
        // rest without the reset (no register move a row to join two definitions)
        int b = 0;
        for (; b < nblk_warp && 8 * b < L; b++) {
            uint32_t wb[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                wb[h] = wbn[h];
                wbn[h] = load_window16<L, K>(A, wstart[h], b + 1, g);
            }
#pragma unroll 1
            for (int u = 0; u < 8; u++)
                step(b, 8 * b + u, (wb[0] >> (2 * u)) & 3u, (wb[1] >> (2 * u)) & 3u, true);
        }
        for (; b < nblk_warp; b++) {
            uint32_t wb[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                wb[h] = wbn[h];
                wbn[h] = load_window16<L, K>(A, wstart[h], b + 1, g);
            }
            // four steps a loop body (the whole eight overflow the instruction cache)
#pragma unroll 4
            for (int u = 0; u < 8; u++)
                step(b, 8 * b + u, (wb[0] >> (2 * u)) & 3u, (wb[1] >> (2 * u)) & 3u, false);
        }
        __syncwarp();
    }
}

}  // namespace sa
