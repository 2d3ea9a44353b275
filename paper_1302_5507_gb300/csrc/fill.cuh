// Wavefront DP kernels (32-bit).
//
// Computes the recurrence of SOAP3-dp, Methods section 3 (the I/D/M tables,
// here E/F/H) for one job per group of L lanes.  Lane g of the group owns the
// K consecutive read rows g*K .. g*K+K-1 and keeps, for each of them, H(i-1,j)
// + S_GO and F(i-1,j) in registers.  At wavefront step s lane g computes
// column i = s - g + 1 (the window streams through the group, skewed by one
// column per lane); the H and E values of the lane's bottom row and the
// running column maximum move to the next lane with a shuffle.  No DP table
// is kept in memory: the paper's improved form already keeps only two rows of
// M and D, this form keeps none (the direction bits, when wanted, are the
// only per-cell output).
//
// LOCAL pads the group's rows at the top (rows j <= 0 never match, so they
// stay at H = 0 and feed row 1 exactly the border values H(i,0) = 0,
// E(i,0) = -inf); so does the GLOCAL score pass (its padding rows score 0
// against every base and stay at H = 0), which puts row n on the last lane's
// last row; the GLOCAL direction passes pad at the bottom.
//
// The score pass and the rectangle direction pass take the match term from a
// per-lane shared-memory profile; the plain form uses per-lane match masks.
//
// Four variants (template flags):
//   BEST && !DIR  score pass: best cell, colbest(i), second best
//   DIR && !BEST  direction pass over a sub-rectangle (reduced traceback)
//   DIR && !BEST && HGT  the same sub-rectangle, storing each cell's H as a byte
//                 (LOCAL, every score below 255) instead of a direction nibble:
//                 the score pass's arithmetic, and the walk re-derives the
//                 decisions from the heights
//   DIR && BEST   plain form: direction bits over the whole window + best
#pragma once

#include "sa_internal.cuh"

namespace sa {

__device__ __forceinline__ int32_t addmax(int32_t a, int32_t b, int32_t c) {
    return __viaddmax_s32(a, b, c);   // max(a + b, c)
}

// x + y issued as an integer multiply-add (x * one + y) with a `one` the compiler
// cannot see, so the add runs on the FMA pipe and leaves the ALU pipe (where the
// max operations of the recurrence run) to the maxima
__device__ __forceinline__ int32_t add_fma(int32_t x, int32_t y, int32_t one) { return x * one + y; }

// Shared-memory words of the score pass's per-lane profile: for each window base
// t and read row r of the lane, the diagonal term (a or b) minus S_GO, rows
// padded to a multiple of 4 so that one 16-byte load serves four rows.
template <int K>
constexpr int prof_words_per_warp() { return 4 * ((K + 3) / 4) * 4 * 32; }

template <int L, int K>
__device__ __forceinline__ uint32_t load_window16(const FillArgs& A, int64_t wstart, int b, int g) {
    // 8 bases for columns of block b of lane g: positions wstart + 8b - g .. +7
    int64_t p0 = wstart + 8 * (int64_t)b - g;
    if (p0 > A.ref_len) p0 = A.ref_len;          // junk steps past the data: stay in the padding
    const int64_t wi = p0 >> 4;                  // floor (p0 >= -32 > -16*kRefFrontPad)
    const uint32_t sh = (uint32_t)(p0 & 15) * 2u;
    const uint32_t* base = A.ref + kRefFrontPad;
    const uint64_t v = ((uint64_t)__ldg(base + wi + 1) << 32) | (uint64_t)__ldg(base + wi);
    return (uint32_t)(v >> sh) & 0xFFFFu;
}

template <int L, int K, int MODE, bool DIR, bool BEST, bool HGT = false>
__global__ void __launch_bounds__(128) k_fill32(FillArgs A) {
    static_assert(32 % L == 0, "L must divide 32");
    static_assert(K >= 1 && K <= 32, "K in 1..32");
    static_assert(!HGT || (DIR && !BEST && MODE == SA_LOCAL), "heights: LOCAL sub-rectangle pass only");
    constexpr int KH = (K + 3) / 4;                 // height words of a lane per step
    constexpr int G = 32 / L;
    constexpr bool LOCAL = (MODE == SA_LOCAL);
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int g = lane % L;
    const int grp = lane / L;
    const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int64_t cb_base = (int64_t)(gwarp * G + grp) * A.cb_stride + kCbFront;     // column 1's slot
    int32_t* cb = BEST ? A.colbest + cb_base : nullptr;
    auto cb_ok = [&](int i) { return SA_GUARD((uint64_t)(cb_base + i - 1) < A.cb_cap, A.dbg, kSiteCb32); };
    const Score S = A.sc;
    const uint32_t count = A.count_ptr ? *A.count_ptr : A.pos_count;
    // the score pass and the rectangle direction pass take the match/mismatch term
    // from a shared-memory profile (SPROF); PROF marks the score pass
    constexpr bool PROF = BEST && !DIR;
    constexpr bool SPROF = PROF || (DIR && !BEST);
    constexpr int K4 = (K + 3) / 4;
    extern __shared__ __align__(16) int32_t s_prof[];
    int32_t* prof = s_prof + (threadIdx.x >> 5) * prof_words_per_warp<K>();
    // 1 at run time (every launch uses 128-thread blocks), unknown to the compiler
    const int32_t one = (int32_t)(blockDim.x >> 7);
    // lane 0 of a group takes the top border instead of a neighbour's values:
    // x * nf + c with (nf, c) = (1, 0) on other lanes, (0, border) on lane 0
    const int32_t nf = g != 0 ? one : 0;
    const int32_t hg_c = g != 0 ? 0 : S.GO, e_c = g != 0 ? 0 : kNeg32;
    // score pass, LOCAL: column-maximum keys H * 1024 + (1023 - row index in the
    // group); the lane's own keys use its row r and are shifted by -g*K in the
    // max that passes them down the group
    const int32_t key_shift = -g * K;

    for (;;) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(A.item_counter, 1u);
        item = __shfl_sync(FULL, item, 0);
        if (item * (uint32_t)G >= count) break;
        const uint32_t p = item * G + grp;
        const bool has = p < count;
        const uint32_t job = has ? __ldg(A.order + A.pos_begin + p) : 0u;

        // geometry of this group's task
        int n = 0, rows = 0, w = 0;
        int64_t wstart = 0;
        uint64_t aoff = 0;
        if (has) {
            const sa_job J = A.jobs[job];
            n = (int)J.read_len;
            if (DIR) {
                const Rect R = A.rect[job];
                if (R.w > 0 && R.wave == A.wave) {
                    rows = R.rows;
                    w = R.w;
                    wstart = (int64_t)J.ref_pos + R.i_lo - 1;
                    aoff = R.off;
                }
            } else {
                rows = n;
                w = (int)J.win_len;
                wstart = (int64_t)J.ref_pos;
            }
        }
        const int nblk = w > 0 ? (w + L - 1 + 7) >> 3 : 0;
        int nblk_warp = nblk;
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) nblk_warp = max(nblk_warp, __shfl_xor_sync(FULL, nblk_warp, o));
        if (nblk_warp == 0) continue;

        // LOCAL and the score pass pad the group's rows at the top (GLOCAL padding
        // rows score 0 against every base and stay at H = 0); the GLOCAL direction
        // passes pad at the bottom
        const int pad = (LOCAL || PROF) ? (L * K - rows) : 0;
        // match masks: bit r of mX is set when the lane's row r holds base X
        uint32_t mA = 0, mC = 0, mG = 0, mT = 0;
        if (SPROF) {
            // profile: int4 ((t*K4 + r/4)*32 + lane) holds the diagonal terms of rows
            // r..r+3 against window base t (LOCAL padding rows never match, GLOCAL
            // padding rows score 0); written and read as int4, so later reads cannot
            // move above these stores
            const uint32_t* rp = A.rpack + (size_t)job * A.rw;
            int4* prof4 = reinterpret_cast<int4*>(prof);
#pragma unroll
            for (int q = 0; q < K4; q++) {
                int code[4];
                int32_t miss[4];
#pragma unroll
                for (int u = 0; u < 4; u++) {
                    const int r = 4 * q + u;
                    const int j = g * K + r + 1 - pad;
                    code[u] = -1;
                    miss[u] = (!LOCAL && j < 1) ? -S.GO : S.dx;
                    if (r < K && w > 0 && j >= 1 && j <= rows)
                        code[u] = (int)((__ldg(rp + ((j - 1) >> 4)) >> (2 * ((j - 1) & 15))) & 3u);
                }
#pragma unroll
                for (int t = 0; t < 4; t++)
                    prof4[(t * K4 + q) * 32 + lane] =
                        make_int4(code[0] == t ? S.dm : miss[0], code[1] == t ? S.dm : miss[1],
                                  code[2] == t ? S.dm : miss[2], code[3] == t ? S.dm : miss[3]);
            }
        } else {
            const uint32_t* rp = A.rpack + (size_t)job * A.rw;
#pragma unroll
            for (int r = 0; r < K; r++) {
                const int j = g * K + r + 1 - pad;
                if (w > 0 && j >= 1 && j <= rows) {
                    const uint32_t code = (__ldg(rp + ((j - 1) >> 4)) >> (2 * ((j - 1) & 15))) & 3u;
                    const uint32_t bit = 1u << r;
                    mA |= code == 0 ? bit : 0u;
                    mC |= code == 1 ? bit : 0u;
                    mG |= code == 2 ? bit : 0u;
                    mT |= code == 3 ? bit : 0u;
                }
            }
        }

        // column-0 state: H(0,j) (+ S_GO), F(0,j) = -inf
        int32_t HG[K], F[K];
        auto h0 = [&](int j) -> int32_t {   // H(0, j)
            return (!LOCAL && j >= 1) ? S.GO + (j - 1) * S.GE : 0;
        };
        auto reset_col0 = [&]() {
#pragma unroll
            for (int r = 0; r < K; r++) {
                HG[r] = h0(g * K + r + 1 - pad) + S.GO;
                F[r] = kNeg32;
            }
        };
        reset_col0();
        const int32_t hup0 = h0(g * K - pad) + S.GO;   // H(0, first row - 1) + S_GO
        int32_t h_up_prev = hup0;
        int32_t hg_bot = HG[K - 1], e_bot = kNeg32, cm_bot = 0;

        // best tracking of the plain form (LOCAL) and its row of H(., n) (GLOCAL)
        int32_t bv = 0, bi = 0, br = 0;
        const int gn = LOCAL ? 0 : (rows - 1) / K;
        const int rn = LOCAL ? 0 : (rows - 1) % K;

        // the direction passes keep the step loop rolled: their step body (K rows of
        // compare/select and nibble packing) is large, and eight copies of it overflow
        // the instruction cache.  In the other LOCAL passes the first blocks (steps
        // s < L), where lanes before their first column keep resetting it, run one step
        // a loop body and the rest without the reset, so no step of the main loop joins
        // two definitions of the column registers (which cost a register move a row);
        // the GLOCAL score pass measured 1.5 % slower that way and keeps the reset test
        constexpr int kUnrollSteps = (DIR && !HGT) ? 1 : 8;
        constexpr bool kPeel = kUnrollSteps > 1 && LOCAL;
        auto step = [&](const int b, const int u, const uint32_t wb, const bool first) {
            const int s = 8 * b + u;
            const int i = s - g + 1;
            uint32_t dw[(K + 7) / 8];
            uint32_t hw[HGT ? KH : 1];
            if (DIR) {
#pragma unroll
                for (int k = 0; k < (K + 7) / 8; k++) dw[k] = 0u;
            }
            if (HGT) {
#pragma unroll
                for (int k = 0; k < KH; k++) hw[k] = 0u;
            }
            int32_t hg_up = __shfl_up_sync(FULL, hg_bot, 1, L);
            int32_t e_up = __shfl_up_sync(FULL, e_bot, 1, L);
            int32_t cm_up = 0;
            if (BEST && LOCAL) cm_up = __shfl_up_sync(FULL, cm_bot, 1, L);
            if (PROF) {
                hg_up = hg_up * nf + hg_c;
                e_up = e_up * nf + e_c;
                cm_up = cm_up * nf;
            } else if (g == 0) {
                hg_up = S.GO; e_up = kNeg32; cm_up = 0;
            }
            int32_t diag = h_up_prev;
            h_up_prev = hg_up;
            const uint32_t t = (wb >> (2 * u)) & 3u;
            const uint32_t mk = SPROF ? 0u : (t == 0 ? mA : (t == 1 ? mC : (t == 2 ? mG : mT)));
            const int4* pt = reinterpret_cast<const int4*>(prof) + (t * K4) * 32 + lane;
            int4 dq = make_int4(0, 0, 0, 0);
            int32_t e = e_up, hga = hg_up;
            int32_t lm = 0, hpair = 0;
            // score pass: the diagonal term of row r+1 is formed while row r still
            // holds H(i-1, j) (no copy of the old value is kept)
            int32_t gcur = 0;
            if (SPROF) {
                dq = pt[0];
                gcur = add_fma(dq.x, diag, one);
            }
#pragma unroll
            for (int r = 0; r < K; r++) {
                int32_t gv;
                if (SPROF) {
                    gv = gcur;
                    if (r + 1 < K) {
                        const int rn = r + 1;
                        if ((rn & 3) == 0) dq = pt[(rn / 4) * 32];
                        const int32_t dn = (rn & 3) == 0 ? dq.x : (rn & 3) == 1 ? dq.y : (rn & 3) == 2 ? dq.z : dq.w;
                        gcur = add_fma(dn, HG[r], one);
                    }
                } else {
                    const int32_t d = ((mk >> r) & 1u) ? S.dm : S.dx;
                    gv = diag + d;                    // H(i-1,j-1) + delta
                    diag = HG[r];
                }
                int32_t f, h;
                if (!DIR || HGT) {
                    f = addmax(F[r], S.GE, HG[r]);    // max(F(i-1,j)+GE, H(i-1,j)+GO)
                    e = addmax(e, S.GE, hga);         // max(E(i,j-1)+GE, H(i,j-1)+GO)
                    h = LOCAL ? __vimax3_s32_relu(gv, e, f) : __vimax3_s32(gv, e, f);
                    // byte r & 3 of word r / 4 (0..254: every score is below 255)
                    if (HGT) hw[r >> 2] |= (uint32_t)h << (8 * (r & 3));
                } else {
                    const int32_t fe = F[r] + S.GE;
                    const bool fopen = HG[r] >= fe;
                    f = fopen ? HG[r] : fe;
                    const int32_t ee = e + S.GE;
                    const bool eopen = hga >= ee;
                    e = eopen ? hga : ee;
                    const bool pF = f >= e;
                    const int32_t ef = pF ? f : e;
                    const bool pG = gv >= ef;
                    h = pG ? gv : ef;
                    uint32_t src = pG ? 1u : (pF ? 2u : 3u);
                    if (LOCAL && h <= 0) { h = 0; src = 0u; }
                    const uint32_t nib = src | (eopen ? 0u : 4u) | (fopen ? 0u : 8u);
                    dw[r >> 3] |= nib << (4 * (r & 7));
                }
                F[r] = f;
                HG[r] = SPROF ? add_fma(h, S.GO, one) : h + S.GO;
                hga = HG[r];
                if (BEST && LOCAL) {
                    if (PROF) {
                        // column maximum of keys H*1024 + (1023 - r): the maximum key holds the
                        // largest H and, among equal H, the first row (two rows per 3-input max)
                        const int32_t key = add_fma(h, 1023 - r, 1024 * one);
                        if ((r & 1) == 1) lm = __vimax3_s32(lm, hpair, key);
                        else if (r == K - 1) lm = max(lm, key);
                        else hpair = key;
                    } else {
                        lm = max(lm, h);
                    }
                }
            }
            hg_bot = HG[K - 1];
            e_bot = e;
            if (first && s < g) {                     // before this lane's first column
                reset_col0();
                h_up_prev = hup0;
            }
            const bool active = (unsigned)(i - 1) < (unsigned)w;
            if (BEST) {
                if (PROF) {
                    // the group's column maximum (LOCAL: key; GLOCAL: H(n, i) + S_GO)
                    // goes to the column's slot from the last lane, for every step
                    // (steps outside the window land in the slack slots)
                    if (LOCAL) {
                        const int32_t cm = __viaddmax_s32(lm, key_shift, cm_up);
                        cm_bot = cm;
                        if (g == L - 1 && cb_ok(i)) cb[i - 1] = cm;
                    } else {
                        if (g == L - 1 && cb_ok(i)) cb[i - 1] = HG[K - 1];
                    }
                } else if (LOCAL) {
                    const int32_t cm = max(cm_up, lm);
                    cm_bot = cm;
                    if (active) {
                        if (g == L - 1 && cb_ok(i)) cb[i - 1] = cm;
                        if (lm > bv) {
                            bv = lm;
                            bi = i;
                            int rr = K - 1;
#pragma unroll
                            for (int r = K - 1; r >= 0; r--)
                                if (HG[r] - S.GO == lm) rr = r;
                            br = rr;
                        }
                    }
                } else if (active && g == gn) {
                    int32_t hv = HG[0];
#pragma unroll
                    for (int r = 1; r < K; r++)
                        if (r == rn) hv = HG[r];
                    if (cb_ok(i)) cb[i - 1] = hv - S.GO;
                }
            }
            if (DIR && !HGT && b < nblk) {
#pragma unroll
                for (int k = 0; k < (K + 7) / 8; k++) {
                    const uint64_t at = aoff + ((uint64_t)s * ((K + 7) / 8) + k) * L + g;
                    if (SA_GUARD(at < A.arena_cap, A.dbg, kSiteArena)) A.arena[at] = dw[k];
                }
            }
            if (HGT && b < nblk) {
#pragma unroll
                for (int k = 0; k < KH; k++) {
                    const uint64_t at = aoff + ((uint64_t)s * KH + k) * L + g;
                    if (SA_GUARD(at < A.arena_cap, A.dbg, kSiteArena)) A.arena[at] = hw[k];
                }
            }
        };
        uint32_t wb_next = load_window16<L, K>(A, wstart, 0, g);
        int b0 = 0;
        if (kPeel) {
            for (; b0 < nblk_warp && 8 * b0 < L; b0++) {
                const uint32_t wb = wb_next;
                wb_next = load_window16<L, K>(A, wstart, b0 + 1, g);
#pragma unroll 1
                for (int u = 0; u < 8; u++) step(b0, u, wb, true);
            }
        }
        for (; b0 < nblk_warp; b0++) {
            const uint32_t wb = wb_next;
            wb_next = load_window16<L, K>(A, wstart, b0 + 1, g);
#pragma unroll kUnrollSteps
            for (int u = 0; u < 8; u++) step(b0, u, wb, !kPeel && 8 * b0 < L);
        }

        if (BEST) {
            __syncwarp();
            int32_t best;
            int istar, jstar;
            bool empty = false;
            // column value of a slot: colbest(i) of the recurrence
            auto colval = [&](int32_t raw) -> int32_t {
                return PROF ? (LOCAL ? (raw >> 10) : raw - S.GO) : raw;
            };
            if (PROF && LOCAL) {
                // best: the first column holding the largest H; the key of that column
                // holds the first row with it (row index in the group = 1023 - tag)
                int32_t v = -1, key = 0;
                int vi = 0;
                for (int ii = g + 1; ii <= w; ii += L) {
                    const int32_t x = cb[ii - 1];
                    if ((x >> 10) > v) { v = x >> 10; key = x; vi = ii; }
                }
#pragma unroll
                for (int o = 1; o < L; o <<= 1) {
                    const int32_t ov = __shfl_xor_sync(FULL, v, o, L);
                    const int32_t ok = __shfl_xor_sync(FULL, key, o, L);
                    const int oi = __shfl_xor_sync(FULL, vi, o, L);
                    if (ov > v || (ov == v && oi < vi)) { v = ov; key = ok; vi = oi; }
                }
                best = v;
                istar = vi;
                jstar = 1024 - (key & 1023) - pad;
                empty = v <= 0;
            } else if (LOCAL) {
                int bj = g * K + br + 1 - pad;
#pragma unroll
                for (int o = 1; o < L; o <<= 1) {
                    const int32_t ov = __shfl_xor_sync(FULL, bv, o, L);
                    const int oi = __shfl_xor_sync(FULL, bi, o, L);
                    const int oj = __shfl_xor_sync(FULL, bj, o, L);
                    if (ov > bv || (ov == bv && (oi < bi || (oi == bi && oj < bj)))) {
                        bv = ov; bi = oi; bj = oj;
                    }
                }
                best = bv;
                istar = bi;
                jstar = bj;
                empty = bv <= 0;
            } else {
                int32_t v = kNeg32;
                int vi = 0;
                for (int ii = g + 1; ii <= w; ii += L) {
                    const int32_t x = colval(cb[ii - 1]);
                    if (vi == 0 || x > v) { v = x; vi = ii; }
                }
#pragma unroll
                for (int o = 1; o < L; o <<= 1) {
                    const int32_t ov = __shfl_xor_sync(FULL, v, o, L);
                    const int oi = __shfl_xor_sync(FULL, vi, o, L);
                    if (oi != 0 && (vi == 0 || ov > v || (ov == v && oi < vi))) { v = ov; vi = oi; }
                }
                best = v;
                istar = vi;
                jstar = rows;
            }
            // second best; the shuffles stay outside any per-group branch (every
            // lane of the warp must reach them)
            int32_t sv = SA_NO_SCORE;
            int si = 0;
            const int wsec = empty ? 0 : w;
            for (int ii = g + 1; ii <= wsec; ii += L) {
                const int dd = ii > istar ? ii - istar : istar - ii;
                if (dd < n) continue;
                const int32_t x = colval(cb[ii - 1]);
                if (si == 0 || x > sv) { sv = x; si = ii; }
            }
#pragma unroll
            for (int o = 1; o < L; o <<= 1) {
                const int32_t ov = __shfl_xor_sync(FULL, sv, o, L);
                const int oi = __shfl_xor_sync(FULL, si, o, L);
                if (oi != 0 && (si == 0 || ov > sv || (ov == sv && oi < si))) { sv = ov; si = oi; }
            }
            if (g == 0 && has) {
                JobState st;
                st.best = empty ? 0 : best;
                st.i_star = empty ? 0 : istar;
                st.j_star = empty ? 0 : jstar;
                st.second = empty ? SA_NO_SCORE : sv;
                st.second_i = empty ? 0 : si;
                st.flags = empty ? kStEmpty : 0u;
                if (SA_GUARD(job < A.n_state, A.dbg, kSiteState32)) A.state[job] = st;
            }
            __syncwarp();
        }
    }
}

}  // namespace sa
