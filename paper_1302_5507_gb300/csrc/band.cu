// Banded direction pass: one thread per job, direction nibbles of the cells on
// the diagonals that can hold an optimal path ending at the best cell.
//
// Every optimal path ending at (i*, j*) with score `best` consumes at most j*
// read bases, and each insertion costs at least a + e (the match it displaces
// plus its own extension), each deletion at least e.  With S = a*j* - best this
// gives #I <= S/(a+e) and #D <= S/e, so the path stays on the diagonals
// d = i - j in [d* - S/e, d* + S/(a+e)] (d* = i* - j*).  The DP restricted to
// those diagonals (everything else -inf; row 0 and column 0 keep their border
// values) reproduces every value on such paths and every comparison the
// traceback makes, so walking its nibbles from (i*, j*) gives the same CIGAR
// as the full matrix (SOAP3-dp Methods section 3 backtracks from the full D and
// M tables; this stores 4 bits for band-width cells per row instead).
//
// Row j is computed left to right over the band slots k = i - j - d_lo; the
// previous row stays in registers in place: slot k holds H(i-1, j-1) for the
// diagonal move and slot k+1 holds H(i, j-1), E(i, j-1) for the vertical one.
// Rows whose band starts right of column 0 (all but the first few) take a copy
// of the row loop without the border tests.  Nibble words are stored
// interleaved by lane (word w of row j of the job in lane t at ((j-1)*W + w)*32
// + t of its warp's region), so the stores of a warp are coalesced.  The same
// thread then walks its nibbles from (i*, j*): they were written moments before
// and are read back from L2.
#include "kernels.h"
#include "walk.cuh"

namespace sa {

namespace {

// a value the compiler must keep in a register (not re-read from the parameter
// bank at every use)
__device__ __forceinline__ int32_t in_reg(int32_t x) {
    asm volatile("" : "+r"(x));
    return x;
}

template <int B, bool LOCAL, bool EDGE>
__device__ __forceinline__ void band_row(int32_t (&Hs)[B + 1], int32_t (&Es)[B + 1], uint32_t (&words)[(B + 7) / 8],
                                         const uint64_t (&mmh)[B > 32 ? 2 : 1], int i0, int32_t border,
                                         int32_t GO, int32_t GE, int32_t sa, int32_t sb) {
    int32_t hleft = kNeg32, fleft = kNeg32;
#pragma unroll
    for (int k = 0; k < B; k++) {
        int32_t hn, fn, en;
        uint32_t nib = 0u;
        if (EDGE && i0 + k <= 0) {
            hn = (i0 + k == 0) ? border : kNeg32;   // column 0 (H(0, j)) or left of the window
            en = kNeg32;
            fn = kNeg32;
        } else {
            const int32_t diag = Hs[k], up = Hs[k + 1], eup = Es[k + 1];
            const int32_t eo = up + GO, ee = eup + GE;
            en = max(eo, ee);
            const int32_t fo = hleft + GO, fe = fleft + GE;
            fn = max(fo, fe);
            const bool match = (mmh[k >> 5] >> (2 * (k & 31))) & 1ull;
            const int32_t g = diag + (match ? sa : sb);
            // source of H: diagonal > deletion (F) > insertion (E); LOCAL zero: stop.
            // The source is decided by comparing the three candidates with each
            // other, never by comparing a DPX maximum with one of its operands
            // (on this toolchain such a comparison after __vimax3_s32_relu gave
            // wrong predicates)
            const int32_t ef = max(en, fn);
            int32_t h = max(g, ef);
            uint32_t src = g >= ef ? 1u : (fn >= en ? 2u : 3u);
            if (LOCAL && h <= 0) { h = 0; src = 0u; }
            nib = src | (eo >= ee ? 0u : 4u) | (fo >= fe ? 0u : 8u);
            hn = h;
        }
        Hs[k] = hn;
        Es[k] = en;
        hleft = hn;
        fleft = fn;
        words[k >> 3] |= nib << (4 * (k & 7));
    }
}

template <int B, int MODE>
__global__ void __launch_bounds__(128) k_band(BandArgs A) {
    constexpr bool LOCAL = (MODE == SA_LOCAL);
    constexpr int W = (B + 7) / 8;
    static_assert(B == 8 || B == 16 || B == 32 || B == 64, "band widths 8, 16, 32 and 64");
    const uint32_t pos = blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= A.count) return;
    const uint32_t job = A.list[pos];
    const sa_job J = A.jobs[job];
    const Rect R = A.rect[job];
    const int rows = R.rows;
    const int dlo = R.d_lo;
    const int32_t GO = in_reg(A.sc.GO), GE = in_reg(A.sc.GE), sa = in_reg(A.sc.a), sb = in_reg(A.sc.b);
    uint32_t* out = A.arena + (uint64_t)(pos >> 5) * A.warp_stride + (pos & 31);
    const uint32_t* rp = A.rpack + (size_t)job * A.rw;
    const uint32_t* refw = A.ref + kRefFrontPad;

    int32_t Hs[B + 1], Es[B + 1];
#pragma unroll
    for (int k = 0; k <= B; k++) {            // row 0: H(i,0) = 0 for i >= 0, E = -inf
        Hs[k] = (k < B && dlo + k >= 0) ? 0 : kNeg32;
        Es[k] = kNeg32;
    }
    for (int j = 1; j <= rows; j++) {
        const int i0 = j + dlo;               // window column of slot 0
        // match bits of slots 0..B-1 against read base j: window bases at reference
        // positions ref_pos + i0 - 1 + k, 32 slots per 64-bit half; positions before
        // the window start only feed masked slots (column <= 0)
        const uint64_t rb = (uint64_t)((__ldg(rp + ((j - 1) >> 4)) >> (2 * ((j - 1) & 15))) & 3u);
        constexpr int NH = B > 32 ? 2 : 1;
        uint64_t mmh[NH];
#pragma unroll
        for (int hh = 0; hh < NH; hh++) {
            const int64_t ph = (int64_t)J.ref_pos + i0 - 1 + 32 * hh;
            int64_t qh = ph < (int64_t)J.ref_pos ? (int64_t)J.ref_pos : ph;
            if (qh > A.ref_len) qh = A.ref_len;
            const int64_t wi = qh >> 4;
            const uint32_t sh = (uint32_t)(qh & 15) * 2u;
            const uint64_t lo = ((uint64_t)__ldg(refw + wi + 1) << 32) | (uint64_t)__ldg(refw + wi);
            const uint64_t hi = (uint64_t)__ldg(refw + wi + 2);
            uint64_t wb = sh ? ((lo >> sh) | (hi << (64 - sh))) : lo;
            const int64_t lead = qh - ph;     // >= 0
            wb = lead >= 32 ? 0ull : (wb << (2 * lead));
            const uint64_t x = wb ^ (rb * 0x5555555555555555ull);
            mmh[hh] = ~(x | (x >> 1)) & 0x5555555555555555ull;   // bit 2k: slot 32hh+k matches
        }
        uint32_t words[W];
#pragma unroll
        for (int w = 0; w < W; w++) words[w] = 0u;
        if (i0 >= 1) {
            band_row<B, LOCAL, false>(Hs, Es, words, mmh, i0, 0, GO, GE, sa, sb);
        } else {
            const int32_t border = (!LOCAL) ? GO + (j - 1) * GE : 0;  // H(0, j)
            band_row<B, LOCAL, true>(Hs, Es, words, mmh, i0, border, GO, GE, sa, sb);
        }
#pragma unroll
        for (int w = 0; w < W; w++) out[((uint64_t)(j - 1) * W + w) * 32] = words[w];
    }

    const JobState st = A.state[job];
    auto nib = [&](int ii, int jj, bool* bad) -> uint32_t {
        const int k = ii - jj - dlo;
        if (k < 0 || k >= B) { *bad = true; return 0u; }
        const uint32_t word = out[((uint64_t)(jj - 1) * W + (k >> 3)) * 32];
        return (word >> (4 * (k & 7))) & 15u;
    };
    const WalkEnd e = walk_nibbles(st.i_star, st.j_star, st.i_star, rows, MODE, nib,
                                   A.tmp_ops + (uint64_t)job * A.tmp_stride, A.tmp_stride);
    TbOut t;
    t.n_rev = e.n_rev;
    t.read_begin = e.bad ? 0 : e.j;
    t.ref_begin_rel = e.bad ? 0 : e.i;
    A.tb[job] = t;
    if (e.bad) atomicMin(A.err_job, job);
}

}  // namespace

void launch_band(int cls, const BandArgs& a, cudaStream_t st) {
    if (!a.count) return;
    const unsigned grid = (a.count + 127) / 128;
    const bool local = a.sc.mode == SA_LOCAL;
    if (cls == kClsBand8) {
        local ? k_band<8, SA_LOCAL><<<grid, 128, 0, st>>>(a) : k_band<8, SA_GLOCAL><<<grid, 128, 0, st>>>(a);
    } else if (cls == kClsBand16) {
        local ? k_band<16, SA_LOCAL><<<grid, 128, 0, st>>>(a) : k_band<16, SA_GLOCAL><<<grid, 128, 0, st>>>(a);
    } else if (cls == kClsBand32) {
        local ? k_band<32, SA_LOCAL><<<grid, 128, 0, st>>>(a) : k_band<32, SA_GLOCAL><<<grid, 128, 0, st>>>(a);
    } else {
        local ? k_band<64, SA_LOCAL><<<grid, 128, 0, st>>>(a) : k_band<64, SA_GLOCAL><<<grid, 128, 0, st>>>(a);
    }
}

}  // namespace sa
