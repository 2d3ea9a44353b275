// Banded direction pass: one thread per job, direction nibbles of the cells on
// the diagonals that can hold an optimal path ending at the best cell.
//
// Every optimal path ending at (i*, j*) with score `best` consumes at most j*
// read bases, and each insertion costs at least a + e (the match it displaces
// plus its own extension), each deletion at least e, and a path with gaps of a
// kind opens at least one of them (o = gap open).  With S = a*j* - best this
// gives #I <= (S - o)/(a+e) and #D <= (S - o)/e (none when S is below
// o + a + e, resp. o + e), so the path stays on the diagonals d = i - j in
// [d* - #D max, d* + #I max] (d* = i* - j*).  The DP restricted to
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
//
// LOCAL jobs whose scores fit a byte (a * n <= 254) take a lighter form
// (`k_band_h`): the pass stores each in-band H as a byte (255 = -inf) instead
// of a direction nibble, and the walk re-derives every decision from those
// heights: M when H = H(i-1,j-1) + delta; D when H equals F(i,j) = max over
// k >= 1 of H(i-k,j) + S_GO + (k-1) S_GE (the recurrence's deletion value,
// summed along the row); I otherwise; a gap run extends from (i,j) while its
// value is strictly above H(neighbour) + S_GO.  These are the comparisons the
// nibbles record, taken on the same band values, so the CIGAR is the same.
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
    const uint64_t out_base = (uint64_t)(pos >> 5) * A.warp_stride + (pos & 31);
    uint32_t* out = A.arena + out_base;
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
        for (int w = 0; w < W; w++) {
            const uint64_t at = ((uint64_t)(j - 1) * W + w) * 32;
            if (SA_GUARD(out_base + at < A.region_cap, A.dbg, kSiteBand)) out[at] = words[w];
        }
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
    if (SA_GUARD(job < A.n_state, A.dbg, kSiteBandTb)) A.tb[job] = t;
    if (e.bad) atomicMin(A.err_job, job);
}

template <int B, bool EDGE>
__device__ __forceinline__ void band_row_h(int32_t (&Hs)[B + 1], int32_t (&Es)[B + 1], uint32_t (&words)[B / 4],
                                           const uint64_t (&mmh)[B > 32 ? 2 : 1], int i0,
                                           int32_t GO, int32_t GE, int32_t sa, int32_t sb) {
    int32_t hleft = kNeg32, fleft = kNeg32;
#pragma unroll
    for (int k = 0; k < B; k++) {
        int32_t hn, fn, en;
        uint32_t byte;
        if (EDGE && i0 + k <= 0) {
            hn = (i0 + k == 0) ? 0 : kNeg32;        // column 0 (LOCAL: H(0,j) = 0) or left of it
            en = kNeg32;
            fn = kNeg32;
            byte = (i0 + k == 0) ? 0u : 255u;
        } else {
            en = max(Hs[k + 1] + GO, Es[k + 1] + GE);
            fn = max(hleft + GO, fleft + GE);
            const bool match = (mmh[k >> 5] >> (2 * (k & 31))) & 1ull;
            hn = __vimax3_s32_relu(Hs[k] + (match ? sa : sb), en, fn);
            byte = (uint32_t)hn;
        }
        Hs[k] = hn;
        Es[k] = en;
        hleft = hn;
        fleft = fn;
        words[k >> 2] |= byte << (8 * (k & 3));
    }
}

// The walk of a byte-height band job from its best cell, deciding from the
// stored heights (see the file comment); `out` is the job's lane of its region.
template <int B>
__device__ __forceinline__ void band_h_walk(const BandArgs& A, uint32_t pos, uint32_t job, const sa_job& J,
                                            const Rect& R, const uint32_t* out, const uint32_t* rp,
                                            const uint32_t* refw, int32_t GO, int32_t GE, int32_t sa, int32_t sb) {
    constexpr int W = B / 4;
    const int rows = R.rows;
    const int dlo = R.d_lo;
    (void)pos;
    const JobState st = A.state[job];
    auto height = [&](int ii, int jj) -> int32_t {     // band H(ii, jj); kNeg32 outside
        if (jj == 0) return ii >= 0 ? 0 : kNeg32;       // row 0
        const int k = ii - jj - dlo;
        if (k < 0 || k >= B) return kNeg32;
        const uint32_t v = (out[((uint64_t)(jj - 1) * W + (k >> 2)) * 32] >> (8 * (k & 3))) & 255u;
        return v == 255u ? kNeg32 : (int32_t)v;
    };
    // Heights on the walk's diagonal: the walk mostly moves diagonally, staying in
    // one height word column, so the words of the next kPre rows of that column
    // are loaded together (independent loads, one latency) and reused until the
    // walk leaves them.
    uint32_t p0 = 0, p1 = 0, p2 = 0, p3 = 0, p4 = 0, p5 = 0, p6 = 0, p7 = 0;   // 8 rows (scalars:
    int pre_col = -1, pre_row = 0;                       // stay in registers) of word column pre_col,
    auto diag_height = [&](int ii, int jj) -> int32_t {  // rows pre_row, pre_row-1, ...; = height(ii, jj)
        if (jj == 0) return ii >= 0 ? 0 : kNeg32;
        const int k = ii - jj - dlo;
        if (k < 0 || k >= B) return kNeg32;
        int d = pre_row - jj;
        if ((k >> 2) != pre_col || d < 0 || d >= 8) {
            pre_col = k >> 2;
            pre_row = jj;
            d = 0;
            const uint32_t* col = out + (uint64_t)pre_col * 32;
            auto at = [&](int row) -> uint32_t { return row >= 1 ? col[(uint64_t)(row - 1) * W * 32] : 0u; };
            p0 = at(jj); p1 = at(jj - 1); p2 = at(jj - 2); p3 = at(jj - 3);
            p4 = at(jj - 4); p5 = at(jj - 5); p6 = at(jj - 6); p7 = at(jj - 7);
        }
        const uint32_t lo = d & 4 ? (d & 2 ? (d & 1 ? p7 : p6) : (d & 1 ? p5 : p4))
                                  : (d & 2 ? (d & 1 ? p3 : p2) : (d & 1 ? p1 : p0));
        const uint32_t v = (lo >> (8 * (k & 3))) & 255u;
        return v == 255u ? kNeg32 : (int32_t)v;
    };
    // window and read bases, one cached 16-base word each
    uint64_t tw_at = ~0ull, rw_at = ~0ull;
    uint32_t tw = 0, rw_word = 0;
    auto base_t = [&](int ii) -> uint32_t {              // window base of column ii >= 1
        const uint64_t p = J.ref_pos + (uint64_t)(ii - 1);
        if ((p >> 4) != tw_at) { tw_at = p >> 4; tw = __ldg(refw + tw_at); }
        return (tw >> (2 * (p & 15))) & 3u;
    };
    auto base_r = [&](int jj) -> uint32_t {              // read base of row jj >= 1
        const uint64_t q = (uint64_t)(jj - 1) >> 4;
        if (q != rw_at) { rw_at = q; rw_word = __ldg(rp + q); }
        return (rw_word >> (2 * ((jj - 1) & 15))) & 3u;
    };
    uint32_t* ops = A.tmp_ops + (uint64_t)job * A.tmp_stride;
    const uint32_t cap = A.tmp_stride;
    int nrev = 0;
    uint32_t cur_op = 15u, cur_len = 0;
    auto emit = [&](uint32_t op) {
        if (op == cur_op) { cur_len++; return; }
        if (cur_len) ops[nrev++] = (cur_len << 4) | cur_op;
        cur_op = op;
        cur_len = 1;
    };
    int i = st.i_star, j = st.j_star;
    int32_t h = st.best, cur = 0;
    int state = 0;                                       // 0 H, 1 E (insertion), 2 F (deletion)
    int budget = 2 * (st.i_star + rows) + 4;
    bool bad = (i < 1 || j < 1 || j > rows || i - j - dlo < 0 || i - j - dlo >= B || height(i, j) != h);
    while (!bad) {
        if (--budget < 0 || nrev >= (int)cap - 1) { bad = true; break; }
        if (state == 0) {
            if (i == 0 || j == 0 || h <= 0) break;
            const int32_t hd = diag_height(i - 1, j - 1);
            if (hd != kNeg32 && hd + (base_t(i) == base_r(j) ? sa : sb) == h) {
                emit(0u);
                i--; j--; h = hd;
                continue;
            }
            // F(i,j) compared with H: the scan stops once it reaches H (F never exceeds
            // it) or once no later term can (H(i',j) <= min(best, a min(i',j)) in LOCAL)
            int32_t f = kNeg32;
            for (int kk = 1; kk <= i; kk++) {
                if (min(st.best, sa * min(j, i - kk)) + GO + (kk - 1) * GE < h) break;
                const int32_t hx = height(i - kk, j);
                if (hx == kNeg32) break;                 // left of the band: the rest is -inf
                f = max(f, hx + GO + (kk - 1) * GE);
                if (f >= h) break;
            }
            state = (f == h) ? 2 : 1;
            cur = h;
        } else if (state == 2) {
            if (i < 1) { bad = true; break; }
            emit(2u);
            const int32_t hn = height(i - 1, j);
            i--;
            if (hn != kNeg32 && cur <= hn + GO) { state = 0; h = hn; }
            else cur -= GE;
        } else {
            if (j < 1) { bad = true; break; }
            emit(1u);
            const int32_t hn = height(i, j - 1);
            j--;
            if (hn != kNeg32 && cur <= hn + GO) { state = 0; h = hn; }
            else cur -= GE;
        }
    }
    TbOut t;
    if (bad) {
        atomicMin(A.err_job, job);
        t.n_rev = 0;
        t.read_begin = 0;
        t.ref_begin_rel = 0;
    } else {
        if (cur_len) ops[nrev++] = (cur_len << 4) | cur_op;
        t.n_rev = nrev;
        t.read_begin = j;
        t.ref_begin_rel = i;
    }
    if (SA_GUARD(job < A.n_state, A.dbg, kSiteBandTb)) A.tb[job] = t;
}

template <int B, bool WALK>
__global__ void __launch_bounds__(128) k_band_h(BandArgs A) {
    constexpr int W = B / 4;                   // words of heights a row
    static_assert(B == 8 || B == 16 || B == 32 || B == 64, "band widths 8, 16, 32 and 64");
    const uint32_t pos = blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= A.count) return;
    const uint32_t job = A.list[pos];
    const sa_job J = A.jobs[job];
    const Rect R = A.rect[job];
    const int rows = R.rows;
    const int dlo = R.d_lo;
    const int32_t GO = in_reg(A.sc.GO), GE = in_reg(A.sc.GE), sa = in_reg(A.sc.a), sb = in_reg(A.sc.b);
    const uint64_t out_base = (uint64_t)(pos >> 5) * A.warp_stride + (pos & 31);
    uint32_t* out = A.arena + out_base;
    const uint32_t* rp = A.rpack + (size_t)job * A.rw;
    const uint32_t* refw = A.ref + kRefFrontPad;

    int32_t Hs[B + 1], Es[B + 1];
#pragma unroll
    for (int k = 0; k <= B; k++) {
        Hs[k] = (k < B && dlo + k >= 0) ? 0 : kNeg32;
        Es[k] = kNeg32;
    }
    for (int j = 1; j <= rows; j++) {
        const int i0 = j + dlo;
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
            const int64_t lead = qh - ph;
            wb = lead >= 32 ? 0ull : (wb << (2 * lead));
            const uint64_t x = wb ^ (rb * 0x5555555555555555ull);
            mmh[hh] = ~(x | (x >> 1)) & 0x5555555555555555ull;
        }
        uint32_t words[W];
#pragma unroll
        for (int w = 0; w < W; w++) words[w] = 0u;
        if (i0 >= 1) band_row_h<B, false>(Hs, Es, words, mmh, i0, GO, GE, sa, sb);
        else band_row_h<B, true>(Hs, Es, words, mmh, i0, GO, GE, sa, sb);
#pragma unroll
        for (int w = 0; w < W; w++) {
            const uint64_t at = ((uint64_t)(j - 1) * W + w) * 32;
            if (SA_GUARD(out_base + at < A.region_cap, A.dbg, kSiteBand)) out[at] = words[w];
        }
    }

    if (WALK) band_h_walk<B>(A, pos, job, J, R, out, rp, refw, GO, GE, sa, sb);
}

// the walk of a byte-height band job on its own (the pass ran without it): a
// light kernel, many resident warps to hide the walk's dependent loads
template <int B>
__global__ void __launch_bounds__(128) k_band_h_walk(BandArgs A) {
    const uint32_t pos = blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= A.count) return;
    const uint32_t job = A.list[pos];
    const sa_job J = A.jobs[job];
    const Rect R = A.rect[job];
    const int32_t GO = in_reg(A.sc.GO), GE = in_reg(A.sc.GE), sa = in_reg(A.sc.a), sb = in_reg(A.sc.b);
    const uint64_t out_base = (uint64_t)(pos >> 5) * A.warp_stride + (pos & 31);
    band_h_walk<B>(A, pos, job, J, R, A.arena + out_base, A.rpack + (size_t)job * A.rw, A.ref + kRefFrontPad,
                   GO, GE, sa, sb);
}

// Match bits of one row of a job's band: bit 2k of word k >> 5 is set when the
// window base of slot k (column i0 + k) equals read base rb.  Slots left of
// column 1 never match (see k_band_h2).
template <int NH>
__device__ __forceinline__ void band_match_bits(const uint32_t* refw, int64_t ref_len, int64_t ref_pos, int i0,
                                                uint32_t rb, uint64_t (&mm)[NH]) {
#pragma unroll
    for (int hh = 0; hh < NH; hh++) {
        const int64_t ph = ref_pos + i0 - 1 + 32 * hh;
        int64_t qh = ph < ref_pos ? ref_pos : ph;
        if (qh > ref_len) qh = ref_len;
        const int64_t wi = qh >> 4;
        const uint32_t sh = (uint32_t)(qh & 15) * 2u;
        const uint64_t lo = ((uint64_t)__ldg(refw + wi + 1) << 32) | (uint64_t)__ldg(refw + wi);
        const uint64_t hi = (uint64_t)__ldg(refw + wi + 2);
        const uint64_t wb = sh ? ((lo >> sh) | (hi << (64 - sh))) : lo;
        const uint64_t x = wb ^ ((uint64_t)rb * 0x5555555555555555ull);
        const uint64_t m = ~(x | (x >> 1)) & 0x5555555555555555ull;
        // lead slots (left of column 1): shifted in as non-matches; a half past the
        // reference's end (lead < 0) matches nothing
        const int64_t lead = qh - ph;
        mm[hh] = (lead < 0 || lead >= 32) ? 0ull : (m << (2 * lead));
    }
}

__device__ __forceinline__ uint32_t pack_s16x2(int32_t lo, int32_t hi) {
    return ((uint32_t)lo & 0xFFFFu) | ((uint32_t)hi << 16);
}

// Byte-height band pass, two jobs a thread in 16-bit halves: job A (list entry
// 64c + t) in the low and job B (entry 64c + 32 + t) in the high half of every
// register, so each store of a warp still covers 32 consecutive words of one
// region.  Per half, with beta = o + e (= -S_GO):
//   X = H,   E~ = E + beta,   F~ = F + beta
//   E~(i,j) = max(E~(i,j-1) + S_GE, X(i,j-1))
//   F~(i,j) = max(F~(i-1,j) + S_GE, X(i-1,j))
//   G~(i,j) = max(X(i-1,j-1) + delta + beta, beta)       (the LOCAL zero floor)
//   X(i,j)  = max(G~, E~, F~) - beta
// which is the recurrence of SOAP3-dp Methods section 3 shifted by beta.  The
// last subtraction is one 32-bit multiply-add on both halves: every maximum is at
// least beta, so the low half always carries and the high half's constant is one
// less.  delta + beta is one multiply-add of the two match bits (it needs
// mismatch <= o + e, so that no half goes negative).
// Cells left of column 0 are computed like window columns whose bases never
// match: all of them get H = 0 (their E and F stay negative), so column 0 holds
// the border's H = 0 and column 1 sees F = H(0,j) + S_GO as from the border; no
// slot needs an edge test.  The walk never reads left of column 0.  A job with
// fewer rows than its partner computes the extra rows without storing them.
template <int B, bool ROWS2>
__global__ void __launch_bounds__(128) k_band_h2(BandArgs A) {
    constexpr int W = B / 4;                   // words of heights a row
    constexpr int NH = B > 32 ? 2 : 1;
    static_assert(B == 8 || B == 16 || B == 32 || B == 64, "band widths 8, 16, 32 and 64");
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t posA = (tid >> 5) * 64u + (tid & 31u);
    if (posA >= A.count) return;
    const uint32_t posB = posA + 32u;
    const bool hasB = posB < A.count;
    const uint32_t jobA = A.list[posA];
    const uint32_t jobB = hasB ? A.list[posB] : jobA;
    const int64_t refA = (int64_t)A.jobs[jobA].ref_pos, refB = (int64_t)A.jobs[jobB].ref_pos;
    const int rowsA = A.rect[jobA].rows, rowsB = hasB ? A.rect[jobB].rows : 0;
    const int dloA = A.rect[jobA].d_lo, dloB = A.rect[jobB].d_lo;
    const uint32_t* rpA = A.rpack + (size_t)jobA * A.rw;
    const uint32_t* rpB = A.rpack + (size_t)jobB * A.rw;
    const uint32_t* refw = A.ref + kRefFrontPad;
    // the two entries' regions: entry p's words at (p >> 5) * warp_stride + (p & 31)
    const uint64_t baseA = (uint64_t)(posA >> 5) * A.warp_stride + (posA & 31u);
    const uint64_t baseB = baseA + A.warp_stride;
    uint32_t* outA = A.arena + baseA;
    uint32_t* outB = A.arena + baseB;

    const int32_t beta = -A.sc.GO;
    const uint32_t one = blockDim.x >> 7;               // 1 at run time (keeps the multiply-add)
    const uint32_t GE2 = pack_s16x2(A.sc.GE, A.sc.GE);
    const uint32_t BETA2 = pack_s16x2(beta, beta);
    const uint32_t SB2 = pack_s16x2(A.sc.b + beta, A.sc.b + beta);
    const uint32_t AB = (uint32_t)(A.sc.a - A.sc.b);
    const uint32_t GO2C = beta == 0 ? 0u : (((uint32_t)(-beta) & 0xFFFFu) + ((uint32_t)(-beta - 1) << 16));
    const uint32_t NEG2 = pack_s16x2(-16384, -16384);   // outside the band (+ S_GE stays in range)

    uint32_t Xs[B + 1], Es[B + 1];
#pragma unroll
    for (int k = 0; k <= B; k++) {
        Xs[k] = k < B ? 0u : NEG2;             // row 0: H = 0 (left of column 0 too)
        Es[k] = NEG2;
    }
    const int rows = max(rowsA, rowsB);
    // one row of the pair: its match bits, the ends of its F chain and four slots'
    // heights awaiting their byte stores
    struct Row {
        uint64_t mA[NH], mB[NH];
        uint32_t wd, xleft, fleft, xq[4];
        int j;
        bool stA, stB;
    };
    auto row_begin = [&](Row& R, const int j) {
        const uint32_t rbA = (__ldg(rpA + ((j - 1) >> 4)) >> (2 * ((j - 1) & 15))) & 3u;
        const uint32_t rbB = (__ldg(rpB + ((j - 1) >> 4)) >> (2 * ((j - 1) & 15))) & 3u;
        band_match_bits<NH>(refw, A.ref_len, refA, j + dloA, rbA, R.mA);
        band_match_bits<NH>(refw, A.ref_len, refB, j + dloB, rbB, R.mB);
        R.j = j;
        R.stA = j <= rowsA;
        R.stB = j <= rowsB;
        R.xleft = NEG2;
        R.fleft = NEG2;
        R.wd = 0u;
    };
    // slot k of row R.j: reads the previous row's slots k (diagonal) and k + 1 (up)
    // and leaves its own values in slot k
    auto slot = [&](Row& R, const int k) {
        if ((k & 7) == 0) {                    // slots 8c .. 8c+7: A's bits low, B's high
            const int c = k >> 3;
            const uint32_t wa = (uint32_t)(R.mA[c >> 2] >> (16 * (c & 3))) & 0xFFFFu;
            const uint32_t wb = (uint32_t)(R.mB[c >> 2] >> (16 * (c & 3))) << 16;
            R.wd = wa | wb;
        }
        const uint32_t sel = (R.wd >> (2 * (k & 7))) & 0x00010001u;
        const uint32_t d2 = sel * AB + SB2;                         // delta + beta, both halves
        const uint32_t en = __viaddmax_s16x2(Es[k + 1], GE2, Xs[k + 1]);
        const uint32_t fn = __viaddmax_s16x2(R.fleft, GE2, R.xleft);
        const uint32_t gt = __viaddmax_s16x2(Xs[k], d2, BETA2);
        const uint32_t x = __vimax3_s16x2(gt, en, fn) * one + GO2C;
        Xs[k] = x;
        Es[k] = en;
        R.xleft = x;
        R.fleft = fn;
        R.xq[k & 3] = x;
        if ((k & 3) == 3) {
            // bytes of four slots: [A0 A1 B0 B1], [A2 A3 B2 B3] -> A0..A3, B0..B3
            const uint32_t t01 = __byte_perm(R.xq[0], R.xq[1], 0x6240);
            const uint32_t t23 = __byte_perm(R.xq[2], R.xq[3], 0x6240);
            const uint64_t at = ((uint64_t)(R.j - 1) * W + (k >> 2)) * 32;
            if (R.stA && SA_GUARD(baseA + at < A.region_cap, A.dbg, kSiteBand)) outA[at] = __byte_perm(t01, t23, 0x5410);
            if (R.stB && SA_GUARD(baseB + at < A.region_cap, A.dbg, kSiteBand)) outB[at] = __byte_perm(t01, t23, 0x7632);
        }
    };
    int j = 1;
    if (ROWS2) {
        // two rows at once, the second one slot behind: its slot k - 1 reads the first
        // row's slots k - 1 and k, both final by then, and the first row's slot k still
        // finds the row above in slots k and k + 1; two independent F chains a thread
        for (; j + 1 <= rows; j += 2) {
            Row r0, r1;
            row_begin(r0, j);
            row_begin(r1, j + 1);
#pragma unroll
            for (int k = 0; k <= B; k++) {
                if (k < B) slot(r0, k);
                if (k >= 1) slot(r1, k - 1);
            }
        }
    }
    for (; j <= rows; j++) {
        Row r0;
        row_begin(r0, j);
#pragma unroll
        for (int k = 0; k < B; k++) slot(r0, k);
    }
}

}  // namespace

int launch_band(int cls, const BandArgs& a, bool heights, cudaStream_t st) {
    if (!a.count) return 0;
    const unsigned grid = (a.count + 127) / 128;
    const bool local = a.sc.mode == SA_LOCAL;
    if (heights) {                     // LOCAL, scores below 255
        // the narrow classes walk right after their pass in the same thread; the wide
        // ones (96 and 168 registers a thread) hand the walk to a light kernel on the
        // same stream, which keeps many more warps resident for its dependent loads.
        // With mismatch <= o + e the wide passes take two jobs a thread in 16-bit
        // halves (k_band_h2); for the narrow classes the pair form, whose walk must
        // then run in its own kernel, measured slower
        const bool pairs = a.sc.b - a.sc.GO >= 0;
        const unsigned grid2 = (a.count + 255) / 256;
        if (cls == kClsBand8) {
            k_band_h<8, true><<<grid, 128, 0, st>>>(a);
            return 1;
        }
        if (cls == kClsBand16) {
            k_band_h<16, true><<<grid, 128, 0, st>>>(a);
            return 1;
        }
        if (cls == kClsBand32) {
            if (pairs) k_band_h2<32, true><<<grid2, 128, 0, st>>>(a);
            else k_band_h<32, false><<<grid, 128, 0, st>>>(a);
            k_band_h_walk<32><<<grid, 128, 0, st>>>(a);
        } else {
            if (pairs) k_band_h2<64, true><<<grid2, 128, 0, st>>>(a);
            else k_band_h<64, false><<<grid, 128, 0, st>>>(a);
            k_band_h_walk<64><<<grid, 128, 0, st>>>(a);
        }
        return 2;
    }
    if (cls == kClsBand8) {
        local ? k_band<8, SA_LOCAL><<<grid, 128, 0, st>>>(a) : k_band<8, SA_GLOCAL><<<grid, 128, 0, st>>>(a);
    } else if (cls == kClsBand16) {
        local ? k_band<16, SA_LOCAL><<<grid, 128, 0, st>>>(a) : k_band<16, SA_GLOCAL><<<grid, 128, 0, st>>>(a);
    } else if (cls == kClsBand32) {
        local ? k_band<32, SA_LOCAL><<<grid, 128, 0, st>>>(a) : k_band<32, SA_GLOCAL><<<grid, 128, 0, st>>>(a);
    } else {
        local ? k_band<64, SA_LOCAL><<<grid, 128, 0, st>>>(a) : k_band<64, SA_GLOCAL><<<grid, 128, 0, st>>>(a);
    }
    return 1;
}

}  // namespace sa
