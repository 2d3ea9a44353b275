// Internal definitions shared by the CUDA translation units of libsa.
//
// Notation follows SOAP3-dp, Methods section 3: T = window (length m, column
// index i), R = read (length n, row index j).  H = M (best), E = I (read base
// against a space, runs along j), F = D (window base against a space, runs
// along i).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sa.h"

namespace sa {

// "minus infinity" of the 32-bit kernels: far below any reachable score
// (|score| < 2^28 by the interface limits) and safe to add one gap penalty to.
constexpr int32_t kNeg32 = -(1 << 29);
// "minus infinity" of the 16-bit packed kernels; host checks keep every
// reachable 16-bit value above it (see width selection in api.cu).
constexpr int32_t kNeg16 = -16384;

// Reference: 2-bit codes A=0 C=1 G=2 T=3, 16 bases per uint32 (base p in bits
// 2*(p&15) of word p>>4).  The device copy has kRefFrontPad words before base
// 0 and kRefTailPad after the last word, so the wavefront can load whole words
// around the window edges without bounds checks.
constexpr int kRefFrontPad = 4;
constexpr int kRefTailPad = 8;

// SA_DEBUG builds check the index of every indexed global store of the kernels
// against its buffer; a store out of range is skipped and its site code (the
// smallest one) recorded in a device word that the call reports as an internal
// error.  Release builds compile the guard to `true`.
#ifdef SA_DEBUG
#define SA_GUARD(ok, word, site) ((ok) || (atomicMin((word), (unsigned)(site)), false))
#else
#define SA_GUARD(ok, word, site) true
#endif
enum {
    kSiteCb16 = 1, kSiteLaneKeys = 2, kSiteState16 = 3, kSiteCb32 = 4, kSiteArena = 5, kSiteState32 = 6,
    kSiteBand = 7, kSiteBandTb = 8, kSiteTraceTb = 9
};

// Lane-group configurations of the wavefront kernels: a group of L lanes
// (L divides 32) works on one job (two jobs in the packed 16-bit kernel); each
// lane owns K consecutive read rows, so a group covers L*K >= n rows.
// Groups of 8 lanes take every K from 4 to 32 (reads up to 256 bases in steps of
// 8 rows, so a read is padded by at most 7 rows); groups of 32 lanes take
// K = 10, 16, 24, 32 (reads up to 1024 bases).
struct Cfg { int L, K; };
constexpr int kNumCfg8 = 29;               // L = 8, K = 4 .. 32
constexpr int kNumCfg = kNumCfg8 + 4;
__host__ __device__ constexpr int cfg_L(int c) { return c < kNumCfg8 ? 8 : 32; }
__host__ __device__ constexpr int cfg_K(int c) {
    return c < kNumCfg8 ? c + 4 : (c == kNumCfg8 ? 10 : c == kNumCfg8 + 1 ? 16 : c == kNumCfg8 + 2 ? 24 : 32);
}
struct CfgTable {
    Cfg c[kNumCfg];
    constexpr CfgTable() : c() {
        for (int i = 0; i < kNumCfg; i++) c[i] = Cfg{cfg_L(i), cfg_K(i)};
    }
    constexpr const Cfg& operator[](int i) const { return c[i]; }
};
constexpr CfgTable kCfgs{};

__host__ __device__ inline int cfg_for_rows(int n) {
    for (int c = 0; c < kNumCfg; c++)
        if (cfg_L(c) * cfg_K(c) >= n) return c;
    return -1;
}

// The plan: the configuration serving each read length and the width of each
// configuration's score pass (0: 16-bit where no job of the bucket can reach the
// overflow threshold, else 32-bit; 16 or 32: that width).  The default maps n
// to the first configuration with L*K >= n; a tuning run may pick another one
// (any configuration with L*K >= n is valid for n).
struct Plan {
    uint8_t cfg[SA_MAX_READ + 1];      // cfg[0] unused
    int8_t width[kNumCfg];
};
inline void default_plan(Plan* p) {
    for (int n = 0; n <= SA_MAX_READ; n++) p->cfg[n] = (uint8_t)cfg_for_rows(n < 1 ? 1 : n);
    for (int c = 0; c < kNumCfg; c++) p->width[c] = 0;
}
inline bool plan_valid(const Plan& p) {
    for (int n = 1; n <= SA_MAX_READ; n++)
        if (p.cfg[n] >= kNumCfg || cfg_L(p.cfg[n]) * cfg_K(p.cfg[n]) < n) return false;
    for (int c = 0; c < kNumCfg; c++)
        if (p.width[c] != 0 && p.width[c] != 16 && p.width[c] != 32) return false;
    return true;
}

// Size classes order jobs inside one configuration (largest windows first).
// Sixteenth-octave classes (16 * floor(log2 m) + the next four bits of m):
// the jobs that share a warp of the packed score pass (which runs as many
// steps as the longest of them) differ in window length by at most 4.5 % in
// one class.
constexpr int kNumSizeCls = 16 * 17;      // m <= 65536 = 2^16
__host__ __device__ inline int size_class(uint32_t m) {
    int lg = 0;
    for (uint32_t v = m; v > 1u; v >>= 1) lg++;
    const int frac = lg >= 4 ? (int)((m >> (lg - 4)) & 15u) : (int)((m << (4 - lg)) & 15u);
    const int c = 16 * lg + frac;
    return c < kNumSizeCls ? c : kNumSizeCls - 1;
}
constexpr int kNumKeys = kNumCfg * kNumSizeCls;

// Signed scoring in the paper's form plus the constants the kernels use.
struct Score {
    int32_t a, b, GO, GE;     // S_MA, S_MI, S_GO, S_GE
    int32_t dm, dx;           // a - GO, b - GO (diagonal term in the H+GO representation)
    int32_t mode;             // SA_LOCAL / SA_GLOCAL
};

// Per-job result of the score pass.
struct JobState {
    int32_t best;       // best score
    int32_t i_star;     // 1-based window column of the best cell (0: none)
    int32_t j_star;     // 1-based read row of the best cell
    int32_t second;     // second best (SA_NO_SCORE if none)
    int32_t second_i;   // 1-based column of the second best (0: none)
    uint32_t flags;     // kStEmpty, kStOverflow
};
constexpr uint32_t kStEmpty = 1u;      // LOCAL: no positive cell
constexpr uint32_t kStOverflow = 2u;   // 16-bit pass may have overflowed: recompute in 32-bit

// The fields of a result row that the score pass alone decides: score, ends,
// second best and flags (SA_RES_BELOW_MIN when best < min_score, then
// SA_RES_EMPTY with score 0 and no ends or second when no cell was positive);
// begins -1 and no CIGAR.  Every entry point that writes sa_result rows starts
// from this row.
__device__ __forceinline__ sa_result score_result(const sa_job& J, const JobState& st, int32_t min_score) {
    sa_result r;
    r.score = st.best;
    r.second = SA_NO_SCORE;
    r.read_begin = -1;
    r.read_end = -1;
    r.ref_begin = -1;
    r.ref_end = -1;
    r.second_ref_end = -1;
    r.cigar_off = 0;
    r.cigar_len = 0;
    r.flags = 0;
    r._pad = 0;
    if (st.best < min_score) r.flags |= SA_RES_BELOW_MIN;
    if (st.flags & kStEmpty) {
        r.flags |= SA_RES_EMPTY;
        r.score = 0;
    } else {
        r.second = st.second;
        r.second_ref_end = st.second_i ? (int64_t)J.ref_pos + st.second_i : -1;
        r.read_end = st.j_star;
        r.ref_end = (int64_t)J.ref_pos + st.i_star;
    }
    return r;
}

// Sub-problem of the direction-bit pass: rows 1..rows of the read against the
// window columns i_lo..i_lo+w-1 (1-based); w == 0 means "no traceback".
struct Rect {
    uint64_t off;       // first word of its direction bits in the arena (within its wave)
    int32_t i_lo;
    int32_t w;
    int32_t rows;
    int32_t start_i;    // traceback start cell in rect coordinates
    int32_t start_j;
    int32_t wave;
    // banded classes: diagonals d = i - j in [d_lo, d_lo + band width)
    int32_t cls;        // kCls*
    int32_t d_lo;
    uint32_t lpos;      // position in its class list
    int32_t cfg;        // lane-group configuration of the job's score pass (its bucket)
};
// direction-pass classes: none (no traceback), banded passes of 8/16/32/64
// diagonals, the wavefront rectangle, and the gapless diagonal (the traceback
// is a run of `rows` diagonal steps from the best cell, found by scoring the
// diagonal: its CIGAR needs no direction bits)
enum { kClsNone = 0, kClsBand16 = 1, kClsBand32 = 2, kClsRect = 3, kClsBand64 = 4, kClsDiag = 5,
       kClsBand8 = 6, kNumCls = 7 };
constexpr int kNumBand = 4;                       // band classes 8, 16, 32, 64
__host__ __device__ inline int band_cls(int b) {
    return b == 0 ? kClsBand8 : (b == 1 ? kClsBand16 : (b == 2 ? kClsBand32 : kClsBand64));
}
__host__ __device__ inline int band_index(int cls) {
    return cls == kClsBand8 ? 0 : (cls == kClsBand16 ? 1 : (cls == kClsBand32 ? 2 : (cls == kClsBand64 ? 3 : -1)));
}
__host__ __device__ inline int band_width_of(int b) { return 8 << b; }

// Column-maximum slots of a lane group: window column i (1-based) at slot
// kCbFront + i - 1.  The slack on both sides takes the stores of the skewed
// wavefront's steps before column 1 and past the window end, which are then
// written without a bounds test.
constexpr int kCbFront = 32;
constexpr int kCbTail = 40;
__host__ __device__ inline uint32_t cb_words(uint32_t max_m) { return max_m + kCbFront + kCbTail; }
// per-warp words of the 16-bit score pass's stored lane keys (one key pair per
// wavefront step and lane; a job pair takes at most max_m + 38 steps)
__host__ __device__ inline uint32_t lane_key_words(uint32_t max_m) { return (max_m + 48) * 32; }

// Arguments of the wavefront kernels.
struct FillArgs {
    const uint32_t* ref;          // padded packed reference (base 0 at ref + kRefFrontPad words)
    int64_t ref_len;              // bases
    const sa_job* jobs;
    const uint32_t* rpack;        // packed reads, rw words per job
    uint32_t rw;
    const uint32_t* order;        // job ids in processing order
    uint32_t pos_begin;           // first position of this launch in `order`
    uint32_t pos_count;           // positions in this launch (if count_ptr == nullptr)
    const uint32_t* count_ptr;    // device count (overflow rerun lists)
    uint32_t* item_counter;       // persistent work counter (zeroed before launch)
    Score sc;
    JobState* state;              // per job id
    int32_t* colbest;             // per group scratch, cb_stride words each
    uint32_t cb_stride;           // cb_words(longest window)
    uint32_t* lane_keys;          // 16-bit score pass: per warp scratch, lk_stride words each
    uint32_t lk_stride;
    // capacities of the buffers above (elements) and the debug word (SA_DEBUG builds)
    uint64_t n_state, cb_cap, lk_cap, arena_cap;
    unsigned* dbg;
    const Rect* rect;             // direction pass: per job id
    uint32_t* arena;              // direction bits
    int32_t wave;                 // direction pass: only jobs of this wave
    int32_t plain;                // direction pass over whole windows (plain form)
};

struct FillLaunch {
    FillArgs args;
    int kind;                     // kFillScore / kFillRect / kFillPlain / kFillScore16
    int grid, block;
    cudaStream_t stream;
};
enum { kFillScore = 0, kFillRect = 1, kFillPlain = 2, kFillScore16 = 3, kFillRectH = 4, kFillRectH16 = 5 };

// per-configuration launchers (one translation unit per configuration)
template <int C> void launch_fill(const FillLaunch& fl);
template <int C> int fill_blocks_per_sm(int kind, int mode);   // resident 128-thread blocks per SM

// direction-bit layout shared by the wavefront kernels and the traceback:
// at wavefront step s lane g of the group stores KW = ceil(K/8) words, word w
// at ((s*KW + w) * L + g); the nibble of its row r is in word r/8, bits
// 4*(r%8).  Steps are counted in whole blocks of 8.
// A nibble: bits 0-1 source of H (0 stop, 1 diagonal, 2 F/deletion,
// 3 E/insertion), bit 2 E extends, bit 3 F extends.
__host__ __device__ inline uint64_t dir_words(int L, int K, int w) {
    uint64_t blocks = (uint64_t)(w + L - 1 + 7) / 8;
    return blocks * 8 * (uint64_t)((K + 7) / 8) * (uint64_t)L;
}
// the byte-height form of the same layout (LOCAL, every score below 255): KH =
// ceil(K/4) words a step and lane, the height of row r in byte r%4 of word r/4
__host__ __device__ inline uint64_t hgt_words(int L, int K, int w) {
    uint64_t blocks = (uint64_t)(w + L - 1 + 7) / 8;
    return blocks * 8 * (uint64_t)((K + 3) / 4) * (uint64_t)L;
}
__host__ __device__ inline uint64_t rect_words(int L, int K, int w, bool heights) {
    return heights ? hgt_words(L, K, w) : dir_words(L, K, w);
}

}  // namespace sa
