// Traceback walk over direction nibbles (SOAP3-dp Methods section 3 backtracks
// from the D and M tables; here from 4-bit nibbles: bits 0-1 the source of H --
// 0 stop, 1 diagonal, 2 F (deletion), 3 E (insertion) -- bit 2 "E extends",
// bit 3 "F extends").  Priority stop > M > D > I is already in the nibbles; the
// walk follows them from (i, j), emits run-merged ops in reverse order and stops
// at a stop nibble or a border.  It is bounded: a valid walk emits at most
// imax + rows ops and enters at most as many gap runs (one extra iteration
// each), so a longer walk, a cell outside [0, imax] x [0, rows] or an access the
// caller rejects is reported as an internal error (`bad`), never run on.
#pragma once

#include "sa_internal.cuh"

namespace sa {

struct WalkEnd {
    int n_rev;        // ops written, reversed
    int i, j;         // end cell (0-based begin coordinates of the alignment)
    bool bad;
};

// nib(ii, jj, &bad) returns the nibble of cell (ii, jj) or sets bad
template <class Nib>
__device__ __forceinline__ WalkEnd walk_nibbles(int i, int j, int imax, int rows, int mode, Nib nib,
                                                uint32_t* ops, uint32_t cap) {
    int nrev = 0;
    uint32_t cur_op = 15u, cur_len = 0;
    auto emit = [&](uint32_t op, uint32_t len) {
        if (op == cur_op) { cur_len += len; return; }
        if (cur_len) ops[nrev++] = (cur_len << 4) | cur_op;
        cur_op = op;
        cur_len = len;
    };
    int state = 0;   // 0 H, 1 E (insertion), 2 F (deletion)
    int budget = 2 * (imax + rows) + 4;
    bool bad = (i < 0 || j < 0 || i > imax || j > rows);
    while (!bad) {
        if (--budget < 0) { bad = true; break; }
        if (state == 0) {
            if (i == 0 || j == 0) break;
            const uint32_t nb = nib(i, j, &bad);
            if (bad) break;
            const uint32_t src = nb & 3u;
            if (src == 0u) break;
            if (src == 1u) { emit(0u, 1u); i--; j--; }
            else if (src == 2u) state = 2;
            else state = 1;
        } else if (state == 2) {
            if (i < 1 || j < 1) { bad = true; break; }
            const uint32_t nb = nib(i, j, &bad);
            if (bad) break;
            emit(2u, 1u);
            i--;
            state = (nb & 8u) ? 2 : 0;
        } else {
            if (i < 1 || j < 1) { bad = true; break; }
            const uint32_t nb = nib(i, j, &bad);
            if (bad) break;
            emit(1u, 1u);
            j--;
            state = (nb & 4u) ? 1 : 0;
        }
        if (nrev >= (int)cap - 1) { bad = true; break; }
    }
    WalkEnd w;
    w.bad = bad;
    if (bad) {
        w.n_rev = 0; w.i = 0; w.j = 0;
        return w;
    }
    if (mode == SA_GLOCAL && j > 0) { emit(1u, (uint32_t)j); j = 0; }   // window start reached
    if (cur_len) ops[nrev++] = (cur_len << 4) | cur_op;
    w.n_rev = nrev;
    w.i = i;
    w.j = j;
    return w;
}

}  // namespace sa

namespace sa {

// Traceback walk over stored heights (LOCAL, every score below 255): the walk
// re-derives each decision the direction nibbles would record, from the same
// DP values -- in state H at (i, j): the diagonal when H(i-1,j-1) + delta = H;
// else a deletion when H equals F(i,j) = max over k >= 1 of H(i-k,j) + S_GO +
// (k-1) S_GE, an insertion otherwise; a gap run extends from (i, j) while its
// value is strictly above H(neighbour) + S_GO -- so the CIGAR is the one the
// nibble walk gives.  E(i,j) (the same maximum up the column) is looked at first:
// below H it leaves the deletion as the only source, and only an E equal to H
// needs F.  height(ii, jj) gives the DP value or kNeg32 off the stored area (row
// 0 and column 0 are borders of value 0); match(ii, jj) tells whether window
// base ii equals read base jj.
//
// The walk is one flat loop that reads one height an iteration: the two gap scans
// are states of it (SCAN_E, SCAN_F), not inner loops, so a lane scanning a long
// row or column no longer holds the other lanes of its warp at every step.  A
// scan term H(i',j') + S_GO + (k-1) S_GE is bounded with H(i',j') <= hmax and,
// in LOCAL, H(i',j') <= a min(i',j') (a path to (i',j') has at most that many
// matches); once the bound is below H no later term can reach it, and the scan
// stops -- only its comparison with H is used, so the decisions are unchanged.
template <class Height, class Match>
__device__ __forceinline__ WalkEnd walk_heights(int i, int j, int32_t h, int imax, int rows, int32_t hmax,
                                                int32_t GO, int32_t GE, int32_t sa, int32_t sb, Height height,
                                                Match match, uint32_t* ops, uint32_t cap) {
    enum { kAtH = 0, kInsRun = 1, kDelRun = 2, kScanE = 3, kScanF = 4 };
    int nrev = 0;
    uint32_t cur_op = 15u, cur_len = 0;
    auto emit = [&](uint32_t op) {
        if (op == cur_op) { cur_len++; return; }
        if (cur_len) ops[nrev++] = (cur_len << 4) | cur_op;
        cur_op = op;
        cur_len = 1;
    };
    int32_t cur = 0, acc = kNeg32;                    // gap run value; a scan's running maximum
    int state = kAtH, kk = 0;
    int budget = 2 * (imax + rows) + 4;
    bool bad = (i < 1 || j < 1 || j > rows || i > imax || height(i, j) != h);
    while (!bad) {
        // the cell this iteration reads (ii < 0: none, the scan stops)
        int ii = -1, jj = 0;
        if (state == kScanE || state == kScanF) {
            const bool up = state == kScanE;
            const int n = up ? j : i;
            const int32_t hb = min(hmax, sa * (up ? j - kk : min(j, i - kk)));
            if (kk <= n && hb + GO + (kk - 1) * GE >= h) {
                ii = up ? i : i - kk;
                jj = up ? j - kk : j;
            }
        } else {
            if (--budget < 0 || nrev >= (int)cap - 1) { bad = true; break; }
            if (state == kAtH) {
                if (i == 0 || j == 0 || h <= 0) break;
                ii = i - 1;
                jj = j - 1;
            } else if (state == kDelRun) {
                if (i < 1) { bad = true; break; }
                ii = i - 1;
                jj = j;
            } else {
                if (j < 1) { bad = true; break; }
                ii = i;
                jj = j - 1;
            }
        }
        const int32_t hx = ii >= 0 ? height(ii, jj) : kNeg32;
        if (state == kAtH) {
            if (hx != kNeg32 && hx + (match(i, j) ? sa : sb) == h) {
                emit(0u);
                i--; j--; h = hx;
            } else {
                state = kScanE;
                kk = 1;
                acc = kNeg32;
                cur = h;
            }
        } else if (state == kScanE || state == kScanF) {
            bool stop = hx == kNeg32;                 // off the stored area or the bound: done
            if (!stop) {
                acc = max(acc, hx + GO + (kk - 1) * GE);
                stop = acc >= h;                      // F and E never exceed H: acc == h
            }
            if (!stop) {
                kk++;
            } else if (state == kScanE) {
                if (acc < h) state = kDelRun;         // F is the only source left
                else { state = kScanF; kk = 1; acc = kNeg32; }
            } else {
                state = (acc == h) ? kDelRun : kInsRun;
            }
        } else if (state == kDelRun) {
            emit(2u);
            i--;
            if (hx != kNeg32 && cur <= hx + GO) { state = kAtH; h = hx; }
            else cur -= GE;
        } else {
            emit(1u);
            j--;
            if (hx != kNeg32 && cur <= hx + GO) { state = kAtH; h = hx; }
            else cur -= GE;
        }
    }
    WalkEnd w;
    w.bad = bad;
    if (bad) {
        w.n_rev = 0; w.i = 0; w.j = 0;
        return w;
    }
    if (cur_len) ops[nrev++] = (cur_len << 4) | cur_op;
    w.n_rev = nrev;
    w.i = i;
    w.j = j;
    return w;
}

}  // namespace sa
