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
