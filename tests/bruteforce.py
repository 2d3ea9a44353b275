"""Exhaustive enumeration of alignments (test helper, independent of the oracle).

An alignment of read R (length n) inside window T (length m) is a start cell
(i0, j0) and a string over {M, I, D}: M consumes T[i] and R[j], I consumes
R[j] only (read base against a space), D consumes T[i] only.  Its score is
the sum of the match/mismatch scores of its M columns plus, for every
*maximal* run of I or of D of length L, S_GO + (L-1) * S_GE (the paper's
convention: the first gap base costs S_GO, each further one S_GE).

LOCAL: every start cell, every end cell, plus the empty alignment (score 0).
GLOCAL: starts on row 0 (j0 = 0) at any column, must consume the whole read.

This walks every path explicitly (no dynamic programming), so it is only for
tiny inputs (n <= 5, m <= 7).
"""
from __future__ import annotations

LOCAL, GLOCAL = 0, 1


def signed(scoring):
    a, b, o, e = scoring
    return a, -b, -(o + e), -e


def enumerate_paths(T: str, R: str, scoring, mode):
    """Yield (score, i0, j0, i1, j1, ops) for every alignment path."""
    a, b, GO, GE = signed(scoring)
    m, n = len(T), len(R)
    starts = [(i0, j0) for i0 in range(m + 1) for j0 in range(n + 1)] if mode == LOCAL \
        else [(i0, 0) for i0 in range(m + 1)]
    for i0, j0 in starts:
        # iterative DFS over (i, j, last_op, score, ops)
        stack = [(i0, j0, "", 0, "")]
        while stack:
            i, j, last, sc, ops = stack.pop()
            if ops:
                if mode == LOCAL or j == n:
                    yield sc, i0, j0, i, j, ops
            if i < m and j < n:
                stack.append((i + 1, j + 1, "M", sc + (a if T[i] == R[j] else b), ops + "M"))
            if j < n:
                stack.append((i, j + 1, "I", sc + (GE if last == "I" else GO), ops + "I"))
            if i < m:
                stack.append((i + 1, j, "D", sc + (GE if last == "D" else GO), ops + "D"))


def best_score(T: str, R: str, scoring, mode):
    best = 0 if mode == LOCAL else None
    for sc, i0, j0, i1, j1, ops in enumerate_paths(T, R, scoring, mode):
        if mode == GLOCAL and i1 < 1:
            continue  # the recurrence's result ranges over columns 1..m
        if best is None or sc > best:
            best = sc
    return best


def colbest(T: str, R: str, scoring, mode):
    """colbest(i) for i = 1..m: the best path ending in window column i
    (LOCAL: any read row, floor 0; GLOCAL: ending on the last read row)."""
    m = len(T)
    cb = [0 if mode == LOCAL else None] * (m + 1)
    for sc, i0, j0, i1, j1, ops in enumerate_paths(T, R, scoring, mode):
        if i1 >= 1 and j1 >= 1 and (cb[i1] is None or sc > cb[i1]):
            cb[i1] = sc
    return cb[1:]


def rescore(T: str, R: str, ref_begin: int, read_begin: int, cigar_ops, scoring):
    """Score a CIGAR (list of (op_char, length)) placed at (ref_begin, read_begin);
    returns (score, ref_end, read_end).  Soft clips are skipped."""
    a, b, GO, GE = signed(scoring)
    i, j, sc = ref_begin, read_begin, 0
    for op, L in cigar_ops:
        if op == "S":
            continue
        if op == "M":
            for _ in range(L):
                sc += a if T[i] == R[j] else b
                i += 1
                j += 1
        elif op == "I":
            sc += GO + (L - 1) * GE
            j += L
        elif op == "D":
            sc += GO + (L - 1) * GE
            i += L
    return sc, i, j
