"""Pin the CPU oracle to exhaustive enumeration of alignments (no DP on this side).

For tiny reads and windows every alignment path is enumerated (tests/bruteforce.py)
and scored with the affine convention of the paper's recurrence (Methods section 3:
first gap base S_GO, each further one S_GE).  The oracle must return

* the maximum score (LOCAL floor 0; GLOCAL whole read),
* the end cell that the scan order fixes: smallest reference end, then smallest read end,
* the traceback that the priority rule fixes: among optimal paths ending at that cell,
  the one whose reversed op string is smallest under stop < M < D < I,
* the second best over window columns at distance >= n from the best end.
"""
import itertools
import random

import numpy as np
import pytest

import oracle
from bruteforce import LOCAL, GLOCAL, best_score, colbest, enumerate_paths, rescore

SCHEMES = [(1, 2, 2, 1), (1, 4, 6, 1), (2, 3, 5, 2), (3, 1, 0, 1), (1, 1, 1, 0), (2, 5, 1, 3)]
MODES = [LOCAL, GLOCAL]


def parse_cigar(ops):
    return [("MIDNSHP=X"[int(x) & 15], int(x) >> 4) for x in ops]


def expected(T, R, scoring, mode):
    """Everything the oracle returns, derived from the path enumeration."""
    n = len(R)
    paths = [p for p in enumerate_paths(T, R, scoring, mode) if not (mode == GLOCAL and p[3] < 1)]
    best = best_score(T, R, scoring, mode)
    if mode == LOCAL and best == 0:
        return dict(score=0, empty=True)
    opt = [p for p in paths if p[0] == best]
    # end cell: smallest (i1, j1)
    i1, j1 = min((p[3], p[4]) for p in opt)
    at_end = [p for p in opt if (p[3], p[4]) == (i1, j1)]
    rank = {"M": 1, "D": 2, "I": 3}
    chosen = min(at_end, key=lambda p: [rank[c] for c in reversed(p[5])])
    cb = colbest(T, R, scoring, mode)
    cand = [(v, i) for i, v in enumerate(cb, start=1) if abs(i - i1) >= n]
    if cand:
        sv = max(v for v, _ in cand)
        si = min(i for v, i in cand if v == sv)
    else:
        sv, si = oracle.NO_SCORE, None
    return dict(score=best, empty=False, ref_end=i1, read_end=j1, ref_begin=chosen[1],
                read_begin=chosen[2], ops=chosen[5], second=sv, second_end=si)


def compress(ops):
    return [(k, len(list(g))) for k, g in itertools.groupby(ops)]


def check(T, R, scoring, mode):
    exp = expected(T, R, scoring, mode)
    r, cig = oracle.align_pair(T, R, scoring=scoring, mode=mode)
    ctx = f"T={T} R={R} scoring={scoring} mode={mode}"
    assert r["score"] == exp["score"], ctx
    if exp["empty"]:
        assert r["flags"] & oracle.EMPTY, ctx
        assert r["ref_end"] == -1 and r["read_end"] == -1 and r["n_ops"] == 0, ctx
        return
    assert (r["ref_end"], r["read_end"]) == (exp["ref_end"], exp["read_end"]), ctx
    assert (r["ref_begin"], r["read_begin"]) == (exp["ref_begin"], exp["read_begin"]), ctx
    ops = [(op, L) for op, L in _parse(cig) if op != "S"]
    assert ops == compress(exp["ops"]), ctx + f" cigar={cig}"
    assert r["second"] == exp["second"], ctx
    assert r["second_ref_end"] == (exp["second_end"] if exp["second_end"] is not None else -1), ctx


def _parse(cig):
    out, num = [], ""
    for c in cig:
        if c.isdigit():
            num += c
        else:
            out.append((c, int(num)))
            num = ""
    return out


@pytest.mark.parametrize("mode", MODES)
def test_exhaustive_two_letter_tiny(mode):
    """Every read of length 1..3 against every window of length 1..4 over {A, C}."""
    for scoring in [(1, 2, 2, 1), (2, 1, 1, 1)]:
        for n in range(1, 4):
            for m in range(1, 5):
                for R in itertools.product("AC", repeat=n):
                    for T in itertools.product("AC", repeat=m):
                        check("".join(T), "".join(R), scoring, mode)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("scoring", SCHEMES)
def test_random_small(mode, scoring):
    rng = random.Random(hash((mode, scoring)) & 0xFFFF)
    for _ in range(25):
        n = rng.randint(1, 4)
        m = rng.randint(1, 6)
        alpha = rng.choice(["AC", "ACG", "ACGT"])
        T = "".join(rng.choice(alpha) for _ in range(m))
        R = "".join(rng.choice(alpha) for _ in range(n))
        check(T, R, scoring, mode)


@pytest.mark.parametrize("mode", MODES)
def test_random_n5_m7(mode):
    rng = random.Random(7 + mode)
    for _ in range(6):
        T = "".join(rng.choice("ACGT") for _ in range(7))
        R = "".join(rng.choice("ACGT") for _ in range(5))
        check(T, R, (1, 2, 2, 1), mode)


def test_cigar_rescores_to_score_on_workload():
    """Rescoring every CIGAR reproduces the score; op lengths are consistent."""
    import workloads
    wl = workloads.small(11, 300, n_range=(1, 60), m_range=(1, 150))
    for mode in MODES:
        for scoring in [(1, 2, 2, 1), (1, 4, 6, 1)]:
            res, ops = oracle.align(wl, scoring=scoring, mode=mode)
            for k in range(wl.n_jobs):
                r = res[k]
                n = int(wl.read_len[k])
                o = int(wl.read_off[k])
                read = bytes(wl.reads[o:o + n]).decode()
                if wl.flags[k] & 1:
                    read = read[::-1].translate(str.maketrans("ACGT", "TGCA"))
                pos = int(wl.ref_pos[k])
                T = bytes(wl.ref[pos:pos + int(wl.win_len[k])]).decode()
                if r["flags"] & oracle.EMPTY:
                    assert mode == LOCAL and r["score"] == 0 and r["n_ops"] == 0
                    continue
                cig = parse_cigar(ops[k][: r["n_ops"]])
                sc, i_end, j_end = rescore(T, read, int(r["ref_begin"]) - pos,
                                           int(r["read_begin"]), cig, scoring)
                assert sc == r["score"]
                assert i_end == r["ref_end"] - pos and j_end == r["read_end"]
                read_ops = sum(L for op, L in cig if op in "MIS")
                assert read_ops == n
                if mode == GLOCAL:
                    assert all(op != "S" for op, _ in cig)
                    assert r["read_begin"] == 0 and r["read_end"] == n
                else:
                    assert r["score"] >= 0
                    # a local alignment starts and ends with a match column
                    core = [op for op, _ in cig if op != "S"]
                    assert core[0] == "M" and core[-1] == "M"


# Schemes where an insertion and a deletion cost less than a mismatch, and where
# opening and extending a gap tie, so the traceback priority and the open-on-tie
# rule decide between several optimal paths.
TIE_SCHEMES = [(1, 10, 0, 1), (1, 5, 1, 1), (2, 9, 1, 1), (3, 8, 0, 2), (1, 3, 1, 0)]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("scoring", TIE_SCHEMES)
def test_tie_rich_small(mode, scoring):
    rng = random.Random(1000 + 7 * mode + scoring[1])
    for _ in range(60):
        n = rng.randint(2, 3)
        m = rng.randint(4, 8)
        T = "".join(rng.choice("AC") for _ in range(m))
        R = "".join(rng.choice("AC") for _ in range(n))
        check(T, R, scoring, mode)


def test_free_extension_tie_cases():
    """With a free gap extension (e = 0) long and short deletions tie; opening on
    ties makes the walk leave the gap as early as possible (found by search)."""
    for T, R in [("ACCCAACA", "CAC"), ("CAACAACC", "CCC"), ("ACCCAAAC", "CCAAC")]:
        check(T, R, (1, 3, 1, 0), GLOCAL)
