"""Pins of the CPU oracle beyond brute force: the paper's printed gap tolerance,
invariants, hand-worked golden cases, and the paper's second (register) form.
"""
import os
import random

import numpy as np
import pytest

import oracle
from bruteforce import GLOCAL, LOCAL

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT = (1, 2, 2, 1)


# ---------------------------------------------------------------------------
# Closed forms from the paper's default tolerance ("for a 100bp read, one gap up
# to 68bp, to 23 one-bp gaps"; Experiments, simulated data, and Variant Calling).
# A 100 bp read with one deletion of L bases scores 100a - (o + L e); with k
# isolated 1 bp deletions it scores 100a - k (o + e).  Under the default BWA-form
# scheme (a=1, o=2, e=1) the threshold 30 separates exactly as printed:
# L = 68 -> 30 (kept), 69 -> 29 (dropped); k = 23 -> 31 (kept), 24 -> 28 (dropped).

def _read_cgt(seed, n=100):
    rng = random.Random(seed)
    return "".join(rng.choice("CGT") for _ in range(n))


@pytest.mark.parametrize("L,expected", [(68, 30), (69, 29), (1, 97), (10, 88)])
def test_one_long_deletion(L, expected):
    # read over {C,G,T}, deleted block all A: an A can never match a read base, so the
    # only way across the block is the deletion itself (a mismatch costs 2 plus a lost match)
    read = _read_cgt(L)
    window = read[:50] + "A" * L + read[50:]
    r, cig = oracle.align_pair(window, read, scoring=DEFAULT, mode=oracle.GLOCAL)
    assert r["score"] == expected
    assert cig == f"50M{L}D50M"
    assert (r["ref_begin"], r["ref_end"]) == (0, len(window))


@pytest.mark.parametrize("k,expected", [(23, 31), (24, 28), (1, 97)])
def test_isolated_one_base_deletions(k, expected):
    read = _read_cgt(100 + k)
    cuts = [4 * (t + 1) for t in range(k)]        # deletions 4 bases apart
    window, last = "", 0
    for c in cuts:
        window += read[last:c] + "A"
        last = c
    window += read[last:]
    r, cig = oracle.align_pair(window, read, scoring=DEFAULT, mode=oracle.GLOCAL)
    assert r["score"] == expected
    assert cig.count("1D") == k


def test_default_scheme_reproduces_printed_tolerance():
    """Among small BWA-form schemes with a = 1, only gap open = 2 x gap extend (o = 2e)
    is consistent with both printed limits at a single threshold; (1, *, 2, 1) gives 30."""
    consistent = []
    for o in range(0, 9):
        for e in range(1, 5):
            one_gap = lambda L: 100 - (o + L * e)          # noqa: E731
            k_gaps = lambda k: 100 - k * (o + e)           # noqa: E731
            for s in range(1, 100):
                if one_gap(68) >= s > one_gap(69) and k_gaps(23) >= s > k_gaps(24):
                    consistent.append((o, e, s))
    assert (2, 1, 30) in consistent
    assert all(o == 2 * e for o, e, _ in consistent)


# ---------------------------------------------------------------------------
# invariants

@pytest.mark.parametrize("mode", [LOCAL, GLOCAL])
@pytest.mark.parametrize("scoring", [DEFAULT, (1, 4, 6, 1), (3, 2, 4, 2)])
def test_identical_strings_score_n_times_match(mode, scoring):
    rng = random.Random(5)
    for n in [1, 2, 7, 31, 100, 250]:
        s = "".join(rng.choice("ACGT") for _ in range(n))
        r, cig = oracle.align_pair(s, s, scoring=scoring, mode=mode)
        assert r["score"] == n * scoring[0]
        assert cig == f"{n}M"


def test_local_never_negative_and_glocal_spans_read():
    import workloads
    wl = workloads.small(3, 200, n_range=(1, 80), m_range=(1, 200), alphabet=2)
    loc, _ = oracle.align(wl, scoring=DEFAULT, mode=oracle.LOCAL)
    glo, _ = oracle.align(wl, scoring=DEFAULT, mode=oracle.GLOCAL)
    assert (loc["score"] >= 0).all()
    assert (glo["read_begin"] == 0).all() and (glo["read_end"] == wl.read_len.astype(np.int32)).all()
    # the local optimum dominates the glocal one (every glocal path is a local path)
    assert (loc["score"] >= glo["score"]).all()
    assert (glo["flags"] & oracle.EMPTY == 0).all()


def test_all_mismatch_is_empty_local_alignment():
    r, cig = oracle.align_pair("CCCCCCCC", "AAAA", scoring=DEFAULT, mode=oracle.LOCAL)
    assert r["score"] == 0 and r["flags"] & oracle.EMPTY and cig == ""
    assert r["second"] == oracle.NO_SCORE and r["second_ref_end"] == -1


def test_planted_duplicate_gives_second_equal_best():
    rng = random.Random(9)
    read = "".join(rng.choice("ACGT") for _ in range(40))
    spacer = "".join(rng.choice("ACGT") for _ in range(60))
    window = spacer[:10] + read + spacer + read + spacer[:5]
    r, _ = oracle.align_pair(window, read, scoring=DEFAULT, mode=oracle.LOCAL)
    assert r["score"] == 40 and r["second"] == 40
    assert r["ref_end"] == 10 + 40 and r["second_ref_end"] == 10 + 40 + 60 + 40


def test_reverse_complement_flag():
    import workloads
    wl = workloads.small(4, 50, n_range=(5, 30), m_range=(20, 60))
    res, ops = oracle.align(wl)
    flipped = wl.subset(slice(None))
    for k in range(wl.n_jobs):
        o, n = int(flipped.read_off[k]), int(flipped.read_len[k])
        seg = bytes(flipped.reads[o:o + n]).decode()
        if flipped.flags[k] & 1:
            seg = seg[::-1].translate(str.maketrans("ACGT", "TGCA"))
            flipped.reads[o:o + n] = np.frombuffer(seg.encode(), np.uint8)
    flipped.flags[:] = 0
    res2, ops2 = oracle.align(flipped)
    assert (res == res2).all()
    assert (ops == ops2).all()


def test_invalid_base_is_rejected():
    with pytest.raises(ValueError):
        oracle.align_pair("ACGTN", "ACG")


# ---------------------------------------------------------------------------
# hand-worked golden cases

def _golden():
    rows = []
    with open(os.path.join(HERE, "golden", "hand_cases.tsv")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append(line.rstrip("\n").split("\t"))
    return rows


@pytest.mark.parametrize("row", _golden(), ids=lambda r: f"{r[0]}-{r[2]}-{r[3]}")
def test_hand_worked(row):
    mode, sc, T, R, score, rb, re_, qb, qe, cig, second, second_end = row
    scoring = tuple(int(x) for x in sc.split(","))
    r, c = oracle.align_pair(T, R, scoring=scoring, mode=oracle.LOCAL if mode == "LOCAL" else oracle.GLOCAL)
    assert r["score"] == int(score)
    assert (r["ref_begin"], r["ref_end"], r["read_begin"], r["read_end"]) == \
        (int(rb), int(re_), int(qb), int(qe))
    assert c == ("" if cig == "*" else cig)
    assert r["second"] == (oracle.NO_SCORE if second == "NONE" else int(second))
    assert r["second_ref_end"] == int(second_end)


# ---------------------------------------------------------------------------
# the paper's second form: the row-register variant that keeps only the previous
# window row of M and D and carries M(i-1,j-1), M(i-1,j), V_M, V_I, V_D in scalars
# (Methods section 3, "Improved implementation").  Written here independently of the
# oracle's full-matrix fill; both must give the same scores.

def register_form(T, R, scoring, mode):
    a, b = scoring[0], -scoring[1]
    GO, GE = -(scoring[2] + scoring[3]), -scoring[3]
    NEG = -(2 ** 29)
    n = len(R)
    Mprev = [0] + [(GO + (j - 1) * GE) if mode == GLOCAL else 0 for j in range(1, n + 1)]
    Dprev = [NEG] * (n + 1)
    best = None if mode == GLOCAL else 0
    for i in range(1, len(T) + 1):
        m_up = 0           # M(i-1, 0)
        vm, vi = 0, NEG    # M(i, 0), I(i, 0)
        Mcur, Dcur = [0] * (n + 1), [NEG] * (n + 1)
        for j in range(1, n + 1):
            diag, m_up = m_up, Mprev[j]
            vi = max(vm + GO, vi + GE)
            vd = max(m_up + GO, Dprev[j] + GE)
            vm = max(diag + (a if T[i - 1] == R[j - 1] else b), vi, vd)
            if mode == LOCAL:
                vm = max(vm, 0)
                best = max(best, vm)
            Mcur[j], Dcur[j] = vm, vd
        if mode == GLOCAL:
            best = Mcur[n] if best is None else max(best, Mcur[n])
        Mprev, Dprev = Mcur, Dcur
    return best


@pytest.mark.parametrize("mode", [LOCAL, GLOCAL])
def test_register_form_agrees(mode):
    rng = random.Random(21 + mode)
    for _ in range(150):
        n, m = rng.randint(1, 30), rng.randint(1, 60)
        alpha = rng.choice(["AC", "ACGT"])
        T = "".join(rng.choice(alpha) for _ in range(m))
        R = "".join(rng.choice(alpha) for _ in range(n))
        scoring = rng.choice([DEFAULT, (1, 4, 6, 1), (2, 3, 5, 2)])
        r, _ = oracle.align_pair(T, R, scoring=scoring, mode=mode)
        assert r["score"] == register_form(T, R, scoring, mode)
