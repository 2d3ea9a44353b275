"""The gapless traceback rule of the traceback classification, checked against the
oracle's full-matrix traceback (no GPU).

Let c_m be the score of the m diagonal cells ending at the best cell (i*, j*).
When c_k equals the best score (LOCAL: the first such k; GLOCAL: k = j*, the run
starting on row 0), every H on the run is forced (at least the run's prefix score,
at most the next cell's H minus its delta), and the traceback, which takes the
diagonal first on ties (Methods section 3), walks exactly that run.  So the CIGAR
between the soft clips is k matches/mismatches and the alignment begins k cells
before its end.  The GPU path gives such jobs no direction pass; these cases pin
the rule on the oracle's own results, over schemes with and without a gap-extend
cost, both modes, a two-letter alphabet (many ties) and gapped low-similarity jobs.
"""
import numpy as np
import pytest

import oracle
import workloads

COMP = bytes.maketrans(b"ACGT", b"TGCA")
SCHEMES = [(1, 2, 2, 1), (1, 4, 6, 1), (2, 3, 5, 2), (1, 3, 1, 0), (3, 1, 0, 1), (1, 10, 0, 1)]


def job_read(wl, k):
    o, n = int(wl.read_off[k]), int(wl.read_len[k])
    s = wl.reads[o:o + n].tobytes()
    if int(wl.flags[k]) & workloads.FLAG_RC:
        s = s.translate(COMP)[::-1]
    return s


def gapless_steps(window, read, istar, jstar, best, scoring, mode):
    """k of the rule, or 0 (written from the rule's statement, not from the kernel)."""
    a, b = scoring[0], -scoring[1]
    if mode == oracle.GLOCAL and jstar > istar:
        return 0
    c = 0
    for m in range(1, min(istar, jstar) + 1):
        c += a if window[istar - m] == read[jstar - m] else b
        if mode == oracle.LOCAL and c == best:
            return m
    return jstar if (mode == oracle.GLOCAL and c == best) else 0


def check(wl, scoring, mode):
    res, ops = oracle.align(wl, scoring=scoring, mode=mode)
    fired = 0
    for k in range(wl.n_jobs):
        r = res[k]
        if int(r["flags"]) & oracle.EMPTY or int(r["read_end"]) <= 0:
            continue
        pos, m = int(wl.ref_pos[k]), int(wl.win_len[k])
        window = wl.ref[pos:pos + m].tobytes()
        read = job_read(wl, k)
        istar, jstar, best = int(r["ref_end"]) - pos, int(r["read_end"]), int(r["score"])
        steps = gapless_steps(window, read, istar, jstar, best, scoring, mode)
        if not steps:
            continue
        fired += 1
        core = [int(x) for x in ops[k][: int(r["n_ops"])] if int(x) & 15 != 4]   # drop soft clips
        assert core == [(steps << 4) | 0], (k, steps, core)
        assert int(r["read_begin"]) == jstar - steps, (k, steps, int(r["read_begin"]))
        assert int(r["ref_begin"]) == pos + istar - steps, (k, steps, int(r["ref_begin"]))
    return fired


@pytest.mark.parametrize("scoring", SCHEMES)
@pytest.mark.parametrize("mode", [oracle.LOCAL, oracle.GLOCAL])
@pytest.mark.parametrize("alphabet", [4, 2])
def test_gapless_rule_small_random(scoring, mode, alphabet):
    wl = workloads.small(seed=11 + alphabet, n_jobs=1500, alphabet=alphabet)
    assert check(wl, scoring, mode) > 0


@pytest.mark.parametrize("scoring", [(1, 2, 2, 1), (1, 4, 6, 1)])
@pytest.mark.parametrize("mode", [oracle.LOCAL, oracle.GLOCAL])
def test_gapless_rule_uneven_and_low_similarity(scoring, mode):
    for wl in (workloads.uneven(seed=4, n_jobs=800, genome_len=2_000_000),
               workloads.lowsim(seed=4, n_jobs=150, genome_len=2_000_000)):
        assert check(wl, scoring, mode) > 0
