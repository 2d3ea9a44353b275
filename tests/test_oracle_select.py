"""Pin the read-level oracle (effort limit, best/second across candidates,
mapping quality, proper pairs) to closed forms and invariants (CPU).

The alignments come from the pinned DP oracle on planted sequences whose scores
are known in closed form (an exact copy of an n-base read scores n*a, a copy
with one substitution in the middle n*a - (a + b)), so every expected value
below follows from the construction, not from the code under test."""
import random

import numpy as np
import pytest

import oracle
from oracle import select as S

A, B, O, E = oracle.DEFAULT_SCORING
RC = {ord("A"): "T", ord("C"): "G", ord("G"): "C", ord("T"): "A"}


def revcomp(s: str) -> str:
    return "".join(RC[ord(c)] for c in reversed(s))


def random_genome(seed, n=20_000):
    rng = random.Random(seed)
    return [rng.choice("ACGT") for _ in range(n)]


def run(genome, reads, cands, **kw):
    """cands: per read a list of (window start, window length, rc flag).  Aligns
    every candidate with the DP oracle and selects."""
    g = "".join(genome)
    ref = np.frombuffer(g.encode(), np.uint8)
    read_buf = np.frombuffer("".join(reads).encode(), np.uint8)
    offs = np.cumsum([0] + [len(r) for r in reads])[:-1]
    read_off, read_len, flags, ref_pos, win_len, first = [], [], [], [], [], [0]
    for r, cl in enumerate(cands):
        for pos, m, rc in cl:
            read_off.append(offs[r]); read_len.append(len(reads[r])); flags.append(rc)
            ref_pos.append(pos); win_len.append(m)
        first.append(len(read_off))
    arr = lambda x, t: np.array(x, t)
    res, _ = oracle.align_arrays(ref, read_buf, arr(read_off, np.uint64), arr(read_len, np.uint32),
                                 arr(flags, np.uint32), arr(ref_pos, np.uint64), arr(win_len, np.uint32))
    out = S.select(arr(flags, np.uint32), arr(read_len, np.uint32), res, arr(first, np.int64),
                   match=A, mismatch=B, **kw)
    return out, res


def plant(genome, src, dst, n, sub_at=None):
    seg = genome[src:src + n]
    if sub_at is not None:
        seg = list(seg)
        seg[sub_at] = {"A": "C", "C": "G", "G": "T", "T": "A"}[seg[sub_at]]
    genome[dst:dst + n] = seg


# --- effort limit ---------------------------------------------------------------

def test_effort_limit_hand_example():
    kept, first = S.effort_limit([5, 1, 5, 3, 5, 2, 2], [0, 5, 7], 2)
    # read 0: supports 5,1,5,3,5 -> the two earliest 5s; read 1: both
    assert kept.tolist() == [0, 2, 5, 6]
    assert first.tolist() == [0, 2, 4]


def test_effort_limit_invariants():
    rng = random.Random(3)
    for _ in range(200):
        n_reads = rng.randint(1, 6)
        sizes = [rng.randint(0, 12) for _ in range(n_reads)]
        first = np.cumsum([0] + sizes)
        support = [rng.randint(0, 4) for _ in range(first[-1])]
        c = rng.randint(1, 8)
        kept, kf = S.effort_limit(support, first, c)
        assert (np.diff(kept) > 0).all() if len(kept) > 1 else True
        for r in range(n_reads):
            lo, hi = first[r], first[r + 1]
            mine = [k for k in kept if lo <= k < hi]
            assert kf[r + 1] - kf[r] == len(mine) == min(hi - lo, c)
            dropped = [k for k in range(lo, hi) if k not in mine]
            for k in mine:
                for d in dropped:
                    assert support[k] > support[d] or (support[k] == support[d] and k < d)


# --- mapping quality ------------------------------------------------------------

def test_mapq_closed_forms():
    assert S.mapq_of(100, S.NO_SCORE, A, B) == 60
    assert S.mapq_of(100, 100, A, B) == 0
    assert S.mapq_of(100, 101, A, B) == 0
    assert S.mapq_of(100, 97, A, B) == 20          # one mismatch-equivalent
    assert S.mapq_of(100, 99, A, B) == 6
    assert S.mapq_of(100, 91, A, B) == 60          # three mismatch-equivalents: capped


# --- single-end selection -------------------------------------------------------

def test_unique_read_gets_full_quality():
    g = random_genome(1)
    read = "".join(g[1000:1100])
    out, _ = run(g, [read], [[(5000, 200, 0), (950, 200, 0)]])
    r = out[0]
    assert r["job"] == 1 and r["score"] == 100 * A and r["mapq"] == 60
    assert r["flags"] == S.ALIGNED and r["n_cand"] == 2


def test_exact_repeat_is_ambiguous_and_the_smaller_end_wins():
    g = random_genome(2)
    plant(g, 1000, 8000, 100)
    read = "".join(g[1000:1100])
    out, _ = run(g, [read], [[(7950, 200, 0), (950, 200, 0)]])
    r = out[0]
    assert r["job"] == 1                      # equal scores: reference end 1100 < 8100
    assert r["score"] == 100 and r["second"] == 100 and r["mapq"] == 0


def test_one_substitution_copy_gives_twenty():
    g = random_genome(3)
    plant(g, 1000, 8000, 100, sub_at=50)
    read = "".join(g[1000:1100])
    out, _ = run(g, [read], [[(950, 200, 0), (7950, 200, 0)]])
    r = out[0]
    assert r["job"] == 0 and r["score"] == 100 and r["second"] == 100 - (A + B)
    assert r["mapq"] == 20


def test_overlapping_candidates_of_one_location_are_not_a_second_hit():
    g = random_genome(4)
    read = "".join(g[1000:1100])
    out, res = run(g, [read], [[(950, 200, 0), (960, 200, 0)]])
    assert res["ref_end"][0] == res["ref_end"][1] == 1100
    assert out[0]["mapq"] == 60 and out[0]["job"] == 0


def test_unaligned_read():
    g = random_genome(5)
    out, _ = run(g, ["ACGT"], [[]])
    r = out[0]
    assert r["job"] == S.NO_JOB and r["flags"] == 0 and r["mapq"] == 0 and r["second"] == S.NO_SCORE


# --- pairs ----------------------------------------------------------------------

def _pair_setup(seed, end2_rc=True):
    g = random_genome(seed)
    plant(g, 2400, 500, 100)                  # a copy of end 2's source upstream
    end1 = "".join(g[2000:2100])
    end2 = "".join(g[2400:2500])
    if end2_rc:
        end2 = revcomp(end2)
    rc = 1 if end2_rc else 0
    cands = [[(1950, 200, 0)], [(450, 200, rc), (2350, 200, rc)]]
    return g, [end1, end2], cands


def test_proper_pair_resolves_a_repeat():
    g, reads, cands = _pair_setup(6)
    single, _ = run(g, reads, cands)
    assert single[1]["job"] == 1 and single[1]["mapq"] == 0      # the copy (end 600) wins alone
    out, _ = run(g, reads, cands, paired=True, frag_min=400, frag_max=600)
    e1, e2 = out[0], out[1]
    assert e1["job"] == 0 and e2["job"] == 2                     # the proper placement
    both = S.ALIGNED | S.PAIRED | S.PROPER | S.MATE_ALIGNED
    assert e1["flags"] == both and e2["flags"] == both | S.REVERSE
    assert e1["frag_len"] == e2["frag_len"] == 500
    assert e2["second"] == 100                                   # the copy is still a hit
    assert e2["mapq"] == 60 and e1["mapq"] == 60                 # but the pair is unique


def test_out_of_range_fragment_falls_back_to_single_ends():
    g, reads, cands = _pair_setup(6)
    out, _ = run(g, reads, cands, paired=True, frag_min=100, frag_max=300)
    e1, e2 = out[0], out[1]
    assert e2["job"] == 1 and e2["mapq"] == 0                    # alone again
    assert e1["flags"] == S.ALIGNED | S.PAIRED | S.MATE_ALIGNED
    assert e2["flags"] == S.ALIGNED | S.PAIRED | S.MATE_ALIGNED | S.REVERSE
    assert e1["frag_len"] == 0


def test_orientation():
    g, reads, cands = _pair_setup(7)
    out, _ = run(g, reads, cands, paired=True, orientation=S.PAIR_FF, frag_min=400, frag_max=600)
    assert not out[0]["flags"] & S.PROPER                        # FR reads are not FF
    g, reads, cands = _pair_setup(7, end2_rc=False)
    out, _ = run(g, reads, cands, paired=True, orientation=S.PAIR_FF, frag_min=400, frag_max=600)
    assert out[0]["flags"] & S.PROPER and out[1]["job"] == 2 and out[0]["frag_len"] == 500
    out, _ = run(g, reads, cands, paired=True, orientation=S.PAIR_FR, frag_min=400, frag_max=600)
    assert not out[0]["flags"] & S.PROPER


def test_reverse_end_first_is_still_fr():
    """End 1 reverse-complemented at the right, end 2 forward at the left."""
    g = random_genome(8)
    end1 = revcomp("".join(g[2400:2500]))
    end2 = "".join(g[2000:2100])
    out, _ = run(g, [end1, end2], [[(2350, 200, 1)], [(1950, 200, 0)]], paired=True,
                 frag_min=400, frag_max=600)
    assert out[0]["flags"] & S.PROPER and out[0]["frag_len"] == 500


def test_pair_ambiguity_keeps_a_unique_end_confident():
    """End 2 has two proper placements 150 bases apart (a planted copy of its
    source): the pair is ambiguous, end 1 on its own is not."""
    g = random_genome(9)
    plant(g, 2400, 2250, 100)                 # a second copy of end 2's source, 150 upstream
    end1 = "".join(g[2000:2100])
    end2 = revcomp("".join(g[2400:2500]))
    out, _ = run(g, [end1, end2], [[(1950, 200, 0)], [(2200, 200, 1), (2350, 200, 1)]],
                 paired=True, frag_min=300, frag_max=600)
    e1, e2 = out[0], out[1]
    assert e1["flags"] & S.PROPER
    assert e2["job"] == 1 and e2["frag_len"] == 350               # smaller job index on equal sums
    assert e2["mapq"] == 0 and e1["mapq"] == 60


@pytest.mark.parametrize("seed", [11, 12])
def test_gapped_begin_without_traceback_uses_the_read_length(seed):
    """Without a traceback (ref_begin -1) the forward end's first base is taken
    as ref_end - n."""
    res = np.zeros(2, oracle.RESULT_DTYPE)
    res["score"] = [90, 95]
    res["second"] = S.NO_SCORE
    res["second_ref_end"] = -1
    res["ref_begin"] = -1
    res["ref_end"] = [1100, 1600]
    out = S.select(np.array([0, 1], np.uint32), np.array([100, 100], np.uint32), res,
                   np.array([0, 1, 2]), paired=True, frag_min=600, frag_max=600)
    assert out[0]["frag_len"] == 600 and out[0]["flags"] & S.PROPER


# --- invariants on random result tables -----------------------------------------

def _random_results(rng, n_reads, paired):
    """Per-read candidate lists with random scores, ends, seconds and flags."""
    sizes = rng.integers(0, 6, n_reads)
    first = np.zeros(n_reads + 1, np.int64)
    first[1:] = np.cumsum(sizes)
    n = int(first[-1])
    res = np.zeros(n, oracle.RESULT_DTYPE)
    res["score"] = rng.integers(1, 60, n)
    res["ref_end"] = rng.integers(100, 3000, n)
    res["ref_begin"] = np.where(rng.random(n) < 0.5, res["ref_end"] - rng.integers(20, 60, n), -1)
    has2 = rng.random(n) < 0.6
    res["second"] = np.where(has2, np.minimum(res["score"], rng.integers(0, 60, n)), S.NO_SCORE)
    res["second_ref_end"] = np.where(has2, rng.integers(100, 3000, n), -1)
    res["flags"] = np.where(rng.random(n) < 0.15, S.EMPTY, 0)
    flags = (rng.random(n) < 0.5).astype(np.uint32)
    read_len = np.full(n, 50, np.uint32)
    return flags, read_len, res, first


@pytest.mark.parametrize("paired", [False, True])
def test_selection_invariants(paired):
    rng = np.random.default_rng(17 + paired)
    for _ in range(40):
        n_reads = 2 * int(rng.integers(1, 8))
        flags, read_len, res, first = _random_results(rng, n_reads, paired)
        out = S.select(flags, read_len, res, first, paired=paired, frag_min=50, frag_max=400)
        for r in range(n_reads):
            o = out[r]
            lo, hi = int(first[r]), int(first[r + 1])
            assert o["n_cand"] == hi - lo
            aligned = [j for j in range(lo, hi) if not res["flags"][j] & (S.EMPTY | S.BELOW_MIN)]
            if not aligned:
                assert o["job"] == S.NO_JOB and not o["flags"] & S.ALIGNED and o["mapq"] == 0
                continue
            assert lo <= o["job"] < hi and o["job"] in aligned and o["flags"] & S.ALIGNED
            assert o["score"] == res["score"][o["job"]]
            assert 0 <= o["mapq"] <= S.MAPQ_MAX
            assert bool(o["flags"] & S.REVERSE) == bool(flags[o["job"]] & 1)
            if o["flags"] & S.PROPER:
                assert paired and o["flags"] & S.PAIRED and o["flags"] & S.MATE_ALIGNED
                assert 50 <= o["frag_len"] <= 400
            else:
                assert o["frag_len"] == 0
                # on its own: the best aligned candidate and a second that is not better
                best = max(int(res["score"][j]) for j in aligned)
                assert o["score"] == best
                assert o["second"] == S.NO_SCORE or o["second"] <= best
            assert bool(o["flags"] & S.PAIRED) == paired
        if paired:
            for p in range(n_reads // 2):
                a, b = out[2 * p], out[2 * p + 1]
                assert bool(a["flags"] & S.PROPER) == bool(b["flags"] & S.PROPER)
                if a["flags"] & S.PROPER:
                    assert a["frag_len"] == b["frag_len"]
