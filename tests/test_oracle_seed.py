"""Pins of the seeding oracle (oracle/seed.py): closed forms of planted
structures and a brute-force occurrence scan on tiny inputs.

Every expected value here follows from the definition of the step (seeds at
regular intervals on both strands, exact occurrences, diagonals, regions cut
where diagonals jump by more than `join`, support = distinct seeds) and the
planted sequence, not from the oracle's code."""
import numpy as np
import pytest

from oracle import seed as S

LAM, STEP, PAD, JOIN = 20, 10, 24, 16


def _rand(rng, n):
    return np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, n)].copy()


def _rc(s):
    comp = {ord("A"): ord("T"), ord("C"): ord("G"), ord("G"): ord("C"), ord("T"): ord("A")}
    return np.array([comp[x] for x in s[::-1]], np.uint8)


def _cands(ref, reads, **kw):
    reads = [np.asarray(r, np.uint8) for r in reads]
    off = np.concatenate([[0], np.cumsum([len(r) for r in reads[:-1]])]).astype(np.uint64)
    n = np.array([len(r) for r in reads], np.uint32)
    par = dict(lam=LAM, step=STEP, max_occ=256, pad=PAD, join=JOIN)
    par.update(kw)
    return S.seed_candidates(ref, np.concatenate(reads), off, n, **par)


def n_seeds(n, lam=LAM, step=STEP):
    return 0 if n < lam else (n - lam) // step + 1


def test_planted_repeats_give_one_full_support_region_each():
    rng = np.random.default_rng(1)
    ref = _rand(rng, 60_000)
    seg = _rand(rng, 200)
    at = [5_000, 17_000, 33_333, 51_000]
    for p in at:
        ref[p:p + 200] = seg
    read = seg[20:170]
    c, first = _cands(ref, [read])
    assert list(first) == [0, 4]
    assert list(c["flags"]) == [0] * 4
    assert list(c["ref_pos"]) == [p + 20 - PAD for p in at]
    assert list(c["win_len"]) == [150 + 2 * PAD] * 4
    assert list(c["support"]) == [n_seeds(150)] * 4
    # the same read reverse-complemented: the regions move to the other strand
    c2, first2 = _cands(ref, [_rc(read)])
    assert list(first2) == [0, 4] and list(c2["flags"]) == [S.FLAG_RC] * 4
    assert list(c2["ref_pos"]) == list(c["ref_pos"]) and list(c2["support"]) == list(c["support"])


def test_substitution_removes_the_seeds_that_cover_it():
    rng = np.random.default_rng(2)
    ref = _rand(rng, 40_000)
    read = ref[10_000:10_150].copy()
    for x in (0, 5, 19, 20, 75, 149):
        mut = read.copy()
        mut[x] = ord("A") if mut[x] != ord("A") else ord("C")
        covering = sum(1 for k in range(n_seeds(150)) if k * STEP <= x < k * STEP + LAM)
        c, first = _cands(ref, [mut])
        assert list(first) == [0, 1]
        assert c["support"][0] == n_seeds(150) - covering
        assert c["ref_pos"][0] == 10_000 - PAD and c["win_len"][0] == 150 + 2 * PAD


def test_deletion_splits_or_joins_by_the_diagonal_gap():
    rng = np.random.default_rng(3)
    ref = _rand(rng, 40_000)
    # the read skips 3 reference bases after its 75th base: seeds after the gap
    # imply a diagonal 3 larger
    read = np.concatenate([ref[20_000:20_075], ref[20_078:20_153]])
    before = sum(1 for k in range(n_seeds(150)) if k * STEP + LAM <= 75)
    after = sum(1 for k in range(n_seeds(150)) if k * STEP >= 75)
    c, _ = _cands(ref, [read], join=3)
    assert list(c["support"]) == [before + after]
    assert c["ref_pos"][0] == 20_000 - PAD and c["win_len"][0] == 150 + 3 + 2 * PAD
    c, _ = _cands(ref, [read], join=2)
    assert list(c["support"]) == [before, after]
    assert list(c["ref_pos"]) == [20_000 - PAD, 20_003 - PAD]


def test_homopolymer_read_and_the_repetitive_seed_cap():
    rng = np.random.default_rng(4)
    ref = _rand(rng, 80_000)
    runs = [10_000, 40_000, 70_000]
    for p in runs:
        ref[p:p + 200] = ord("A")
        ref[p - 1] = ref[p + 200] = ord("C")      # the runs are exactly 200 long
    read = np.full(150, ord("A"), np.uint8)
    occ_per_seed = 3 * (200 - LAM + 1)
    c, first = _cands(ref, [read], max_occ=occ_per_seed)
    # every seed is A^LAM: its hits on one run imply diagonals p - o for p in
    # [R, R + 200 - LAM] and o in {0, 10, ..., 130}: the contiguous range
    # [R - 130, R + 180], one region per run
    assert list(first) == [0, 3]
    assert list(c["flags"]) == [0, 0, 0]
    assert list(c["support"]) == [n_seeds(150)] * 3
    assert list(c["ref_pos"]) == [R - 130 - PAD for R in runs]
    assert list(c["win_len"]) == [(R + 180 + 150 + PAD) - (R - 130 - PAD) for R in runs]
    # one occurrence more than the cap allows: every seed is too repetitive
    c, first = _cands(ref, [read], max_occ=occ_per_seed - 1)
    assert list(first) == [0, 0]


def test_reference_edges_clamp_the_window():
    rng = np.random.default_rng(5)
    ref = _rand(rng, 30_000)
    c, _ = _cands(ref, [ref[0:150], ref[30_000 - 150:]])
    assert list(c["ref_pos"]) == [0, 30_000 - 150 - PAD]
    assert list(c["win_len"]) == [150 + PAD, 150 + PAD]


def test_join_merges_nearby_copies_into_one_window():
    rng = np.random.default_rng(6)
    ref = _rand(rng, 30_000)
    seg = _rand(rng, 150)
    ref[10_000:10_150] = seg
    ref[10_300:10_450] = seg
    c, _ = _cands(ref, [seg], join=299)
    assert list(c["support"]) == [n_seeds(150), n_seeds(150)]
    c, _ = _cands(ref, [seg], join=300)
    assert list(c["support"]) == [n_seeds(150)]
    assert c["ref_pos"][0] == 10_000 - PAD and c["win_len"][0] == 300 + 150 + 2 * PAD


def test_seed_count_and_short_reads():
    rng = np.random.default_rng(7)
    ref = _rand(rng, 20_000)
    c, first = _cands(ref, [ref[100:100 + LAM - 1], ref[500:500 + LAM], ref[900:900 + LAM + STEP]])
    assert list(first) == [0, 0, 1, 2]
    assert list(c["support"]) == [1, 2]


def test_occurrences_match_a_brute_force_scan():
    """Tiny two-letter references: every occurrence list equals the positions a
    plain substring comparison finds."""
    rng = np.random.default_rng(8)
    for lam in (3, 5, 8):
        ref = np.frombuffer(b"AC", np.uint8)[rng.integers(0, 2, 400)].copy()
        t = S.KmerTable(ref, lam)
        s = ref.tobytes()
        for _ in range(50):
            p0 = int(rng.integers(0, 400 - lam))
            seed = ref[p0:p0 + lam]
            want = [p for p in range(400 - lam + 1) if s[p:p + lam] == seed.tobytes()]
            got = t.occurrences(S.kmer_code(S.codes(seed))).tolist()
            assert got == want


def test_invalid_base_is_refused():
    with pytest.raises(ValueError):
        S.codes(np.frombuffer(b"ACGN", np.uint8))
