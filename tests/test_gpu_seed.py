"""GPU parity of the seeding front end (sa_seed_index_create,
sa_seed_candidates[_dev]) against the seeding oracle (oracle/seed.py), field by
field and bit-exact: candidate windows (position, length, strand flag, read),
their support and the per-read offsets; then the whole chain reads -> seeds ->
candidates -> effort limit -> alignment -> selection against the oracle chain."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import seed as OS
from oracle import select as OSel

pytestmark = pytest.mark.gpu

DEFAULT = dict(lam=20, step=10, max_occ=256, pad=24, join=16)


@pytest.fixture(scope="module")
def sa():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1302_5507_gb300 as sa
    return sa


def _reads_of_pairs(w):
    """One entry per read of a paired workload: offset and length of its sequence."""
    first = w.read_first.astype(np.int64)
    off = w.read_off[first[:-1]].astype(np.uint64)
    ln = w.read_len[first[:-1]].astype(np.uint32)
    return off, ln


def _check(sa, idx, ref, reads, off, ln, **kw):
    par = dict(DEFAULT)
    par.update(kw)
    jobs, sup, first = idx.candidates(reads, off, ln, sa.make_seed_params(
        seed_len=par["lam"], seed_step=par["step"], max_occ=par["max_occ"], pad=par["pad"], join=par["join"]))
    want, wfirst = OS.seed_candidates(ref, reads, off, ln, **par)
    assert np.array_equal(first.astype(np.int64), wfirst.astype(np.int64))
    for f in ("read_off", "read_len", "flags", "ref_pos", "win_len"):
        assert np.array_equal(jobs[f].astype(np.int64), want[f].astype(np.int64)), f
    assert np.array_equal(sup.astype(np.int64), want["support"].astype(np.int64))
    return jobs, sup, first


def test_paired_reads_match_the_oracle(sa):
    w = workloads.pairs(seed=3, n_pairs=400, genome_len=2_000_000, dup=0.3)
    off, ln = _reads_of_pairs(w)
    with sa.Reference(w.ref) as ref, sa.SeedIndex(ref) as idx:
        assert idx.info()["ref_len"] == len(w.ref)
        jobs, sup, first = _check(sa, idx, w.ref, w.reads, off, ln)
    # most reads find their source, on the strand they were sequenced from
    n_c = np.diff(first.astype(np.int64))
    assert (n_c > 0).mean() > 0.95


def _planted(with_long=False):
    rng = np.random.default_rng(21)
    ref = np.frombuffer(b"ACGT", np.uint8)[rng.integers(0, 4, 300_000)].copy()
    seg = ref[1000:1200].copy()
    for p in range(20_000, 300_000 - 400, 9_000):          # 31 copies of a 200-base segment
        ref[p:p + 200] = seg
    for p in (5_000, 150_000, 250_000):                     # homopolymer runs
        ref[p - 1] = ord("C")
        ref[p:p + 200] = ord("A")
        ref[p + 200] = ord("C")
    rc = {ord("A"): ord("T"), ord("C"): ord("G"), ord("G"): ord("C"), ord("T"): ord("A")}
    reads = [seg[20:170], np.full(150, ord("A"), np.uint8), ref[0:150].copy(), ref[-150:].copy(),
             ref[70_000:70_100].copy(), ref[80_000:80_019].copy(),
             np.array([rc[x] for x in seg[30:180][::-1]], np.uint8)]
    if with_long:
        reads.append(ref[90_000:91_024].copy())             # SA_MAX_READ bases
    off = np.concatenate([[0], np.cumsum([len(r) for r in reads[:-1]])]).astype(np.uint64)
    ln = np.array([len(r) for r in reads], np.uint32)
    return ref, np.concatenate(reads), off, ln


def test_repeats_homopolymers_and_edges(sa):
    """Planted repeats (hundreds of hits per strand: the block-sort path),
    homopolymer runs, reads at both reference ends, a read shorter than a seed
    and a reverse-complemented repeat read, under several parameter settings
    (seeds x max_occ stays within 8192 hits per strand); then with a read of
    SA_MAX_READ bases."""
    ref, reads, off, ln = _planted()
    with sa.Reference(ref) as r, sa.SeedIndex(r) as idx:
        jobs, sup, first = _check(sa, idx, ref, reads, off, ln, max_occ=585)
        _check(sa, idx, ref, reads, off, ln, step=16, max_occ=900)
        _check(sa, idx, ref, reads, off, ln, lam=12, step=8, max_occ=64, pad=0, join=0)
        _check(sa, idx, ref, reads, off, ln, lam=32, step=31, max_occ=200, pad=100, join=1000)
        _check(sa, idx, ref, reads, off, ln, lam=16, step=16, max_occ=100)
        n_c = np.diff(first.astype(np.int64))
        assert n_c[0] >= 32 and n_c[5] == 0       # the repeat read; the read shorter than a seed
        assert n_c[1] == 3                        # poly-A: one region per run
        assert n_c[6] >= 32 and (jobs["flags"][int(first[6]):int(first[7])] == sa.SA_RC).all()
    ref, reads, off, ln = _planted(with_long=True)
    with sa.Reference(ref) as r, sa.SeedIndex(r) as idx:
        _check(sa, idx, ref, reads, off, ln, step=16, max_occ=130)


def test_invalid_reads_and_small_buffers(sa):
    import torch
    ref, reads, off, ln = _planted()
    with sa.Reference(ref) as r, sa.SeedIndex(r) as idx:
        bad = reads.copy()
        bad[int(off[2]) + 5] = ord("N")
        with pytest.raises(sa.SAError) as e:
            idx.candidates(bad, off, ln)
        assert e.value.code == sa.SA_EINVAL and "read 2" in str(e.value)
        with pytest.raises(sa.SAError) as e:              # 1005 seeds per strand
            idx.candidates(reads, off, ln, sa.make_seed_params(seed_step=1))
        assert e.value.code == sa.SA_EINVAL
        with pytest.raises(sa.SAError) as e:              # seeds x max_occ above 8192
            idx.candidates(reads, off, ln, sa.make_seed_params(max_occ=5000))
        assert e.value.code == sa.SA_EINVAL
        with pytest.raises(sa.SAError) as e:
            idx.candidates(reads, off, ln, sa.make_seed_params(seed_len=11))
        assert e.value.code == sa.SA_EINVAL
        # device buffers too small: the count needed comes back, nothing is written
        p = sa.make_seed_params(seed_step=16, max_occ=500)
        _, want_sup, _ = idx.candidates(reads, off, ln, p)
        dev = torch.device("cuda:0")
        dr = torch.from_numpy(reads).to(dev)
        doff = torch.from_numpy(off.view(np.int64)).to(dev)
        dln = torch.from_numpy(ln.view(np.int32)).to(dev)
        small = torch.full((4 * 32,), 0x5A, dtype=torch.uint8, device=dev)
        dsup = torch.zeros(4, dtype=torch.int32, device=dev)
        dfirst = torch.zeros(len(ln) + 1, dtype=torch.int32, device=dev)
        with pytest.raises(sa.SAError) as e:
            idx.candidates_dev(dr, doff, dln, small, dsup, dfirst, p)
        assert e.value.code == sa.SA_EOVERFLOW and str(len(want_sup)) in str(e.value)
        assert (small.cpu().numpy() == 0x5A).all()
        big = torch.zeros(len(want_sup) * 32, dtype=torch.uint8, device=dev)
        bsup = torch.zeros(len(want_sup), dtype=torch.int32, device=dev)
        n = idx.candidates_dev(dr, doff, dln, big, bsup, dfirst, p)
        torch.cuda.synchronize()
        assert n == len(want_sup) and np.array_equal(bsup.cpu().numpy().astype(np.uint32), want_sup)


def test_reads_to_selection_on_the_device(sa):
    """The whole chain on device buffers -- seeds, candidates, effort limit (30),
    alignment with CIGAR, paired selection -- against the oracle's chain."""
    import torch
    w = workloads.pairs(seed=5, n_pairs=300, genome_len=2_000_000, dup=0.3)
    off, ln = _reads_of_pairs(w)
    dev = torch.device("cuda:0")
    sel = dict(paired=True, frag_min=300, frag_max=700)
    with sa.Reference(w.ref) as ref, sa.SeedIndex(ref) as idx:
        jobs, sup, first = idx.candidates(w.reads, off, ln)
        n = len(jobs)
        dr = torch.from_numpy(w.reads).to(dev)
        dc = torch.empty(n * 32, dtype=torch.uint8, device=dev)
        ds = torch.empty(n, dtype=torch.int32, device=dev)
        df = torch.empty(len(ln) + 1, dtype=torch.int32, device=dev)
        assert idx.candidates_dev(dr, torch.from_numpy(off.view(np.int64)).to(dev),
                                  torch.from_numpy(ln.view(np.int32)).to(dev), dc, ds, df) == n
        dk = torch.empty(n * 32, dtype=torch.uint8, device=dev)
        dfrom = torch.empty(n, dtype=torch.int32, device=dev)
        dkf = torch.empty(len(ln) + 1, dtype=torch.int32, device=dev)
        nk = ref.effort_limit_dev(dc, ds, df, 30, dk, dfrom, dkf)
        dres = torch.empty(nk * 56, dtype=torch.uint8, device=dev)
        dcig = torch.empty(int(nk) * (2 * 150 + 3), dtype=torch.int32, device=dev)
        ref.align_dev(dk[: nk * 32], dr, dres, dcig, sa.make_params())
        dout = torch.empty(len(ln) * 32, dtype=torch.uint8, device=dev)
        ref.select_dev(dk[: nk * 32], dres, dkf, dout, sa.make_select_params(**sel))
        torch.cuda.synchronize()
        got = dout.cpu().numpy().view(sa.READ_RESULT_DTYPE)
        kept_from = dfrom.cpu().numpy()[:nk].astype(np.int64)
    # the oracle chain
    cand, cfirst = OS.seed_candidates(w.ref, w.reads, off, ln, **DEFAULT)
    kept, kf = OSel.effort_limit(cand["support"].astype(np.int64), cfirst.astype(np.int64), 30)
    sub = workloads.Workload("seeded", w.ref, w.reads, cand["read_off"][kept], cand["read_len"][kept],
                             cand["flags"][kept], cand["ref_pos"][kept], cand["win_len"][kept],
                             cand["ref_pos"][kept])
    ores, _ = oracle.align(sub)
    exp = OSel.select(sub.flags, sub.read_len, ores, kf, **sel)
    assert np.array_equal(kept_from, kept.astype(np.int64))
    for f in ("job", "score", "second", "mapq", "flags", "n_cand", "frag_len"):
        assert np.array_equal(got[f].astype(np.int64), exp[f].astype(np.int64)), f
    # most fragments come out properly paired near their source
    assert (got["flags"] & sa.SA_READ_PROPER > 0).mean() > 0.9


def test_full_size_pairs_sampled(sa):
    """The benchmark's paired reads (100k pairs on the 100 Mbp genome) seeded in
    one call; a seeded sample of reads is recomputed by the oracle."""
    w = workloads.pairs(seed=1, n_pairs=100_000)
    off, ln = _reads_of_pairs(w)
    with sa.Reference(w.ref) as ref, sa.SeedIndex(ref) as idx:
        jobs, sup, first = idx.candidates(w.reads, off, ln)
    rng = np.random.default_rng(77)
    rows = np.sort(rng.choice(len(ln), 600, replace=False))
    table = OS.KmerTable(w.ref, 20)
    want, wfirst = OS.seed_candidates(w.ref, w.reads, off[rows], ln[rows], table=table, **DEFAULT)
    f = first.astype(np.int64)
    idx_c = np.concatenate([np.arange(f[r], f[r + 1]) for r in rows])
    assert np.array_equal(np.diff(wfirst.astype(np.int64)), (f[rows + 1] - f[rows]))
    for k in ("read_off", "read_len", "flags", "ref_pos", "win_len"):
        assert np.array_equal(jobs[k][idx_c].astype(np.int64), want[k].astype(np.int64)), k
    assert np.array_equal(sup[idx_c].astype(np.int64), want["support"].astype(np.int64))
