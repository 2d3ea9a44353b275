"""Reads with several candidate windows: the effort limit and the per-read /
per-pair selection of the CUDA library against the oracle (field by field).

The oracle side runs entirely on the CPU (oracle.select.effort_limit, the DP
oracle on the kept jobs, oracle.select.select); the GPU side runs the library's
effort limit, alignment and selection on the same seeded inputs."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import select as S

pytestmark = pytest.mark.gpu

FIELDS = ("job", "score", "second", "mapq", "flags", "n_cand", "frag_len")


@pytest.fixture(scope="module")
def sa():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1302_5507_gb300 as sa
    return sa


def _diff(got, exp, what):
    bad = []
    for f in FIELDS:
        idx = np.nonzero(got[f].astype(np.int64) != exp[f].astype(np.int64))[0]
        for r in idx[:5]:
            bad.append(f"{what} read {r} {f}: gpu {got[f][r]} oracle {exp[f][r]}")
    return bad


def _random_candidates(seed, n_reads, sizes, support_hi):
    rng = np.random.default_rng(seed)
    counts = rng.choice(sizes, n_reads)
    first = np.zeros(n_reads + 1, np.uint32)
    first[1:] = np.cumsum(counts)
    support = rng.integers(0, support_hi, int(first[-1]), dtype=np.uint64).astype(np.uint32)
    return first, support


@pytest.mark.parametrize("ceiling", [1, 5, 30, 64])
def test_effort_limit_matches_the_oracle(sa, ceiling):
    import torch
    g = workloads.genome(seed=5, length=2_000_000)
    sizes = [0, 1, 2, 7, 31, 32, 33, 40, 64, 65, 100, 300]
    for seed, hi in ((1, 4), (2, 1 << 32)):            # many ties / full 32-bit supports
        first, support = _random_candidates(seed + ceiling, 240, sizes, hi)
        n_jobs = int(first[-1])
        jobs = np.zeros(n_jobs, sa.JOB_DTYPE)
        jobs["read_len"] = 100
        jobs["ref_pos"] = np.arange(n_jobs)                # tags to check the gather
        jobs["win_len"] = 200
        exp_kept, exp_first = S.effort_limit(support.astype(np.int64), first.astype(np.int64), ceiling)
        with sa.Reference(g[:10_000]) as ref:
            kept, kept_from, kept_first = ref.effort_limit(jobs, support, first, ceiling)
            assert (kept_from.astype(np.int64) == exp_kept).all()
            assert (kept_first.astype(np.int64) == exp_first).all()
            assert (kept["ref_pos"] == jobs["ref_pos"][kept_from]).all()
            # device form
            dev = torch.device("cuda", 0)
            dj = torch.from_numpy(jobs.view(np.uint8)).to(dev)
            ds = torch.from_numpy(support.view(np.int32)).to(dev)
            df = torch.from_numpy(first.view(np.int32)).to(dev)
            dk = torch.empty(max(1, n_jobs) * 32, dtype=torch.uint8, device=dev)
            dfrom = torch.empty(max(1, n_jobs), dtype=torch.int32, device=dev)
            dkf = torch.empty(len(first), dtype=torch.int32, device=dev)
            n = ref.effort_limit_dev(dj, ds, df, ceiling, dk, dfrom, dkf)
            assert n == len(exp_kept)
            assert (dfrom.cpu().numpy()[:n].astype(np.int64) == exp_kept).all()
            assert (dkf.cpu().numpy().astype(np.int64) == exp_first).all()


def test_effort_limit_on_a_read_with_thousands_of_candidates(sa):
    """One read with 6,000 candidates (the poly-A case of the paper): exactly
    `ceiling` kept, every kept one ranked above every dropped one."""
    rng = np.random.default_rng(9)
    n = 6000
    support = rng.integers(0, 50, n).astype(np.uint32)
    first = np.array([0, n], np.uint32)
    jobs = np.zeros(n, sa.JOB_DTYPE)
    jobs["read_len"], jobs["win_len"] = 100, 200
    with sa.Reference(workloads.genome(seed=5, length=2_000_000)[:10_000]) as ref:
        _, kept_from, kept_first = ref.effort_limit(jobs, support, first, 30)
    assert kept_first.tolist() == [0, 30]
    k = kept_from.astype(np.int64)
    assert (np.diff(k) > 0).all()
    dropped = np.setdiff1d(np.arange(n), k)
    worst_kept = min((int(support[i]), -int(i)) for i in k)
    best_dropped = max((int(support[i]), -int(i)) for i in dropped)
    assert worst_kept > best_dropped


def _oracle_flow(w, ceiling, kw, align_kw):
    kept, kf = S.effort_limit(w.support.astype(np.int64), w.read_first.astype(np.int64), ceiling)
    sub = w.subset(kept)
    res, _ = oracle.align(sub, **align_kw)
    return kept, kf, S.select(sub.flags, sub.read_len, res, kf, **kw)


def _gpu_flow(sa, ref, w, ceiling, params, sel):
    import torch
    dev = torch.device("cuda", 0)
    jobs = sa.jobs_array(w.read_off, w.read_len, w.flags, w.ref_pos, w.win_len)
    n_jobs = len(jobs)
    dj = torch.from_numpy(jobs.view(np.uint8)).to(dev)
    ds = torch.from_numpy(w.support.view(np.int32)).to(dev)
    df = torch.from_numpy(w.read_first.astype(np.uint32).view(np.int32)).to(dev)
    dr = torch.from_numpy(w.reads).to(dev)
    dk = torch.empty(n_jobs * 32, dtype=torch.uint8, device=dev)
    dfrom = torch.empty(n_jobs, dtype=torch.int32, device=dev)
    dkf = torch.empty(w.n_reads + 1, dtype=torch.int32, device=dev)
    n = ref.effort_limit_dev(dj, ds, df, ceiling, dk, dfrom, dkf)
    kept = dk[: n * 32]
    dres = torch.empty(n * 56, dtype=torch.uint8, device=dev)
    kept_np = kept.cpu().numpy().view(sa.JOB_DTYPE)
    dcig = torch.empty(max(1, sa.cigar_max_ops(kept_np["read_len"])), dtype=torch.int32, device=dev)
    ref.align_dev(kept, dr, dres, dcig, params)
    dout = torch.empty(w.n_reads * 32, dtype=torch.uint8, device=dev)
    ref.select_dev(kept, dres, dkf, dout, sel)
    torch.cuda.synchronize()
    return (dfrom.cpu().numpy()[:n].astype(np.int64), dkf.cpu().numpy().astype(np.int64),
            dout.cpu().numpy().view(sa.READ_RESULT_DTYPE))


@pytest.mark.parametrize("paired", [False, True])
def test_pairs_workload_matches_the_oracle(sa, paired):
    w = workloads.pairs(seed=4, n_pairs=1500, genome_len=2_000_000, dup=0.3)
    kw = dict(match=1, mismatch=2, paired=paired, frag_min=300, frag_max=700)
    exp_kept, exp_first, exp = _oracle_flow(w, 30, kw, {})
    with sa.Reference(w.ref) as ref:
        kept, first, got = _gpu_flow(sa, ref, w, 30, sa.make_params(),
                                     sa.make_select_params(paired=paired, frag_min=300, frag_max=700))
    assert (kept == exp_kept).all() and (first == exp_first).all()
    bad = _diff(got, exp, "pairs")
    assert not bad, "\n".join(bad)
    if paired:
        assert (got["flags"] & sa.SA_READ_PROPER).mean() > 0.9
        assert (got["mapq"] == 0).any() and (got["mapq"] == 60).any()


@pytest.mark.parametrize("case", ["no_cigar", "ff", "below_min", "glocal", "no_limit"])
def test_selection_variants_match_the_oracle(sa, case):
    w = workloads.pairs(seed=6, n_pairs=400, genome_len=2_000_000, dup=0.4, decoy_max=12)
    params = dict(scoring=(1, 2, 2, 1))
    align_kw = {}
    kw = dict(match=1, mismatch=2, paired=True, frag_min=300, frag_max=700)
    ceiling = 30
    if case == "no_cigar":
        params["want_cigar"] = False
        align_kw["want_cigar"] = False
    elif case == "ff":
        kw["orientation"] = S.PAIR_FF
    elif case == "below_min":
        params["min_score"] = 140
        align_kw["min_score"] = 140
    elif case == "glocal":
        params["mode"] = sa.SA_GLOCAL
        align_kw["mode"] = oracle.GLOCAL
    elif case == "no_limit":
        ceiling = 1000
    exp_kept, exp_first, exp = _oracle_flow(w, ceiling, kw, align_kw)
    sel = sa.make_select_params(paired=True, orientation=kw.get("orientation", 0), frag_min=300, frag_max=700)
    with sa.Reference(w.ref) as ref:
        kept, first, got = _gpu_flow(sa, ref, w, ceiling, sa.make_params(**params), sel)
    assert (kept == exp_kept).all() and (first == exp_first).all()
    bad = _diff(got, exp, case)
    assert not bad, "\n".join(bad)


def test_host_select_and_wide_pairs(sa):
    """sa_select with host buffers on pairs of 150 x 150 candidates (no limit),
    plus reads without candidates."""
    w = workloads.pairs(seed=8, n_pairs=7, genome_len=2_000_000, decoy_max=61)
    # widen: every read gets its own candidates repeated (shifted windows)
    idx = np.concatenate([np.repeat(np.arange(int(w.read_first[r]), int(w.read_first[r + 1])), 3)
                          for r in range(w.n_reads)])
    first = np.zeros(w.n_reads + 1, np.int64)
    first[1:] = np.cumsum(3 * np.diff(w.read_first.astype(np.int64)))
    # the last pair has no candidates at all
    cut = int(first[-3])
    idx, first = idx[:cut], np.minimum(first, cut)
    sub = w.subset(idx)
    shifted = sub.ref_pos.astype(np.int64) + np.arange(len(idx)) % 3
    sub.ref_pos = np.minimum(shifted, len(w.ref) - sub.win_len.astype(np.int64)).astype(np.uint64)
    res, _ = oracle.align(sub)
    exp = S.select(sub.flags, sub.read_len, res, first, paired=True, frag_min=300, frag_max=700)
    with sa.Reference(w.ref) as ref:
        jobs = sa.jobs_array(sub.read_off, sub.read_len, sub.flags, sub.ref_pos, sub.win_len)
        gres, _ = ref.align(jobs, sub.reads)
        got = ref.select(jobs, gres, first.astype(np.uint32),
                         sa.make_select_params(paired=True, frag_min=300, frag_max=700))
    assert max(np.diff(first)) >= 150
    bad = _diff(got, exp, "wide")
    assert not bad, "\n".join(bad)
    assert got["job"][-1] == sa.SA_NO_JOB and got["flags"][-1] == sa.SA_READ_PAIRED


def test_argument_errors(sa):
    with sa.Reference(workloads.genome(seed=5, length=2_000_000)[:10_000]) as ref:
        jobs = np.zeros(3, sa.JOB_DTYPE)
        res = np.zeros(3, sa.RESULT_DTYPE)
        for first, params in (([0, 1, 2, 3], sa.make_select_params(paired=True)),     # odd read count
                              ([0, 2, 1, 3], sa.make_select_params()),                # not ascending
                              ([1, 2, 3], sa.make_select_params()),                   # not from 0
                              ([0, 1, 3], sa.make_select_params(paired=True, frag_min=5, frag_max=4))):
            with pytest.raises(sa.SAError) as e:
                ref.select(jobs, res, np.array(first, np.uint32), params)
            assert e.value.code == sa.SA_EINVAL
        with pytest.raises(sa.SAError) as e:
            ref.effort_limit(jobs, np.zeros(3, np.uint32), np.array([0, 3], np.uint32), 0)
        assert e.value.code == sa.SA_EINVAL
        out = ref.select(jobs[:0], res[:0], np.array([0], np.uint32))
        assert len(out) == 0
