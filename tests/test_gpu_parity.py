"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle,
field by field and bit-exact (score, ends, begins, second best and its end,
flags, CIGAR), on seeded synthetic inputs."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads
from oracle.compare import compare

pytestmark = pytest.mark.gpu

SCHEMES = [(1, 2, 2, 1), (1, 4, 6, 1), (2, 3, 5, 2), (1, 3, 1, 0), (3, 1, 0, 1), (1, 10, 0, 1)]


@pytest.fixture(scope="module")
def sa():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1302_5507_gb300 as sa
    return sa


def run_pair(sa, ref, wl, *, scoring=(1, 2, 2, 1), mode=0, form=0, width=0, want_cigar=True,
             min_score=oracle.NO_SCORE, arena_mb=0):
    jobs = sa.jobs_array(wl.read_off, wl.read_len, wl.flags, wl.ref_pos, wl.win_len)
    p = sa.make_params(scoring=scoring, mode=mode, form=form, width=width, want_cigar=want_cigar,
                       min_score=min_score, arena_mb=arena_mb)
    res, cig = ref.align(jobs, wl.reads, p)
    ores, oops = oracle.align(wl, scoring=scoring, mode=mode, want_cigar=want_cigar,
                              min_score=min_score)
    return res, cig, ores, oops


def assert_parity(sa, ref, wl, **kw):
    res, cig, ores, oops = run_pair(sa, ref, wl, **kw)
    bad = compare(res, cig, ores, oops if kw.get("want_cigar", True) else None)
    assert not bad, f"{wl.name} {kw}: " + "\n".join(bad)
    return res, ores


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("scoring", SCHEMES)
def test_small_random(sa, mode, form, scoring):
    for seed, alpha in ((1, 4), (2, 2)):
        wl = workloads.small(seed * 100 + sum(scoring), 1500, n_range=(1, 70), m_range=(1, 160),
                             alphabet=alpha)
        with sa.Reference(wl.ref) as ref:
            assert_parity(sa, ref, wl, scoring=scoring, mode=mode, form=form)


@pytest.mark.parametrize("mode", [0, 1])
def test_long_reads_wide_groups(sa, mode):
    """Reads of 257..1024 bases use the 32-lane configurations."""
    wl = workloads.small(5, 60, n_range=(200, 1024), m_range=(1, 2500))
    with sa.Reference(wl.ref) as ref:
        assert_parity(sa, ref, wl, mode=mode)
        assert_parity(sa, ref, wl, mode=mode, form=1)


@pytest.mark.parametrize("mode", [0, 1])
def test_plain_workload_full(sa, mode):
    """10,000 jobs of 100 bp reads in 400 bp windows (every job)."""
    wl = workloads.plain(seed=1)
    with sa.Reference(wl.ref) as ref:
        assert_parity(sa, ref, wl, mode=mode)
        assert_parity(sa, ref, wl, mode=mode, form=1)


def test_mate_rescue_subset(sa):
    wl = workloads.mate_rescue(seed=1, n_pairs=20_000)
    with sa.Reference(wl.ref) as ref:
        res, ores = assert_parity(sa, ref, wl)
        assert_parity(sa, ref, wl, mode=1)
    # mates come from the window: most align (almost) end to end
    assert np.median(res["score"]) >= 140


def test_uneven_subset(sa):
    wl = workloads.uneven(seed=1, n_jobs=20_000)
    with sa.Reference(wl.ref) as ref:
        assert_parity(sa, ref, wl)
        assert_parity(sa, ref, wl, form=1)


def test_low_similarity_subset(sa):
    wl = workloads.lowsim(seed=1, n_jobs=3_000)
    with sa.Reference(wl.ref) as ref:
        assert_parity(sa, ref, wl)
        assert_parity(sa, ref, wl, want_cigar=False)
        assert_parity(sa, ref, wl, mode=1)


def _wl_from_pairs(pairs, flags=None):
    ref = "".join(w for w, _ in pairs)
    reads = "".join(r for _, r in pairs)
    n = np.array([len(r) for _, r in pairs], np.uint32)
    m = np.array([len(w) for w, _ in pairs], np.uint32)
    off = np.concatenate([[0], np.cumsum(n[:-1])]).astype(np.uint64)
    pos = np.concatenate([[0], np.cumsum(m[:-1])]).astype(np.uint64)
    fl = np.zeros(len(pairs), np.uint32) if flags is None else np.asarray(flags, np.uint32)
    return workloads.Workload("edge", np.frombuffer(ref.encode(), np.uint8).copy(),
                              np.frombuffer(reads.encode(), np.uint8).copy(), off, n, fl, pos, m,
                              pos.copy())


def test_edge_cases(sa):
    pairs = [("A", "A"), ("C", "A"), ("ACGT", "ACGTACGT"), ("AAAAAAAAAA", "AAA"), ("CCCCCCCC", "AAAA"),
             ("ACGTTTACGT", "ACGTACGT"), ("AC", "AAC"), ("ACGT", "AGT"), ("T" * 300, "T" * 256),
             ("ACGT" * 50, "TGCA" * 10), ("G", "GGGGGGGGGGGGGGGGGGGGGGGGGGGGGGGGGG")]
    wl = _wl_from_pairs(pairs, flags=[0, 1] * 5 + [0])
    with sa.Reference(wl.ref) as ref:
        for mode in (0, 1):
            for form in (0, 1):
                for scoring in SCHEMES:
                    assert_parity(sa, ref, wl, mode=mode, form=form, scoring=scoring)


def test_maximum_sizes(sa):
    """The largest read (SA_MAX_READ) against the largest window (SA_MAX_WINDOW), and
    the degenerate extremes around them, in both modes and forms."""
    rng = np.random.default_rng(17)
    bases = np.frombuffer(b"ACGT", np.uint8)
    win = bases[rng.integers(0, 4, sa.SA_MAX_WINDOW)].tobytes().decode()
    read = win[30000:30000 + sa.SA_MAX_READ]
    noisy = "".join(c if rng.random() > 0.05 else "ACGT"[rng.integers(0, 4)] for c in read)
    pairs = [(win, noisy), (win, "A"), ("C", noisy), (win[:sa.SA_MAX_READ], noisy)]
    wl = _wl_from_pairs(pairs, flags=[0, 1, 0, 1])
    with sa.Reference(wl.ref) as ref:
        for mode in (0, 1):
            for form in (0, 1):
                assert_parity(sa, ref, wl, mode=mode, form=form)


def test_min_score_and_score_only(sa):
    wl = workloads.small(9, 800, n_range=(5, 60), m_range=(5, 120))
    with sa.Reference(wl.ref) as ref:
        for mode in (0, 1):
            assert_parity(sa, ref, wl, mode=mode, min_score=20)
            assert_parity(sa, ref, wl, mode=mode, want_cigar=False)


def test_invalid_inputs(sa):
    wl = workloads.small(3, 10, n_range=(5, 20), m_range=(30, 60))
    jobs = sa.jobs_array(wl.read_off, wl.read_len, wl.flags, wl.ref_pos, wl.win_len)
    with sa.Reference(wl.ref) as ref:
        bad_reads = wl.reads.copy()
        bad_reads[3] = ord("N")
        with pytest.raises(sa.SAError) as e:
            ref.align(jobs, bad_reads)
        assert e.value.code == sa.SA_EINVAL
        past = jobs.copy()
        past["ref_pos"][2] = len(wl.ref) - 5
        with pytest.raises(sa.SAError) as e:
            ref.align(past, wl.reads)
        assert e.value.code == sa.SA_EINVAL
        zero = jobs.copy()
        zero["read_len"][0] = 0
        with pytest.raises(sa.SAError):
            ref.align(zero, wl.reads)
        long_ = jobs.copy()
        long_["read_len"][0] = sa.SA_MAX_READ + 1
        with pytest.raises(sa.SAError):
            ref.align(long_, wl.reads)
        # a match score above 2047 (a LOCAL best past 21 bits) is refused
        with pytest.raises(sa.SAError) as e:
            ref.align(jobs, wl.reads, sa.make_params(scoring=(2048, 1, 1, 1)))
        assert e.value.code == sa.SA_EINVAL
        # an empty batch is fine
        out, cig = ref.align(jobs[:0], wl.reads)
        assert len(out) == 0 and len(cig) == 0
        # a too-small CIGAR buffer reports the size it needs
        with pytest.raises(sa.SAError) as e:
            ref.align(jobs, wl.reads, cigar=np.zeros(1, np.uint32))
        assert e.value.code == sa.SA_EOVERFLOW
        # and the reference itself is validated
        with pytest.raises(sa.SAError):
            sa.Reference(b"ACGTNACGT")
        # after the errors the same reference still computes correctly
        assert_parity(sa, ref, wl)


def test_device_buffers_match_host_buffers(sa):
    import torch
    wl = workloads.mate_rescue(seed=2, n_pairs=5_000)
    jobs = sa.jobs_array(wl.read_off, wl.read_len, wl.flags, wl.ref_pos, wl.win_len)
    with sa.Reference(wl.ref) as ref:
        h_res, h_cig = ref.align(jobs, wl.reads)
        dev = torch.device("cuda:0")
        d_jobs = torch.from_numpy(jobs.view(np.uint8)).to(dev)
        d_reads = torch.from_numpy(wl.reads).to(dev)
        d_out = torch.zeros(len(jobs) * 56, dtype=torch.uint8, device=dev)
        cap = sa.cigar_max_ops(wl.read_len)
        d_cig = torch.zeros(cap, dtype=torch.int32, device=dev)
        stream = torch.cuda.Stream()
        used = ref.align_dev(d_jobs, d_reads, d_out, d_cig, stream=stream)
        torch.cuda.synchronize()
        res = d_out.cpu().numpy().view(sa.RESULT_DTYPE)
        cig = d_cig[:used].cpu().numpy().view(np.uint32)
        assert (res == h_res).all()
        assert np.array_equal(cig, h_cig)


def test_full_size_mate_rescue_sampled(sa):
    """The benchmark's workload (1M mate-rescue jobs) in one call; a seeded sample
    of jobs is recomputed by the oracle one by one."""
    wl = workloads.mate_rescue(seed=1)
    jobs = sa.jobs_array(wl.read_off, wl.read_len, wl.flags, wl.ref_pos, wl.win_len)
    with sa.Reference(wl.ref) as ref:
        res, cig = ref.align(jobs, wl.reads)
    rng = np.random.default_rng(123)
    idx = np.sort(rng.choice(wl.n_jobs, 3000, replace=False))
    sub = wl.subset(idx)
    ores, oops = oracle.align(sub)
    sres = res[idx].copy()
    # re-base the CIGAR offsets of the sample onto a compacted copy
    parts, off = [], 0
    for k, j in enumerate(idx):
        L = int(res["cigar_len"][j])
        parts.append(cig[int(res["cigar_off"][j]):int(res["cigar_off"][j]) + L])
        sres["cigar_off"][k] = off
        off += L
    scig = np.concatenate(parts) if parts else np.zeros(0, np.uint32)
    bad = compare(sres, scig, ores, oops)
    assert not bad, "\n".join(bad)
    # the CIGAR buffer is compact and in job order
    assert (np.diff(res["cigar_off"].astype(np.int64)) == res["cigar_len"][:-1]).all()


def _sampled_compare(wl, res, cig, idx):
    sub = wl.subset(idx)
    ores, oops = oracle.align(sub)
    sres = res[idx].copy()
    parts, off = [], 0
    for k, j in enumerate(idx):
        L = int(res["cigar_len"][j])
        parts.append(cig[int(res["cigar_off"][j]):int(res["cigar_off"][j]) + L])
        sres["cigar_off"][k] = off
        off += L
    scig = np.concatenate(parts) if parts else np.zeros(0, np.uint32)
    return compare(sres, scig, ores, oops)


def test_full_size_uneven_sampled(sa):
    """The uneven-length workload at its full size (4M jobs, every length bucket,
    16-bit pairs) in one device call, as the benchmark runs it; a seeded sample of
    jobs is recomputed by the oracle one by one."""
    import torch
    wl = workloads.uneven(seed=1)
    jobs = sa.jobs_array(wl.read_off, wl.read_len, wl.flags, wl.ref_pos, wl.win_len)
    dev = torch.device("cuda", 0)
    with sa.Reference(wl.ref) as ref:
        d_out = torch.empty(len(jobs) * 56, dtype=torch.uint8, device=dev)
        d_cig = torch.empty(sa.cigar_max_ops(wl.read_len), dtype=torch.int32, device=dev)
        used = ref.align_dev(torch.from_numpy(jobs.view(np.uint8)).to(dev), torch.from_numpy(wl.reads).to(dev),
                             d_out, d_cig, sa.make_params())
        torch.cuda.synchronize()
        assert ref.stats()["jobs16"] == wl.n_jobs
        res = d_out.cpu().numpy().view(sa.RESULT_DTYPE)
        cig = d_cig[:used].cpu().numpy().view(np.uint32)
    rng = np.random.default_rng(321)
    idx = np.sort(rng.choice(wl.n_jobs, 3000, replace=False))
    bad = _sampled_compare(wl, res, cig, idx)
    assert not bad, "\n".join(bad)


def test_full_size_low_similarity_sampled(sa):
    """The low-similarity workload at its full size (500k jobs of 250 bp against
    1,000 bp windows, divergence 0-40 %) in one device call, with and without a
    traceback (most jobs take the wavefront rectangle pass); a seeded sample of
    jobs is recomputed by the oracle one by one."""
    import torch
    wl = workloads.lowsim(seed=1)
    jobs = sa.jobs_array(wl.read_off, wl.read_len, wl.flags, wl.ref_pos, wl.win_len)
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(555)
    idx = np.sort(rng.choice(wl.n_jobs, 3000, replace=False))
    with sa.Reference(wl.ref) as ref:
        d_jobs = torch.from_numpy(jobs.view(np.uint8)).to(dev)
        d_reads = torch.from_numpy(wl.reads).to(dev)
        d_out = torch.empty(len(jobs) * 56, dtype=torch.uint8, device=dev)
        d_cig = torch.empty(sa.cigar_max_ops(wl.read_len), dtype=torch.int32, device=dev)
        used = ref.align_dev(d_jobs, d_reads, d_out, d_cig, sa.make_params())
        torch.cuda.synchronize()
        st = ref.stats()
        assert st["rect_jobs"] > wl.n_jobs // 2 and st["band_jobs"] > 0 and st["diag_jobs"] > 0, st
        res = d_out.cpu().numpy().view(sa.RESULT_DTYPE).copy()
        cig = d_cig[:used].cpu().numpy().view(np.uint32).copy()
        ref.align_dev(d_jobs, d_reads, d_out, None, sa.make_params(want_cigar=False))
        torch.cuda.synchronize()
        res_score = d_out.cpu().numpy().view(sa.RESULT_DTYPE).copy()
    bad = _sampled_compare(wl, res, cig, idx)
    assert not bad, "\n".join(bad)
    ores, _ = oracle.align(wl.subset(idx), want_cigar=False)
    bad = compare(res_score[idx], None, ores, None)
    assert not bad, "\n".join(bad)


def test_direction_arena_in_waves(sa):
    """A direction arena capped far below the batch's rectangles (arena_mb) makes
    the rectangle direction pass and its walks run in several waves; the results
    stay identical to the oracle's, and to the single-wave run."""
    wl = workloads.lowsim(seed=4, n_jobs=3_000)
    with sa.Reference(wl.ref) as ref:
        jobs = sa.jobs_array(wl.read_off, wl.read_len, wl.flags, wl.ref_pos, wl.win_len)
        one, one_cig = ref.align(jobs, wl.reads)
        assert ref.stats()["waves"] == 1
        for mode in (0, 1):
            res, ores = assert_parity(sa, ref, wl, mode=mode, arena_mb=16)
            st = ref.stats()
            assert st["waves"] >= (3 if mode == 0 else 2) and st["rect_jobs"] > 500, st
        res, cig = ref.align(jobs, wl.reads, sa.make_params(arena_mb=16))
        assert (res == one).all() and np.array_equal(cig, one_cig)


def test_full_size_pairs_sampled(sa):
    """The paired multi-candidate workload at the benchmark's size (100k pairs,
    4.25M candidates): effort limit, alignment and paired selection on the device;
    a seeded sample of pairs is recomputed by the oracle from their own candidates
    (every step is per read or per pair)."""
    import torch
    from oracle import select as S
    w = workloads.pairs(seed=1, n_pairs=100_000)
    jobs = sa.jobs_array(w.read_off, w.read_len, w.flags, w.ref_pos, w.win_len)
    dev = torch.device("cuda", 0)
    first = w.read_first.astype(np.uint32)
    with sa.Reference(w.ref) as ref:
        dk = torch.empty(len(jobs) * 32, dtype=torch.uint8, device=dev)
        dfrom = torch.empty(len(jobs), dtype=torch.int32, device=dev)
        dkf = torch.empty(len(first), dtype=torch.int32, device=dev)
        n = ref.effort_limit_dev(torch.from_numpy(jobs.view(np.uint8)).to(dev),
                                 torch.from_numpy(w.support.view(np.int32)).to(dev),
                                 torch.from_numpy(first.view(np.int32)).to(dev), 30, dk, dfrom, dkf)
        dres = torch.empty(n * 56, dtype=torch.uint8, device=dev)
        dcig = torch.empty(sa.cigar_max_ops(w.read_len), dtype=torch.int32, device=dev)
        ref.align_dev(dk[: n * 32], torch.from_numpy(w.reads).to(dev), dres, dcig, sa.make_params())
        dout = torch.empty(w.n_reads * 32, dtype=torch.uint8, device=dev)
        ref.select_dev(dk[: n * 32], dres, dkf, dout,
                       sa.make_select_params(paired=True, frag_min=300, frag_max=700))
        torch.cuda.synchronize()
        kept_from = dfrom.cpu().numpy()[:n].astype(np.int64)
        kept_first = dkf.cpu().numpy().astype(np.int64)
        got = dout.cpu().numpy().view(sa.READ_RESULT_DTYPE)
    rng = np.random.default_rng(99)
    pairs = np.sort(rng.choice(w.n_reads // 2, 400, replace=False))
    reads = np.stack([2 * pairs, 2 * pairs + 1], 1).ravel()
    # the oracle on the sampled reads' own candidates
    cand = np.concatenate([np.arange(int(w.read_first[r]), int(w.read_first[r + 1])) for r in reads])
    sfirst = np.zeros(len(reads) + 1, np.int64)
    sfirst[1:] = np.cumsum([int(w.read_first[r + 1] - w.read_first[r]) for r in reads])
    kept, kf = S.effort_limit(w.support[cand].astype(np.int64), sfirst, 30)
    sub = w.subset(cand[kept])
    ores, _ = oracle.align(sub)
    exp = S.select(sub.flags, sub.read_len, ores, kf, paired=True, frag_min=300, frag_max=700)
    # the device's choices, mapped back to batch candidates, must be the same
    for k, r in enumerate(reads):
        g, e = got[r], exp[k]
        assert (int(kept_first[r + 1]) - int(kept_first[r])) == int(kf[k + 1] - kf[k])
        gj = -1 if g["job"] == sa.SA_NO_JOB else int(kept_from[g["job"]])
        ej = -1 if e["job"] == S.NO_JOB else int(cand[kept[e["job"]]])
        assert gj == ej, (r, gj, ej)
        for f in ("score", "second", "mapq", "flags", "n_cand", "frag_len"):
            assert int(g[f]) == int(e[f]), (r, f, int(g[f]), int(e[f]))


def test_every_direction_pass_class_is_exercised(sa):
    """The low-similarity sweep puts traced jobs in every traceback class: the
    all-match diagonal (no direction pass), the banded passes and the
    whole-rectangle pass; all must match the oracle."""
    wl = workloads.lowsim(seed=2, n_jobs=1_200)
    with sa.Reference(wl.ref) as ref:
        assert_parity(sa, ref, wl)
        st = ref.stats()
        assert st["diag_jobs"] > 0 and st["band_jobs"] > 0 and st["rect_jobs"] > 0, st
        assert_parity(sa, ref, wl, mode=1)


@pytest.mark.parametrize("width", [16, 32])
def test_width_16_and_32_agree_with_oracle(sa, width):
    """The 16-bit packed score pass (two jobs per lane group) and the 32-bit one."""
    wl = workloads.uneven(seed=3, n_jobs=6_000)
    with sa.Reference(wl.ref) as ref:
        assert_parity(sa, ref, wl, width=width)
        assert_parity(sa, ref, wl, width=width, want_cigar=False)
        assert ref.stats()["overflow_reruns"] == 0


def test_overflow_rerun_is_exact(sa):
    """A large-score scheme pushes long reads past the 16-bit range: those jobs are
    flagged and recomputed in 32-bit; every result still equals the oracle."""
    scoring = (200, 150, 300, 40)
    wl = workloads.uneven(seed=5, n_jobs=3_000)
    with sa.Reference(wl.ref) as ref:
        res, ores = assert_parity(sa, ref, wl, scoring=scoring, width=16)
        st = ref.stats()
        assert st["overflow_reruns"] > 0
        # every job whose best reached the threshold (H + o + e >= 1024 - a) was rerun
        assert st["overflow_reruns"] >= int((ores["score"] >= 1024 - 200 - (300 + 40)).sum())
        assert_parity(sa, ref, wl, scoring=scoring, width=16, want_cigar=False)


def test_results_do_not_depend_on_pairing_or_run(sa):
    """The 16-bit pass pairs jobs in an order that varies between runs; every
    run must give the same (oracle-exact) results."""
    wl = workloads.small(106, 1500, n_range=(1, 70), m_range=(1, 160), alphabet=4)
    jobs = sa.jobs_array(wl.read_off, wl.read_len, wl.flags, wl.ref_pos, wl.win_len)
    ores, oops = oracle.align(wl)
    with sa.Reference(wl.ref) as ref:
        first = None
        for _ in range(4):
            res, cig = ref.align(jobs, wl.reads, sa.make_params(width=16))
            bad = compare(res, cig, ores, oops)
            assert not bad, "\n".join(bad)
            if first is None:
                first = (res.copy(), cig.copy())
            assert (res == first[0]).all() and np.array_equal(cig, first[1])


def test_page_locked_host_buffers(sa):
    """sa_align_batch with page-locked host buffers, mixed with pageable ones,
    matches the oracle; a page-locked CIGAR buffer that is too small is refused."""
    import torch
    wl = workloads.small(77, 2000, n_range=(1, 200), m_range=(1, 600), alphabet=4)
    jobs = sa.jobs_array(wl.read_off, wl.read_len, wl.flags, wl.ref_pos, wl.win_len)
    ores, oops = oracle.align(wl)

    def pinned(a):
        t = torch.empty(a.nbytes, dtype=torch.uint8, pin_memory=True)
        v = t.numpy().view(a.dtype)
        v[:] = a
        return t, v

    cap = sa.cigar_max_ops(wl.read_len)
    with sa.Reference(wl.ref) as ref:
        tj, pj = pinned(jobs)
        tr, pr = pinned(wl.reads)
        for out_pinned, cig_pinned in ((True, True), (True, False), (False, True), (False, False)):
            to, out = pinned(np.zeros(len(jobs), sa.RESULT_DTYPE)) if out_pinned else (None, np.zeros(len(jobs), sa.RESULT_DTYPE))
            tc, cig = pinned(np.zeros(cap, np.uint32)) if cig_pinned else (None, np.zeros(cap, np.uint32))
            res, ops = ref.align(pj, pr, sa.make_params(), out=out, cigar=cig)
            bad = compare(res, ops, ores, oops)
            assert not bad, "\n".join([f"out pinned {out_pinned} cigar pinned {cig_pinned}"] + bad[:10])
        tc, small_cig = pinned(np.zeros(8, np.uint32))
        with pytest.raises(sa.SAError) as e:
            ref.align(pj, pr, sa.make_params(), out=np.zeros(len(jobs), sa.RESULT_DTYPE), cigar=small_cig)
        assert e.value.code == sa.SA_EOVERFLOW
