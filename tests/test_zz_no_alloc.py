"""The allocation-free entry point, sa_align_batch_noalloc.

It is for callers that cannot let a library allocate device memory (a host
framework that owns all device memory through its own allocator, or a
latency-sensitive caller that cannot afford cudaMalloc's synchronisation).
Its results must equal those of sa_align_batch_dev with want_cigar = 0, row
for row and bit for bit (the tolerance of every parity test here), on two
calls in a row: the second call reuses the shared scratch the first one left
behind, with a different batch size, read lengths and mode.  They must also
equal the CPU oracle's score-only results field by field, under two scoring
schemes in both modes, including the largest accepted match score on the
longest read; and every input the entry point refuses must come back as
SA_EINVAL with a message, leaving the output untouched.

This file is named so that pytest collects it last; it also passes alone.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads
from oracle.compare import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sa():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1302_5507_gb300 as sa
    return sa


def _noalloc(sa, ref, wl, params):
    """(rc, message, results) of one call on device copies of `wl`'s jobs and
    reads; the output buffer is poisoned first."""
    import torch
    dev = torch.device("cuda:0")
    jobs = sa.jobs_array(wl.read_off, wl.read_len, wl.flags, wl.ref_pos, wl.win_len)
    d_jobs = torch.from_numpy(jobs.view(np.uint8)).to(dev)
    d_reads = torch.from_numpy(np.ascontiguousarray(wl.reads)).to(dev)
    n = len(jobs)
    d_out = torch.full((max(n, 1) * 56,), 0xA5, dtype=torch.uint8, device=dev)
    rc = sa.sa_align_batch_noalloc(ref.h, params, ctypes.c_void_p(d_jobs.data_ptr()), n,
                                   ctypes.c_void_p(d_reads.data_ptr()), d_reads.numel(),
                                   ctypes.c_void_p(d_out.data_ptr()), None)
    msg = sa.sa_last_error()
    torch.cuda.synchronize()
    return rc, msg, d_out.cpu().numpy()[: n * 56].view(sa.RESULT_DTYPE)


def _wl_from_pairs(pairs):
    ref = "".join(w for w, _ in pairs)
    reads = "".join(r for _, r in pairs)
    n = np.array([len(r) for _, r in pairs], np.uint32)
    m = np.array([len(w) for w, _ in pairs], np.uint32)
    off = np.concatenate([[0], np.cumsum(n[:-1])]).astype(np.uint64)
    pos = np.concatenate([[0], np.cumsum(m[:-1])]).astype(np.uint64)
    return workloads.Workload("edge", np.frombuffer(ref.encode(), np.uint8).copy(),
                              np.frombuffer(reads.encode(), np.uint8).copy(), off, n,
                              np.zeros(len(pairs), np.uint32), pos, m, pos.copy())


def _assert_oracle_parity(sa, ref, wl, scoring, mode, min_score=oracle.NO_SCORE):
    rc, msg, got = _noalloc(sa, ref, wl, sa.make_params(scoring=scoring, mode=mode, want_cigar=False,
                                                        min_score=min_score))
    assert rc == sa.SA_OK, msg
    ores, _ = oracle.align(wl, scoring=scoring, mode=mode, want_cigar=False, min_score=min_score)
    bad = compare(got, None, ores, None)
    assert not bad, f"{wl.name} scoring={scoring} mode={mode}: " + "\n".join(bad)
    assert (got["cigar_len"] == 0).all() and (got["read_begin"] == -1).all()
    return got


def test_noalloc_matches_device_entry_point_on_two_calls(sa):
    import torch

    dev = torch.device("cuda:0")
    first = workloads.mate_rescue(seed=4, n_pairs=6000)
    second = workloads.uneven(seed=4, n_jobs=2500)          # same genome, other shapes
    with sa.Reference(first.ref) as ref:
        for wl, mode, min_score in ((first, sa.SA_LOCAL, sa.SA_NO_SCORE),
                                    (second, sa.SA_GLOCAL, -40)):
            jobs = sa.jobs_array(wl.read_off, wl.read_len, wl.flags, wl.ref_pos, wl.win_len)
            d_jobs = torch.from_numpy(jobs.view(np.uint8)).to(dev)
            d_reads = torch.from_numpy(wl.reads).to(dev)
            n = len(jobs)
            params = sa.make_params(mode=mode, want_cigar=False, min_score=min_score)

            # the existing entry point
            d_ref_out = torch.zeros(n * 56, dtype=torch.uint8, device=dev)
            ref.align_dev(d_jobs, d_reads, d_ref_out, None, params)
            torch.cuda.synchronize()
            expected = d_ref_out.cpu().numpy().view(sa.RESULT_DTYPE)

            # the allocation-free one, through the C ABI (output poisoned first)
            d_out = torch.full((n * 56,), 0xA5, dtype=torch.uint8, device=dev)
            rc = sa.sa_align_batch_noalloc(ref.h, params, ctypes.c_void_p(d_jobs.data_ptr()), n,
                                           ctypes.c_void_p(d_reads.data_ptr()), d_reads.numel(),
                                           ctypes.c_void_p(d_out.data_ptr()), None)
            assert rc == sa.SA_OK, sa.sa_last_error()
            torch.cuda.synchronize()
            got = d_out.cpu().numpy().view(sa.RESULT_DTYPE)
            assert got.tobytes() == expected.tobytes()
            assert (got["cigar_len"] == 0).all() and (got["read_begin"] == -1).all()


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("scoring", [(1, 2, 2, 1), (2, 3, 5, 2)])
def test_noalloc_matches_oracle(sa, mode, scoring):
    """Field by field against the oracle: tiny random jobs (ties, m < n, two-letter
    alphabet) and a slice of the mate-rescue workload."""
    small = workloads.small(900 + 10 * mode + scoring[0], 1200, n_range=(1, 70), m_range=(1, 160),
                            alphabet=2)
    with sa.Reference(small.ref) as ref:
        _assert_oracle_parity(sa, ref, small, scoring, mode)
    mate = workloads.mate_rescue(seed=5, n_pairs=3000)
    with sa.Reference(mate.ref) as ref:
        _assert_oracle_parity(sa, ref, mate, scoring, mode)


def test_noalloc_largest_match_score_on_longest_read(sa):
    """match = 2047, the largest accepted, on a 1,024-base exact hit: the best score
    2047 * 1024 is the largest a LOCAL key of the 32-bit pass holds; match = 2048
    is refused instead of returning a wrapped key."""
    rng = np.random.default_rng(11)
    read = "".join(rng.choice(list("ACGT"), 1024))
    window = "".join(rng.choice(list("ACGT"), 300)) + read + "".join(rng.choice(list("ACGT"), 200))
    other = "".join(rng.choice(list("ACGT"), 1500))
    wl = _wl_from_pairs([(window, read), (other, read)])
    scoring = (2047, 16383, 16000, 383)
    with sa.Reference(wl.ref) as ref:
        for mode in (0, 1):
            got = _assert_oracle_parity(sa, ref, wl, scoring, mode)
            assert got["score"][0] == 2047 * 1024
            assert got["read_end"][0] == 1024 and got["ref_end"][0] == 300 + 1024
        rc, msg, got = _noalloc(sa, ref, wl, sa.make_params(scoring=(2048, 2, 2, 1), want_cigar=False))
        assert rc == sa.SA_EINVAL and "match must be <= 2047" in msg
        assert (got.view(np.uint8) == 0xA5).all()          # nothing written


def test_noalloc_refuses_bad_inputs(sa):
    """Batches too large for the fixed scratch (both size checks), a read with a base
    other than A/C/G/T and an out-of-range job are SA_EINVAL with a message."""
    base = workloads.mate_rescue(seed=6, n_pairs=2000)
    with sa.Reference(base.ref) as ref:
        p = sa.make_params(want_cigar=False)
        # 1.2M jobs: the per-job arrays alone exceed the 32 MiB scratch
        n = 1_200_000
        k = np.arange(n) % base.n_jobs
        big = workloads.Workload("big", base.ref, base.reads, base.read_off[k], np.full(n, 8, np.uint32),
                                 base.flags[k], base.ref_pos[k], np.full(n, 16, np.uint32), base.truth[k])
        rc, msg, got = _noalloc(sa, ref, big, p)
        assert rc == sa.SA_EINVAL and "split the batch" in msg, msg
        assert (got.view(np.uint8) == 0xA5).all()
        # 1M jobs of 150 bases: the per-job arrays fit, the packed reads do not
        n = 1_000_000
        k = np.arange(n) % base.n_jobs
        wide = workloads.Workload("wide", base.ref, base.reads, base.read_off[k], base.read_len[k],
                                  base.flags[k], base.ref_pos[k], base.win_len[k], base.truth[k])
        rc, msg, got = _noalloc(sa, ref, wide, p)
        assert rc == sa.SA_EINVAL and "split the batch" in msg, msg
        assert (got.view(np.uint8) == 0xA5).all()
        # a read with an N
        one = base.subset(np.arange(50))
        reads = one.reads.copy()
        reads[int(one.read_off[7]) + 3] = ord("N")
        bad = workloads.Workload("badbase", one.ref, reads, one.read_off, one.read_len, one.flags,
                                 one.ref_pos, one.win_len, one.truth)
        rc, msg, _ = _noalloc(sa, ref, bad, p)
        assert rc == sa.SA_EINVAL and "A, C, G, T" in msg, msg
        # a window past the reference end
        pos = one.ref_pos.copy()
        pos[3] = len(base.ref) - 10
        past = workloads.Workload("past", one.ref, one.reads, one.read_off, one.read_len, one.flags,
                                  pos, one.win_len, one.truth)
        rc, msg, _ = _noalloc(sa, ref, past, p)
        assert rc == sa.SA_EINVAL and "job 3 is invalid" in msg, msg
        # after the refusals the shared scratch still serves a valid batch
        _assert_oracle_parity(sa, ref, one, (1, 2, 2, 1), 0)


def test_noalloc_empty_alignments_below_min_score(sa):
    """LOCAL jobs with no positive cell are SA_RES_EMPTY with score 0; with a
    positive min_score they are also SA_RES_BELOW_MIN, like every low-scoring job."""
    pairs = [("CCCCCCCC", "AAAA"), ("GGGG", "TTTTTTTT"), ("ACGTACGT", "ACGTACGT"), ("ACGTTTACGT", "ACGTACGT"),
             ("AAAA", "ACCA"), ("T", "G")]
    wl = _wl_from_pairs(pairs)
    with sa.Reference(wl.ref) as ref:
        got = _assert_oracle_parity(sa, ref, wl, (1, 2, 2, 1), 0, min_score=5)
    assert got["flags"][0] == sa.SA_RES_EMPTY | sa.SA_RES_BELOW_MIN and got["score"][0] == 0
    assert got["flags"][2] == 0 and got["score"][2] == 8
