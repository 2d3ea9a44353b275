"""The allocation-free entry point, sa_align_batch_noalloc.

It is for callers that cannot let a library allocate device memory (a host
framework that owns all device memory through its own allocator, or a
latency-sensitive caller that cannot afford cudaMalloc's synchronisation).
Its results must equal those of sa_align_batch_dev with want_cigar = 0, row
for row and bit for bit (the tolerance of every parity test here), on two
calls in a row: the second call reuses the shared scratch the first one left
behind, with a different batch size, read lengths and mode.

This file is named so that pytest collects it last; it also passes alone.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_matches_device_entry_point_on_two_calls():
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_1302_5507_gb300 as sa
    import workloads

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
