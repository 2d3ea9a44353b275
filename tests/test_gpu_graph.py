"""The score segment (order, packing, score passes, overflow rerun) is captured as
a CUDA graph the second time a call's launches are the same and replayed while
they stay so; replayed calls must give the oracle's results, and any change of
the launches drops the graph (a one-off shape runs its launches directly)."""
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


def _dev_call(sa, ref, d, params):
    import torch
    jobs_t, reads_t, out_t, cig_t, n = d
    used = ref.align_dev(jobs_t, reads_t, out_t, cig_t, params)
    torch.cuda.synchronize()
    res = out_t.cpu().numpy().view(sa.RESULT_DTYPE)[:n].copy()
    cig = cig_t.cpu().numpy().view(np.uint32)[:used].copy() if cig_t is not None else None
    return res, cig


def test_replayed_segment_matches_the_oracle(sa):
    import torch
    wl = workloads.uneven(seed=11, n_jobs=3_000)
    other = workloads.uneven(seed=11, n_jobs=2_000, first_item=3_000)
    ores, oops = oracle.align(wl)
    dev = torch.device("cuda", 0)

    def put(w):
        jobs = sa.jobs_array(w.read_off, w.read_len, w.flags, w.ref_pos, w.win_len)
        return (torch.from_numpy(jobs.view(np.uint8)).to(dev), torch.from_numpy(w.reads).to(dev),
                torch.empty(len(jobs) * 56, dtype=torch.uint8, device=dev),
                torch.empty(sa.cigar_max_ops(w.read_len), dtype=torch.int32, device=dev), w.n_jobs)

    with sa.Reference(wl.ref) as ref:
        d = put(wl)
        replays = []
        for width in (0, 0, 0, 32, 32, 32, 0, 0, 0):
            res, cig = _dev_call(sa, ref, d, sa.make_params(width=width))
            replays.append(ref.stats()["graph_replays"])
            bad = compare(res, cig, ores, oops)
            assert not bad, "\n".join(bad[:10])
        # first sight runs directly, the second captures, later identical calls
        # replay; a width change starts over
        assert replays == [0, 0, 1, 0, 0, 1, 0, 0, 1]
        # another batch (other sizes) runs directly and is exact too
        res, cig = _dev_call(sa, ref, put(other), sa.make_params())
        assert ref.stats()["graph_replays"] == 0
        o2, p2 = oracle.align(other)
        assert not compare(res, cig, o2, p2)
