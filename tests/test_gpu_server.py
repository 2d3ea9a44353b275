"""Serving loop (sa_server_create / sa_submit / sa_poll) against the oracle.

Requests queued behind a running one are coalesced into one device batch; the
results must still come back per request, exactly as the oracle computes them,
with each request's CIGAR ops and offsets of its own."""
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


def _requests(n_req=12, seed=41):
    wl = workloads.small(seed, 3000, n_range=(1, 150), m_range=(1, 500), alphabet=4)
    rng = np.random.default_rng(seed)
    cuts = np.sort(rng.choice(np.arange(1, wl.n_jobs), n_req - 1, replace=False))
    bounds = np.concatenate([[0], cuts, [wl.n_jobs]])
    return wl, [wl.subset(np.arange(bounds[k], bounds[k + 1])) for k in range(n_req)]


def test_coalesced_requests_match_the_oracle(sa):
    wl, reqs = _requests()
    with sa.Reference(wl.ref) as ref, sa.Server(ref, max_inflight=2) as srv:
        # submit everything before polling so that queued requests share batches
        tickets = [srv.submit(sa.jobs_array(r.read_off, r.read_len, r.flags, r.ref_pos, r.win_len), r.reads)
                   for r in reqs]
        for r, tk in zip(reqs, tickets):
            rc, res, cig = srv.poll(tk, r.n_jobs, sa.cigar_max_ops(r.read_len))
            assert rc == sa.SA_OK
            ores, oops = oracle.align(r)
            bad = compare(res, cig, ores, oops)
            assert not bad, "\n".join(bad)
            # each request's CIGAR buffer is its own, compact, in job order
            assert res["cigar_off"][0] == 0
            assert (np.diff(res["cigar_off"].astype(np.int64)) == res["cigar_len"][:-1]).all()
        st = srv.stats()
        assert st["submitted"] == st["completed"] == len(reqs) and st["failed"] == 0
        assert st["batches"] + st["coalesced"] == len(reqs) and st["coalesced"] > 0
        assert st["jobs"] == wl.n_jobs and 1 <= st["max_queue"] <= len(reqs)


def test_one_bad_request_does_not_fail_its_batch_mates(sa):
    wl, reqs = _requests(n_req=5, seed=43)
    with sa.Reference(wl.ref) as ref, sa.Server(ref, max_inflight=1) as srv:
        arrays = [sa.jobs_array(r.read_off, r.read_len, r.flags, r.ref_pos, r.win_len) for r in reqs]
        bad_reads = reqs[2].reads.copy()
        bad_reads[0] = ord("N")
        tickets = [srv.submit(a, bad_reads if k == 2 else r.reads)
                   for k, (a, r) in enumerate(zip(arrays, reqs))]
        for k, (r, tk) in enumerate(zip(reqs, tickets)):
            if k == 2:
                with pytest.raises(sa.SAError) as e:
                    srv.poll(tk, r.n_jobs, sa.cigar_max_ops(r.read_len))
                assert e.value.code == sa.SA_EINVAL
                continue
            rc, res, cig = srv.poll(tk, r.n_jobs, sa.cigar_max_ops(r.read_len))
            assert rc == sa.SA_OK
            ores, oops = oracle.align(r)
            assert not compare(res, cig, ores, oops)
        st = srv.stats()
        assert st["submitted"] == 5 and st["completed"] == 4 and st["failed"] == 1


def test_poll_states_and_budget(sa):
    wl, reqs = _requests(n_req=2, seed=47)
    r = reqs[0]
    jobs = sa.jobs_array(r.read_off, r.read_len, r.flags, r.ref_pos, r.win_len)
    with sa.Reference(wl.ref) as ref:
        with sa.Server(ref) as srv:
            tk = srv.submit(jobs, r.reads)
            rc, _, _ = srv.poll(tk, r.n_jobs, sa.cigar_max_ops(r.read_len), timeout_ms=0)
            assert rc in (sa.SA_OK, sa.SA_PENDING)
            if rc == sa.SA_PENDING:
                rc, res, cig = srv.poll(tk, r.n_jobs, sa.cigar_max_ops(r.read_len))
                assert rc == sa.SA_OK
            # a ticket is consumed by its successful poll
            with pytest.raises(sa.SAError) as e:
                srv.poll(tk, r.n_jobs, sa.cigar_max_ops(r.read_len))
            assert e.value.code == sa.SA_ENOTFOUND
        # a request larger than the whole device-memory budget is refused at submit
        with sa.Server(ref, hbm_budget=1 << 10) as srv:
            with pytest.raises(sa.SAError) as e:
                srv.submit(jobs, r.reads)
            assert e.value.code == sa.SA_EBUSY


def test_serving_shaped_requests_and_poll_timeout(sa):
    """Requests shaped like the serving configuration (n U[50,250], m U[2n,6n]) on a
    smaller genome match the oracle; a poll with a short timeout on a request that
    is still running returns SA_ETIMEOUT and the ticket stays valid."""
    genome = workloads.genome(seed=5, length=2_000_000)
    reqs = [workloads.serving_request(genome, 5, k, n) for k, n in enumerate((1, 37, 400, 2500))]
    big = workloads.serving_request(genome, 5, 9, 60_000)
    with sa.Reference(genome) as ref, sa.Server(ref, max_inflight=1) as srv:
        tk_big = srv.submit(sa.jobs_array(big.read_off, big.read_len, big.flags, big.ref_pos, big.win_len),
                            big.reads)
        rc, _, _ = srv.poll(tk_big, big.n_jobs, sa.cigar_max_ops(big.read_len), timeout_ms=1)
        assert rc in (sa.SA_ETIMEOUT, sa.SA_OK)
        if rc == sa.SA_ETIMEOUT:
            rc, res, cig = srv.poll(tk_big, big.n_jobs, sa.cigar_max_ops(big.read_len))
            assert rc == sa.SA_OK
        tickets = [srv.submit(sa.jobs_array(r.read_off, r.read_len, r.flags, r.ref_pos, r.win_len), r.reads)
                   for r in reqs]
        for r, tk in zip(reqs, tickets):
            rc, res, cig = srv.poll(tk, r.n_jobs, sa.cigar_max_ops(r.read_len))
            assert rc == sa.SA_OK
            ores, oops = oracle.align(r)
            bad = compare(res, cig, ores, oops)
            assert not bad, "\n".join(bad[:10])


def test_full_size_serving_reference(sa):
    """The serving configuration's own reference: 3.1 Gbp, 2-bit packed and
    device-resident (775 MB), so window starts pass 2^31 and the packed word
    index passes 2^27.  Serving-shaped requests (n U[50,250], m U[2n,6n]) run
    through sa_align_batch as one batch and through a server as separate
    requests; every job of both is compared with the oracle."""
    genome = workloads.serving_reference(seed=1)
    reqs = [workloads.serving_request(genome, 3, k, n) for k, n in enumerate((2500, 1, 1800, 2700))]
    allj = workloads.Workload(
        "serving", genome, np.concatenate([r.reads for r in reqs]),
        np.concatenate([r.read_off + np.uint64(o) for r, o in
                        zip(reqs, np.cumsum([0] + [r.reads.size for r in reqs[:-1]]))]),
        np.concatenate([r.read_len for r in reqs]), np.concatenate([r.flags for r in reqs]),
        np.concatenate([r.ref_pos for r in reqs]), np.concatenate([r.win_len for r in reqs]),
        np.concatenate([r.truth for r in reqs]))
    assert (allj.ref_pos.astype(np.int64) >= 2 ** 31).sum() > 1000
    assert int(allj.ref_pos.max()) + int(allj.win_len.max()) > 3_000_000_000
    ores, oops = oracle.align(allj)
    with sa.Reference(genome) as ref:
        assert len(ref) == 3_100_000_000
        res, cig = ref.align(sa.jobs_array(allj.read_off, allj.read_len, allj.flags, allj.ref_pos,
                                           allj.win_len), allj.reads)
        bad = compare(res, cig, ores, oops)
        assert not bad, "\n".join(bad[:10])
        with sa.Server(ref, max_inflight=2) as srv:
            tickets = [srv.submit(sa.jobs_array(r.read_off, r.read_len, r.flags, r.ref_pos, r.win_len),
                                  r.reads) for r in reqs]
            first = 0
            for r, tk in zip(reqs, tickets):
                rc, res, cig = srv.poll(tk, r.n_jobs, sa.cigar_max_ops(r.read_len))
                assert rc == sa.SA_OK
                sl = slice(first, first + r.n_jobs)
                bad = compare(res, cig, ores[sl], oops[sl])
                assert not bad, "\n".join(bad[:10])
                first += r.n_jobs


def test_admission_follows_device_memory(sa):
    """Admission re-reads the device's free memory: with almost all of it taken
    by another allocation of the process after the server started, a request
    waits instead of failing; once the memory is released it runs and its
    results match the oracle."""
    import torch
    genome = workloads.genome(seed=6, length=2_000_000)
    # 20,000 serving-shaped jobs: an estimate of several GB (the rectangle arena is
    # charged at its largest), far above what is left free below
    r = workloads.serving_request(genome, 6, 0, 20_000)
    jobs = sa.jobs_array(r.read_off, r.read_len, r.flags, r.ref_pos, r.win_len)
    with sa.Reference(genome) as ref, sa.Server(ref, max_inflight=1) as srv:
        torch.cuda.synchronize()
        hog = []
        free, _ = torch.cuda.mem_get_info()
        chunk = 1 << 30
        while free > (256 << 20) and chunk >= (8 << 20):     # leave less than 256 MB free
            try:
                hog.append(torch.empty(min(chunk, free - (128 << 20)), dtype=torch.uint8, device="cuda"))
            except RuntimeError:
                chunk //= 2
            free, _ = torch.cuda.mem_get_info()
        try:
            tk = srv.submit(jobs, r.reads)
            rc, _, _ = srv.poll(tk, r.n_jobs, sa.cigar_max_ops(r.read_len), timeout_ms=300)
            assert rc in (sa.SA_ETIMEOUT, sa.SA_PENDING)      # held back, not failed
        finally:
            del hog
            torch.cuda.empty_cache()
        rc, res, cig = srv.poll(tk, r.n_jobs, sa.cigar_max_ops(r.read_len), timeout_ms=-1)
        assert rc == sa.SA_OK
        ores, oops = oracle.align(r)
        bad = compare(res, cig, ores, oops)
        assert not bad, "\n".join(bad[:10])
        st = srv.stats()
        assert st["admission_stalls"] >= 1 and st["failed"] == 0
