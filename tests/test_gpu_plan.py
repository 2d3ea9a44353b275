"""Tuned plan (sa_tune, sa_plan_get/set): results never depend on the plan, a
plan round-trips through its bytes, and malformed plans are refused."""
import numpy as np
import pytest

import oracle
import workloads
from oracle.compare import compare

pytestmark = pytest.mark.gpu

N_CFG8 = 29                                       # lane groups of 8, K = 4 .. 32
N_CFG = N_CFG8 + 4                                # plus lane groups of 32, K = 10, 16, 24, 32
MAX_READ = 1024
CFG_ROWS = [8 * k for k in range(4, 33)] + [32 * k for k in (10, 16, 24, 32)]
FIRST32 = N_CFG8


@pytest.fixture(scope="module")
def sa():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1302_5507_gb300 as sa
    return sa


def _parity(sa, ref, wl, **kw):
    jobs = sa.jobs_array(wl.read_off, wl.read_len, wl.flags, wl.ref_pos, wl.win_len)
    res, cig = ref.align(jobs, wl.reads, sa.make_params(**kw))
    ores, oops = oracle.align(wl, mode=kw.get("mode", 0))
    bad = compare(res, cig, ores, oops)
    assert not bad, "\n".join(bad[:10])
    return ref.stats()


def _plan_bytes(cfg, width):
    head = np.array([0x4C504153, 2], np.uint32).tobytes()
    return head + np.asarray(cfg, np.uint8).tobytes() + np.asarray(width, np.int8).tobytes()


def test_tune_then_align_matches_the_oracle(sa):
    sample = workloads.uneven(seed=7, n_jobs=20_000)
    wl = workloads.uneven(seed=7, n_jobs=2_000, first_item=20_000)    # same genome, other jobs
    with sa.Reference(sample.ref) as ref:
        jobs = sa.jobs_array(sample.read_off, sample.read_len, sample.flags, sample.ref_pos, sample.win_len)
        assert ref.tune(jobs, sample.reads) >= 1
        plan = ref.plan()
        cfg = np.frombuffer(plan[8:8 + MAX_READ + 1], np.uint8)
        assert all(CFG_ROWS[cfg[n]] >= n for n in range(1, MAX_READ + 1))
        for mode in (0, 1):
            _parity(sa, ref, wl, mode=mode)


def test_plan_round_trip_and_explicit_plans(sa):
    wl = workloads.small(61, 1500, n_range=(1, 300), m_range=(1, 400), alphabet=4)
    with sa.Reference(wl.ref) as ref:
        default = ref.plan()
        assert len(default) == 8 + MAX_READ + 1 + N_CFG
        ref.set_plan(default)
        assert ref.plan() == default
        # every length on the 32-lane configurations, 32-bit everywhere
        cfg = [FIRST32] + [next(c for c in range(FIRST32, N_CFG) if CFG_ROWS[c] >= n)
                           for n in range(1, MAX_READ + 1)]
        ref.set_plan(_plan_bytes(cfg, [32] * N_CFG))
        st = _parity(sa, ref, wl)
        assert st["jobs16"] == 0
        # 16-bit forced on every configuration
        ref.set_plan(_plan_bytes(cfg, [16] * N_CFG))
        st = _parity(sa, ref, wl)
        assert st["jobs16"] == wl.n_jobs
        ref.set_plan(None)
        assert ref.plan() == default


def test_malformed_plans_are_refused(sa):
    wl = workloads.small(62, 10)
    with sa.Reference(wl.ref) as ref:
        default = bytearray(ref.plan())
        too_small = bytearray(default)
        too_small[8 + 200] = 0                  # 200 bases on 8 x 4 = 32 rows
        for bad in (bytes(too_small), bytes(default[:-1]), b"XXXX" + bytes(default[4:])):
            with pytest.raises(sa.SAError) as e:
                ref.set_plan(bad)
            assert e.value.code == sa.SA_EINVAL
        bad_width = bytearray(default)
        bad_width[-1] = 8
        with pytest.raises(sa.SAError):
            ref.set_plan(bytes(bad_width))
        assert ref.plan() == bytes(default)


def test_plan_json_cache_round_trip(sa, tmp_path):
    """save_plan / load_plan: the JSON cache shows the tables and reinstalls the
    exact plan bytes."""
    wl = workloads.uneven(seed=3, n_jobs=2_000)
    cfg = [0] + [next(c for c in range(N_CFG) if CFG_ROWS[c] >= n) for n in range(1, MAX_READ + 1)]
    cfg[150] = FIRST32                              # a 32-lane configuration for length 150
    width = [0] * N_CFG
    width[15] = 32
    plan = _plan_bytes(cfg, width)
    with sa.Reference(wl.ref) as ref:
        ref.set_plan(plan)
        path = tmp_path / "plan.json"
        ref.save_plan(str(path))
        import json
        doc = json.loads(path.read_text())
        assert doc["cfg_of_read_length"][150] == FIRST32 and doc["width_of_cfg"][15] == 32
        ref.set_plan(None)
        assert ref.plan() != plan
        ref.load_plan(str(path))
        assert ref.plan() == plan
        _parity(sa, ref, wl)
