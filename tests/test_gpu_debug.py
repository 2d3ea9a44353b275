"""Bounds-checked build (SA_DEBUG): every indexed global store of the kernels
checks its index against its buffer and reports an out-of-range store as an
internal error.  The checked library must give the oracle's results on every
path (both widths, both modes, both forms, every traceback class, the rectangle
arena in waves, the rectangle pass two jobs a lane group) without reporting a store."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHECK = r"""
import sys
sys.path.insert(0, ROOT)
import numpy as np
import oracle, workloads
from oracle.compare import compare
import paper_1302_5507_gb300 as sa
assert sa.LIB_PATH.endswith("libsa_debug.so"), sa.LIB_PATH
cases = [workloads.small(71, 1500, n_range=(1, 300), m_range=(1, 500), alphabet=4),
         workloads.small(72, 800, n_range=(1, 60), m_range=(1, 120), alphabet=2),
         workloads.mate_rescue(3, 3000, genome_len=4_000_000),
         workloads.uneven(3, 2000, genome_len=4_000_000),
         workloads.lowsim(3, 400, genome_len=4_000_000)]
for wl in cases:
    jobs = sa.jobs_array(wl.read_off, wl.read_len, wl.flags, wl.ref_pos, wl.win_len)
    with sa.Reference(wl.ref) as ref:
        for mode in (0, 1):
            ores, oops = oracle.align(wl, mode=mode)
            for form, width in ((0, 0), (0, 16), (0, 32), (1, 0)):
                res, cig = ref.align(jobs, wl.reads, sa.make_params(mode=mode, form=form, width=width))
                bad = compare(res, cig, ores, oops)
                assert not bad, (wl.name, mode, form, width, bad[:5])
            # the rectangle arena capped so that its passes and walks run in waves
            res, cig = ref.align(jobs, wl.reads, sa.make_params(mode=mode, arena_mb=4))
            bad = compare(res, cig, ores, oops)
            assert not bad, (wl.name, mode, "waves", bad[:5])
# enough rectangle jobs in one bucket for its pass to run two jobs a lane group
wl = workloads.lowsim(4, 60_000, genome_len=4_000_000)
jobs = sa.jobs_array(wl.read_off, wl.read_len, wl.flags, wl.ref_pos, wl.win_len)
ores, oops = oracle.align(wl)
with sa.Reference(wl.ref) as ref:
    for arena_mb in (0, 64):
        res, cig = ref.align(jobs, wl.reads, sa.make_params(arena_mb=arena_mb))
        assert ref.stats()["rect_pairs"] > 0, ref.stats()
        bad = compare(res, cig, ores, oops)
        assert not bad, (wl.name, "rectangle pairs", arena_mb, bad[:5])
print("bounds-checked build: all cases exact")
""".replace("ROOT", repr(ROOT))


def test_bounds_checked_build_matches_the_oracle():
    sys.path.insert(0, ROOT)
    from paper_1302_5507_gb300 import build
    lib = build.build(debug=True)
    r = subprocess.run([sys.executable, "-c", CHECK], env={**os.environ, "SA_LIBRARY": lib},
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "all cases exact" in r.stdout
