"""The seeding front end's host index (csrc/seed_index.h) against plain
definitions, without a GPU: the suffix order, the 12-base lookup table and
backward search over the chunked BWT counts (occurrence lists equal to a
direct scan), on small references with planted runs and repeats, in four- and
two-letter alphabets (many equal prefixes) and with lengths that end inside and
at the edge of a 192-row chunk."""
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1302_5507_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("seedidx") / "seed_index_check")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-pthread", f"-I{CSRC}",
                           os.path.join(HERE, "seed_index_check.cpp"), "-o", exe])
    return exe


@pytest.mark.parametrize("length,seed,alpha", [(3000, 1, 4), (2000, 2, 2), (191, 3, 4), (383, 4, 2),
                                               (5000, 5, 4), (40, 6, 4)])
def test_index_matches_plain_definitions(driver, length, seed, alpha):
    out = subprocess.run([driver, str(length), str(seed), str(alpha)], capture_output=True, text=True,
                         timeout=600)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
