"""The serving loop's admission policy (csrc/admission.h), host logic only:
compiled into a small driver with the system C++ compiler and fed a sequence of
decisions, no GPU.  Device memory that shrinks between submissions (another
allocation of the process) must hold the head request back; memory that comes
free again must let it start; queued requests coalesce behind the head while
the job limit and the memory allow."""
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1302_5507_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("adm") / "admission_check")
    subprocess.check_call(["g++", "-O1", "-std=c++17", f"-I{CSRC}", os.path.join(HERE, "admission_check.cpp"),
                           "-o", exe])
    return exe


def run(driver, lines):
    out = subprocess.run([driver], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    return out.stdout.split("\n")[:-1]


def test_cap_follows_free_memory(driver):
    GB = 1 << 30
    out = run(driver, [f"cap {80 * GB} {100 * GB} 0",        # budget binds
                       f"cap {80 * GB} {30 * GB} {5 * GB}",   # memory taken elsewhere binds
                       f"cap {80 * GB} 0 {7 * GB}"])           # only the server's own workspaces
    assert [int(x) for x in out] == [80 * GB, 35 * GB, 7 * GB]


def test_admission_follows_shrinking_and_growing_memory(driver):
    GB = 1 << 30
    q = "3 " + " ".join([f"1000 {4 * GB}", f"500 {2 * GB}", f"2000 {1 * GB}"])
    budget = 40 * GB
    steps = []
    # submissions while the free memory shrinks (another allocation in the process)
    for free in (40, 10, 5, 3, 0, 7):
        cap = min(budget, free * GB)
        steps.append((free, f"admit 0 {cap} 1048576 {q}"))
    out = run(driver, [s for _, s in steps])
    got = [tuple(int(v) for v in x.split()) for x in out]
    assert got == [(3, 7 * GB), (3, 7 * GB), (1, 4 * GB), (0, 0), (0, 0), (3, 7 * GB)]


def test_running_batches_and_job_limit(driver):
    GB = 1 << 30
    q = "4 " + " ".join([f"600000 {1 * GB}", f"300000 {1 * GB}", f"200000 {1 * GB}", f"10 {1 * GB}"])
    out = run(driver, [f"admit {30 * GB} {32 * GB} 1048576 {q}",    # 2 GB left beside the running batches
                       f"admit 0 {32 * GB} 1048576 {q}",            # the job limit stops at the third
                       f"admit 0 {32 * GB} 100 {q}",                # the head alone may exceed the limit
                       f"admit {31 * GB + 1} {32 * GB} 1048576 {q}"])  # not even the head fits
    got = [tuple(int(v) for v in x.split()) for x in out]
    assert got == [(2, 2 * GB), (2, 2 * GB), (1, 1 * GB), (0, 0)]
