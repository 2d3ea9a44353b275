"""Build libsa.so (the CUDA library) in-tree with nvcc for sm_103a.

One translation unit per wavefront configuration (fill_cfg.cu with -DSA_CFG=c)
plus the staging, dispatch and API units, compiled in parallel, then linked
into ``paper_1302_5507_gb300/libsa.so``.  Objects go to ``_build/`` next to this
file and are reused while their sources are unchanged.
"""
from __future__ import annotations

import concurrent.futures as cf
import fcntl
import glob
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "libsa.so")
OUT_DEBUG = os.path.join(HERE, "libsa_debug.so")   # SA_DEBUG: bounds-checked stores (tests)
PROBE = os.path.join(HERE, "libsa_probe.so")   # instruction-throughput probe used by bench.py
BUILD = os.path.join(HERE, "_build")
NUM_CFG = 33                 # wavefront configurations (kNumCfg in csrc/sa_internal.cuh)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", f"-I{INCLUDE}", f"-I{CSRC}",
         "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsa")


def _units():
    units = [(os.path.join(CSRC, "fill_cfg.cu"), f"fill_cfg{c}.o", [f"-DSA_CFG={c}"])
             for c in range(NUM_CFG)]
    for name in ("fill_dispatch.cu", "stage.cu", "band.cu", "api.cu", "noalloc.cu", "select.cu", "seed.cu"):
        units.append((os.path.join(CSRC, name), name.replace(".cu", ".o"), []))
    return units


def _deps_mtime() -> float:
    files = glob.glob(os.path.join(CSRC, "*.cu*")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        [os.path.join(INCLUDE, "sa.h"), os.path.abspath(__file__)]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, jobs: int | None = None, verbose: bool = False, debug: bool = False) -> str:
    """Build libsa.so, or with debug=True libsa_debug.so (-DSA_DEBUG: every indexed
    global store of the kernels checks its index against its buffer and records the
    store site instead of writing out of range).  Processes that build at the same
    time (the ranks of a multi-GPU run) take turns on a lock file; the later ones
    find the library up to date."""
    bdir = BUILD + ("_debug" if debug else "")
    os.makedirs(bdir, exist_ok=True)
    with open(os.path.join(bdir, "lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        try:
            return _build_locked(force, jobs, verbose, debug)
        finally:
            fcntl.flock(lock, fcntl.LOCK_UN)


def _build_locked(force: bool, jobs: int | None, verbose: bool, debug: bool) -> str:
    out = OUT_DEBUG if debug else OUT
    bdir = BUILD + ("_debug" if debug else "")
    extra_flags = ["-DSA_DEBUG"] if debug else []
    dep = _deps_mtime()
    # objects and library built on another machine type are never reused
    stamp = os.path.join(bdir, "machine")
    machine = platform.machine()
    if not os.path.exists(stamp) or open(stamp).read().strip() != machine:
        force = True
    if not force and os.path.exists(out) and os.path.getmtime(out) >= dep:
        return out
    nvcc = _nvcc()
    todo = []
    for src, obj, extra in _units():
        objp = os.path.join(bdir, obj)
        if force or not os.path.exists(objp) or os.path.getmtime(objp) < dep:
            todo.append([nvcc, *ARCH, *FLAGS, *extra_flags, *extra, "-c", src, "-o", objp])
    jobs = jobs or max(1, min(len(todo) or 1, os.cpu_count() or 1))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)

    with cf.ThreadPoolExecutor(jobs) as ex:
        list(ex.map(run, todo))
    objs = [os.path.join(bdir, obj) for _, obj, _ in _units()]
    tmp = out + ".tmp"
    subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], check=True, capture_output=True)
    os.replace(tmp, out)
    if not debug:
        ptmp = PROBE + ".tmp"
        subprocess.run([nvcc, *ARCH, *FLAGS, "-shared", "-o", ptmp, os.path.join(CSRC, "dpx_probe.cu")],
                       check=True, capture_output=True)
        os.replace(ptmp, PROBE)
    with open(stamp, "w") as f:
        f.write(machine)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
