"""ORACLE -- test infrastructure only.

Python front end of the plain-C full-matrix Gotoh oracle in ``oracle.c``.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package; the alignment library never
does, and it shares no code with it.

Scoring is given in BWA magnitudes (match a, mismatch b, gap open o, gap
extend e; a gap of length L costs o + L*e) and converted here to the signed
form of the paper's recurrence (Methods section 3): S_MA = a, S_MI = -b,
S_GO = -(o+e), S_GE = -e.
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, f"liboracle.{platform.machine()}.so")
_lib = None

LOCAL, GLOCAL = 0, 1
EMPTY, BELOW_MIN = 1, 2
NO_SCORE = -(2 ** 31)
OPS = "MIDNSHP=X"

RESULT_DTYPE = np.dtype([
    ("score", np.int32), ("second", np.int32), ("read_begin", np.int32), ("read_end", np.int32),
    ("ref_begin", np.int64), ("ref_end", np.int64), ("second_ref_end", np.int64),
    ("n_ops", np.int32), ("flags", np.uint32)])

# BWA-style default implied by the paper's default gap tolerance (see tests/test_oracle_pins.py)
DEFAULT_SCORING = (1, 2, 2, 1)


def build(force: bool = False, src: str | None = None, out: str | None = None,
          defines=()) -> str:
    """Compile the oracle with plain gcc -O2 (no intrinsics)."""
    src = src or os.path.join(_HERE, "oracle.c")
    out = out or _SO
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + f".{os.getpid()}.tmp"       # per process: concurrent builds never share a file
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               *[f"-D{d}" for d in defines], src, "-o", tmp])
        os.replace(tmp, out)
    return out


def _bind(path: str):
    lib = ctypes.CDLL(path)
    p, i32, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64
    lib.oracle_align_batch.argtypes = [p, u64, p, p, p, p, p, p, u64,
                                       i32, i32, i32, i32, ctypes.c_int, ctypes.c_int, i32,
                                       p, p, u64, ctypes.c_int]
    lib.oracle_align_batch.restype = ctypes.c_int
    lib.oracle_matrices.argtypes = [p, ctypes.c_int, p, ctypes.c_int, i32, i32, i32, i32,
                                    ctypes.c_int, p, p, p]
    lib.oracle_sizeof_result.restype = ctypes.c_int
    assert lib.oracle_sizeof_result() == RESULT_DTYPE.itemsize
    return lib


def _load():
    global _lib
    if _lib is None:
        path = os.environ.get("ORACLE_LIB")   # tests load planted-mistake builds this way
        if not path:
            build()
            path = _SO
        _lib = _bind(path)
    return _lib


def signed(scoring):
    """BWA magnitudes (a, b, o, e) -> signed (S_MA, S_MI, S_GO, S_GE)."""
    a, b, o, e = scoring
    return a, -b, -(o + e), -e


def _p(x):
    return ctypes.c_void_p(x.ctypes.data) if x is not None else None


def threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def align_arrays(ref, reads, read_off, read_len, flags, ref_pos, win_len, *, scoring=DEFAULT_SCORING,
                 mode=LOCAL, want_cigar=True, min_score=NO_SCORE, n_threads=None, lib=None):
    """Align every job; returns (results[RESULT_DTYPE], ops[n_jobs, stride] uint32)."""
    lib = lib or _load()
    n_jobs = len(read_len)
    a, b, go, ge = signed(scoring)
    res = np.zeros(n_jobs, RESULT_DTYPE)
    stride = 2 * int(read_len.max()) + 3 if n_jobs else 1
    ops = np.zeros((n_jobs, stride), np.uint32) if want_cigar else None
    conv = [np.ascontiguousarray(x, dt) for x, dt in
            ((ref, np.uint8), (reads, np.uint8), (read_off, np.uint64), (read_len, np.uint32),
             (flags, np.uint32), (ref_pos, np.uint64), (win_len, np.uint32))]
    st = lib.oracle_align_batch(_p(conv[0]), len(conv[0]), _p(conv[1]), _p(conv[2]), _p(conv[3]),
                                _p(conv[4]), _p(conv[5]), _p(conv[6]), n_jobs, a, b, go, ge, mode,
                                int(bool(want_cigar)), min_score, _p(res), _p(ops), stride,
                                n_threads or threads())
    if st != 0:
        raise ValueError(f"oracle_align_batch failed with status {st}")
    return res, ops


def align(wl, **kw):
    """Align a ``workloads.Workload``."""
    return align_arrays(wl.ref, wl.reads, wl.read_off, wl.read_len, wl.flags, wl.ref_pos,
                        wl.win_len, **kw)


def align_pair(window: str, read: str, **kw):
    """Align one read against one window given as strings; returns (result, cigar str)."""
    ref = np.frombuffer(window.encode(), np.uint8)
    reads = np.frombuffer(read.encode(), np.uint8)
    res, ops = align_arrays(ref, reads, np.zeros(1, np.uint64), np.array([len(read)], np.uint32),
                            np.zeros(1, np.uint32), np.zeros(1, np.uint64),
                            np.array([len(window)], np.uint32), **kw)
    r = res[0]
    cig = cigar_string(ops[0][: r["n_ops"]]) if ops is not None else ""
    return r, cig


def cigar_string(ops) -> str:
    return "".join(f"{int(x) >> 4}{OPS[int(x) & 15]}" for x in ops)


_CODE = {ord("A"): 0, ord("C"): 1, ord("G"): 2, ord("T"): 3}


def codes(s: str) -> np.ndarray:
    return np.array([_CODE[c] for c in s.encode()], np.uint8)


def matrices(window: str, read: str, *, scoring=DEFAULT_SCORING, mode=LOCAL):
    """(H, E, F) as (m+1, n+1) int32 arrays."""
    lib = _load()
    T, R = codes(window), codes(read)
    m, n = len(T), len(R)
    H = np.zeros((m + 1, n + 1), np.int32)
    E = np.zeros_like(H)
    F = np.zeros_like(H)
    a, b, go, ge = signed(scoring)
    lib.oracle_matrices(_p(T), m, _p(R), n, a, b, go, ge, mode, _p(H), _p(E), _p(F))
    return H, E, F
