"""Python binding of libsa (include/sa.h): batched affine-gap alignment of short
reads against candidate reference windows on one GB300.

Argument marshalling only: every step of the computation runs in the CUDA
library ``libsa.so`` built from ``csrc/`` (``python -m paper_1302_5507_gb300.build``
or ``__graft_entry__.build()``).  Importing the binding without the library
raises; there is no CPU fallback.

The C entry points are exposed under their own names (``sa_create_reference``,
``sa_align_batch``, ``sa_align_batch_dev``, ``sa_server_create``, ``sa_submit``,
``sa_poll``, ...), and ``Reference`` / ``Server`` wrap them for numpy and torch
buffers.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SA_LIBRARY selects another build of the library (the bounds-checked
# libsa_debug.so in the debug tests); default: the in-tree libsa.so
LIB_PATH = os.environ.get("SA_LIBRARY") or os.path.join(_HERE, "libsa.so")

SA_OK, SA_PENDING = 0, 1
SA_EINVAL, SA_ENOMEM, SA_ECUDA, SA_ETIMEOUT, SA_EOVERFLOW, SA_ENOTFOUND, SA_EBUSY = -1, -2, -3, -4, -5, -6, -7
SA_NO_SCORE = -(2 ** 31)
SA_LOCAL, SA_GLOCAL = 0, 1
SA_FORM_BATCHED, SA_FORM_PLAIN = 0, 1
SA_RC = 1
SA_RES_EMPTY, SA_RES_BELOW_MIN = 1, 2
SA_MAX_READ, SA_MAX_WINDOW = 1024, 65536
OPS = "MIDNSHP=X"
SA_NO_JOB, SA_MAPQ_MAX = 0xFFFFFFFF, 60
SA_READ_ALIGNED, SA_READ_PAIRED, SA_READ_PROPER, SA_READ_MATE_ALIGNED, SA_READ_REVERSE = 1, 2, 4, 8, 16
SA_PAIR_FR, SA_PAIR_FF = 0, 1


class sa_scoring(ctypes.Structure):
    _fields_ = [("match", ctypes.c_int32), ("mismatch", ctypes.c_int32),
                ("gap_open", ctypes.c_int32), ("gap_extend", ctypes.c_int32)]


class sa_params(ctypes.Structure):
    _fields_ = [("sc", sa_scoring), ("mode", ctypes.c_int32), ("want_cigar", ctypes.c_int32),
                ("width", ctypes.c_int32), ("min_score", ctypes.c_int32), ("form", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("arena_mb", ctypes.c_int32), ("_reserved", ctypes.c_int32)]


class sa_stats(ctypes.Structure):
    _fields_ = [("jobs", ctypes.c_uint64), ("cells", ctypes.c_uint64), ("rect_cells", ctypes.c_uint64),
                ("overflow_reruns", ctypes.c_uint32), ("waves", ctypes.c_uint32),
                ("fill_launches", ctypes.c_uint32), ("kernel_launches", ctypes.c_uint32),
                ("ms_stage", ctypes.c_float), ("ms_fill", ctypes.c_float), ("ms_rerun", ctypes.c_float),
                ("ms_rect", ctypes.c_float), ("ms_traceback", ctypes.c_float),
                ("ms_finalize", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("diag_jobs", ctypes.c_uint32), ("band_jobs", ctypes.c_uint32),
                ("rect_jobs", ctypes.c_uint32), ("jobs16", ctypes.c_uint32),
                ("graph_replays", ctypes.c_uint32), ("rect_pairs", ctypes.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class sa_server_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("submitted", "completed", "failed", "batches", "coalesced",
                                                "admission_stalls", "max_queue", "jobs")]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class sa_seed_params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint32) for k in ("seed_len", "seed_step", "max_occ", "pad", "join", "_reserved")]


class sa_select_params(ctypes.Structure):
    _fields_ = [("sc", sa_scoring), ("paired", ctypes.c_int32), ("orientation", ctypes.c_int32),
                ("frag_min", ctypes.c_int64), ("frag_max", ctypes.c_int64)]


JOB_DTYPE = np.dtype([("read_off", np.uint64), ("read_len", np.uint32), ("flags", np.uint32),
                      ("ref_pos", np.uint64), ("win_len", np.uint32), ("_pad", np.uint32)])
RESULT_DTYPE = np.dtype([("score", np.int32), ("second", np.int32), ("read_begin", np.int32),
                         ("read_end", np.int32), ("ref_begin", np.int64), ("ref_end", np.int64),
                         ("second_ref_end", np.int64), ("cigar_off", np.uint32),
                         ("cigar_len", np.uint32), ("flags", np.uint32), ("_pad", np.uint32)])
READ_RESULT_DTYPE = np.dtype([("job", np.uint32), ("score", np.int32), ("second", np.int32),
                              ("mapq", np.int32), ("flags", np.uint32), ("n_cand", np.uint32),
                              ("frag_len", np.int64)])
assert JOB_DTYPE.itemsize == 32 and RESULT_DTYPE.itemsize == 56 and READ_RESULT_DTYPE.itemsize == 32

_lib = None
_VP, _U32, _U64, _I32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32


def lib():
    """Load libsa.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(the CUDA library is required; there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        L.sa_default_params.argtypes = [ctypes.POINTER(sa_params)]
        L.sa_default_params.restype = None
        L.sa_create_reference.argtypes = [ctypes.c_char_p, _U64, ctypes.c_int, ctypes.POINTER(_VP)]
        L.sa_destroy_reference.argtypes = [_VP]
        L.sa_reference_length.argtypes = [_VP]
        L.sa_reference_length.restype = _U64
        L.sa_align_batch.argtypes = [_VP, ctypes.POINTER(sa_params), _VP, _U32, _VP, _U64, _VP, _VP,
                                     _U64, ctypes.POINTER(_U64), _VP]
        L.sa_align_batch_dev.argtypes = L.sa_align_batch.argtypes
        L.sa_align_batch_noalloc.argtypes = [_VP, ctypes.POINTER(sa_params), _VP, _U32, _VP, _U64, _VP, _VP]
        L.sa_last_stats.argtypes = [_VP, ctypes.POINTER(sa_stats)]
        L.sa_server_create.argtypes = [_VP, ctypes.POINTER(sa_params), _U64, _U32, ctypes.POINTER(_VP)]
        L.sa_submit.argtypes = [_VP, _VP, _U32, _VP, _U64, ctypes.POINTER(_U64)]
        L.sa_poll.argtypes = [_VP, _U64, ctypes.c_int, _VP, _VP, _U64, ctypes.POINTER(_U64)]
        L.sa_server_destroy.argtypes = [_VP]
        L.sa_server_get_stats.argtypes = [_VP, ctypes.POINTER(sa_server_stats)]
        L.sa_tune.argtypes = [_VP, ctypes.POINTER(sa_params), _VP, _U32, _VP, _U64, ctypes.POINTER(_U32)]
        L.sa_plan_get.argtypes = [_VP, _VP, _U64, ctypes.POINTER(_U64)]
        L.sa_plan_set.argtypes = [_VP, _VP, _U64]
        L.sa_effort_limit_dev.argtypes = [_VP, _VP, _VP, _VP, _U32, _U32, _VP, _VP, _VP,
                                          ctypes.POINTER(_U32), _VP]
        L.sa_effort_limit.argtypes = [_VP, _VP, _VP, _VP, _U32, _U32, _VP, _VP, _VP, ctypes.POINTER(_U32)]
        L.sa_select_dev.argtypes = [_VP, ctypes.POINTER(sa_select_params), _VP, _VP, _VP, _U32, _VP, _VP]
        L.sa_select.argtypes = [_VP, ctypes.POINTER(sa_select_params), _VP, _VP, _VP, _U32, _VP]
        L.sa_default_seed_params.argtypes = [ctypes.POINTER(sa_seed_params)]
        L.sa_default_seed_params.restype = None
        L.sa_seed_index_create.argtypes = [_VP, ctypes.POINTER(_VP)]
        L.sa_seed_index_destroy.argtypes = [_VP]
        L.sa_seed_index_info.argtypes = [_VP, ctypes.POINTER(_U64), ctypes.POINTER(_U64)]
        L.sa_seed_candidates_dev.argtypes = [_VP, ctypes.POINTER(sa_seed_params), _VP, _U64, _VP, _VP, _U32,
                                             _VP, _VP, _VP, _U64, ctypes.POINTER(_U64), _VP]
        L.sa_seed_candidates.argtypes = [_VP, ctypes.POINTER(sa_seed_params), _VP, _U64, _VP, _VP, _U32,
                                         _VP, _VP, _VP, _U64, ctypes.POINTER(_U64)]
        L.sa_last_error.restype = ctypes.c_char_p
        for name in ("sa_create_reference", "sa_destroy_reference", "sa_align_batch",
                     "sa_align_batch_dev", "sa_align_batch_noalloc", "sa_last_stats",
                     "sa_server_create", "sa_submit",
                     "sa_poll", "sa_server_destroy", "sa_tune", "sa_plan_get", "sa_plan_set",
                     "sa_effort_limit_dev", "sa_effort_limit", "sa_select_dev", "sa_select",
                     "sa_server_get_stats", "sa_seed_index_create", "sa_seed_index_destroy",
                     "sa_seed_index_info", "sa_seed_candidates_dev", "sa_seed_candidates"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


class SAError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libsa error {code}: {msg}")
        self.code = code


def _check(rc):
    if rc < 0:
        raise SAError(rc, lib().sa_last_error().decode(errors="replace"))
    return rc


# ---------------------------------------------------------------------------
# the C entry points under their own names

def sa_default_params() -> sa_params:
    p = sa_params()
    lib().sa_default_params(ctypes.byref(p))
    return p


def sa_last_error() -> str:
    return lib().sa_last_error().decode(errors="replace")


def sa_create_reference(acgt, device: int = 0):
    buf = acgt if isinstance(acgt, (bytes, bytearray)) else np.ascontiguousarray(acgt, np.uint8).tobytes()
    h = _VP()
    _check(lib().sa_create_reference(buf, len(buf), device, ctypes.byref(h)))
    return h


def sa_destroy_reference(h):
    return _check(lib().sa_destroy_reference(h))


def sa_align_batch(h, params, jobs_ptr, n_jobs, reads_ptr, reads_len, out_ptr, cigar_ptr, cigar_cap,
                   stream=None):
    used = _U64(0)
    rc = lib().sa_align_batch(h, ctypes.byref(params), jobs_ptr, n_jobs, reads_ptr, reads_len, out_ptr,
                              cigar_ptr, cigar_cap, ctypes.byref(used), stream)
    return rc, used.value


def sa_align_batch_dev(h, params, jobs_ptr, n_jobs, reads_ptr, reads_len, out_ptr, cigar_ptr, cigar_cap,
                       stream=None):
    used = _U64(0)
    rc = lib().sa_align_batch_dev(h, ctypes.byref(params), jobs_ptr, n_jobs, reads_ptr, reads_len,
                                  out_ptr, cigar_ptr, cigar_cap, ctypes.byref(used), stream)
    return rc, used.value


def sa_align_batch_noalloc(h, params, jobs_ptr, n_jobs, reads_ptr, reads_len, out_ptr, stream=None):
    """Allocation-free score pass (see sa.h); returns the status code."""
    return lib().sa_align_batch_noalloc(h, ctypes.byref(params), jobs_ptr, n_jobs, reads_ptr, reads_len,
                                        out_ptr, stream)


def sa_last_stats(h) -> sa_stats:
    s = sa_stats()
    _check(lib().sa_last_stats(h, ctypes.byref(s)))
    return s


def sa_server_create(h, params, hbm_budget=0, max_inflight=0):
    s = _VP()
    _check(lib().sa_server_create(h, ctypes.byref(params), hbm_budget, max_inflight, ctypes.byref(s)))
    return s


def sa_submit(s, jobs_ptr, n_jobs, reads_ptr, reads_len):
    t = _U64(0)
    _check(lib().sa_submit(s, jobs_ptr, n_jobs, reads_ptr, reads_len, ctypes.byref(t)))
    return t.value


def sa_poll(s, ticket, timeout_ms, out_ptr, cigar_ptr, cigar_cap):
    used = _U64(0)
    rc = lib().sa_poll(s, ticket, timeout_ms, out_ptr, cigar_ptr, cigar_cap, ctypes.byref(used))
    return rc, used.value


def sa_server_destroy(s):
    return _check(lib().sa_server_destroy(s))


# ---------------------------------------------------------------------------
# numpy / torch conveniences

def make_params(scoring=(1, 2, 2, 1), mode=SA_LOCAL, want_cigar=True, width=0,
                min_score=SA_NO_SCORE, form=SA_FORM_BATCHED, profile=False, arena_mb=0) -> sa_params:
    p = sa_default_params()
    p.sc.match, p.sc.mismatch, p.sc.gap_open, p.sc.gap_extend = scoring
    p.mode, p.want_cigar, p.width = mode, int(bool(want_cigar)), width
    p.min_score, p.form, p.profile = min_score, form, int(bool(profile))
    p.arena_mb = arena_mb
    return p


def make_select_params(scoring=(1, 2, 2, 1), paired=False, orientation=SA_PAIR_FR, frag_min=0,
                       frag_max=0) -> sa_select_params:
    p = sa_select_params()
    p.sc.match, p.sc.mismatch, p.sc.gap_open, p.sc.gap_extend = scoring
    p.paired, p.orientation = int(bool(paired)), orientation
    p.frag_min, p.frag_max = frag_min, frag_max
    return p


def sa_effort_limit_dev(h, jobs_ptr, support_ptr, first_ptr, n_reads, ceiling, kept_ptr, from_ptr,
                        kept_first_ptr, stream=None):
    n = _U32(0)
    _check(lib().sa_effort_limit_dev(h, jobs_ptr, support_ptr, first_ptr, n_reads, ceiling, kept_ptr,
                                     from_ptr, kept_first_ptr, ctypes.byref(n), stream))
    return n.value


def sa_select_dev(h, params, jobs_ptr, results_ptr, first_ptr, n_reads, out_ptr, stream=None):
    return _check(lib().sa_select_dev(h, ctypes.byref(params), jobs_ptr, results_ptr, first_ptr, n_reads,
                                      out_ptr, stream))


def jobs_array(read_off, read_len, flags, ref_pos, win_len) -> np.ndarray:
    j = np.zeros(len(read_len), JOB_DTYPE)
    j["read_off"], j["read_len"], j["flags"] = read_off, read_len, flags
    j["ref_pos"], j["win_len"] = ref_pos, win_len
    return j


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None and a.size else None


def cigar_max_ops(read_len) -> int:
    return int((2 * np.asarray(read_len, np.int64) + 3).sum())


def cigar_string(ops) -> str:
    return "".join(f"{int(x) >> 4}{OPS[int(x) & 15]}" for x in ops)


class Reference:
    """A device-resident 2-bit reference (sa_create_reference)."""

    def __init__(self, acgt, device: int = 0):
        self.h = sa_create_reference(acgt, device)
        self.device = device

    def close(self):
        if self.h:
            sa_destroy_reference(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return int(lib().sa_reference_length(self.h))

    def stats(self) -> dict:
        return sa_last_stats(self.h).as_dict()

    def tune(self, jobs: np.ndarray, reads: np.ndarray, params: sa_params | None = None) -> int:
        """sa_tune on a sample of jobs; returns the number of length classes tuned."""
        params = params or make_params()
        jobs = np.ascontiguousarray(jobs, JOB_DTYPE)
        reads = np.ascontiguousarray(reads, np.uint8)
        k = _U32()
        _check(lib().sa_tune(self.h, ctypes.byref(params), _ptr(jobs), len(jobs), _ptr(reads), reads.size,
                             ctypes.byref(k)))
        return int(k.value)

    def plan(self) -> bytes:
        """The reference's plan as bytes (sa_plan_get)."""
        need = _U64()
        lib().sa_plan_get(self.h, None, 0, ctypes.byref(need))
        buf = (ctypes.c_uint8 * need.value)()
        _check(lib().sa_plan_get(self.h, buf, need.value, ctypes.byref(need)))
        return bytes(buf)

    def set_plan(self, plan: bytes | None) -> None:
        """Install a plan (sa_plan_set); None restores the default."""
        if plan is None:
            _check(lib().sa_plan_set(self.h, None, 0))
            return
        buf = (ctypes.c_uint8 * len(plan)).from_buffer_copy(plan)
        _check(lib().sa_plan_set(self.h, buf, len(plan)))

    def save_plan(self, path: str) -> None:
        """Write the plan as a JSON cache: the configuration of every read length and
        the width of every configuration (readable), and the plan bytes that
        load_plan installs."""
        import json
        raw = self.plan()
        body = np.frombuffer(raw[8:], np.uint8)
        with open(path, "w") as f:
            json.dump({"format": "libsa plan", "cfg_of_read_length": body[:SA_MAX_READ + 1].tolist(),
                       "width_of_cfg": body[SA_MAX_READ + 1:].astype(np.int8).tolist(),
                       "plan_hex": raw.hex()}, f)

    def load_plan(self, path: str) -> None:
        """Install a plan written by save_plan (sa_plan_set validates it)."""
        import json
        with open(path) as f:
            doc = json.load(f)
        if doc.get("format") != "libsa plan":
            raise ValueError(f"{path} is not a libsa plan cache")
        self.set_plan(bytes.fromhex(doc["plan_hex"]))

    def align(self, jobs: np.ndarray, reads: np.ndarray, params: sa_params | None = None,
              out: np.ndarray | None = None, cigar: np.ndarray | None = None, stream=None):
        """Host buffers in, host results out (sa_align_batch)."""
        params = params or make_params()
        jobs = np.ascontiguousarray(jobs, JOB_DTYPE)
        reads = np.ascontiguousarray(reads, np.uint8)
        n = len(jobs)
        if out is None:
            out = np.zeros(n, RESULT_DTYPE)
        if cigar is None:
            cigar = np.zeros(max(1, cigar_max_ops(jobs["read_len"])), np.uint32)
        rc, used = sa_align_batch(self.h, params, _ptr(jobs), n, _ptr(reads), reads.size, _ptr(out),
                                  _ptr(cigar), cigar.size, stream)
        _check(rc)
        return out, cigar[:used]

    def align_dev(self, jobs, reads, out, cigar, params: sa_params | None = None, stream=None):
        """Device tensors (torch) in and out (sa_align_batch_dev); returns ops used."""
        params = params or make_params()
        st = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
        rc, used = sa_align_batch_dev(self.h, params, ctypes.c_void_p(jobs.data_ptr()),
                                      jobs.numel() * jobs.element_size() // 32,
                                      ctypes.c_void_p(reads.data_ptr()), reads.numel(),
                                      ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(cigar.data_ptr()) if cigar is not None else None,
                                      cigar.numel() if cigar is not None else 0, st)
        _check(rc)
        return used


    # --- reads with several candidate windows (sa_effort_limit*, sa_select*)

    def effort_limit(self, jobs: np.ndarray, support: np.ndarray, read_first: np.ndarray, ceiling: int):
        """Host buffers: (kept jobs, their batch indices, per-read offsets into them)."""
        jobs = np.ascontiguousarray(jobs, JOB_DTYPE)
        support = np.ascontiguousarray(support, np.uint32)
        first = np.ascontiguousarray(read_first, np.uint32)
        n_reads = len(first) - 1
        kept = np.zeros(max(1, len(jobs)), JOB_DTYPE)
        kept_from = np.zeros(max(1, len(jobs)), np.uint32)
        kept_first = np.zeros(n_reads + 1, np.uint32)
        n = _U32(0)
        _check(lib().sa_effort_limit(self.h, _ptr(jobs), _ptr(support), _ptr(first), n_reads, ceiling,
                                     _ptr(kept), _ptr(kept_from), _ptr(kept_first), ctypes.byref(n)))
        return kept[:n.value], kept_from[:n.value], kept_first

    def effort_limit_dev(self, jobs, support, read_first, ceiling, kept, kept_from, kept_first, stream=None):
        """Device tensors (torch); returns the number of kept jobs."""
        st = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
        return sa_effort_limit_dev(self.h, ctypes.c_void_p(jobs.data_ptr()), ctypes.c_void_p(support.data_ptr()),
                                   ctypes.c_void_p(read_first.data_ptr()), read_first.numel() - 1, ceiling,
                                   ctypes.c_void_p(kept.data_ptr()), ctypes.c_void_p(kept_from.data_ptr()),
                                   ctypes.c_void_p(kept_first.data_ptr()), st)

    def select(self, jobs: np.ndarray, results: np.ndarray, read_first: np.ndarray,
               params: sa_select_params | None = None) -> np.ndarray:
        """Host buffers: per-read results (READ_RESULT_DTYPE)."""
        params = params or make_select_params()
        jobs = np.ascontiguousarray(jobs, JOB_DTYPE)
        results = np.ascontiguousarray(results, RESULT_DTYPE)
        first = np.ascontiguousarray(read_first, np.uint32)
        out = np.zeros(len(first) - 1, READ_RESULT_DTYPE)
        _check(lib().sa_select(self.h, ctypes.byref(params), _ptr(jobs), _ptr(results), _ptr(first),
                               len(first) - 1, _ptr(out)))
        return out

    def select_dev(self, jobs, results, read_first, out, params: sa_select_params | None = None, stream=None):
        """Device tensors (torch) in and out."""
        params = params or make_select_params()
        st = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
        return sa_select_dev(self.h, params, ctypes.c_void_p(jobs.data_ptr()), ctypes.c_void_p(results.data_ptr()),
                             ctypes.c_void_p(read_first.data_ptr()), read_first.numel() - 1,
                             ctypes.c_void_p(out.data_ptr()), st)


def make_seed_params(seed_len=20, seed_step=10, max_occ=256, pad=24, join=16) -> sa_seed_params:
    p = sa_seed_params()
    lib().sa_default_seed_params(ctypes.byref(p))
    p.seed_len, p.seed_step, p.max_occ, p.pad, p.join = seed_len, seed_step, max_occ, pad, join
    return p


class SeedIndex:
    """Seeding front end of a reference (sa_seed_index_create / sa_seed_candidates*)."""

    def __init__(self, ref: "Reference"):
        self.ref = ref
        h = _VP()
        _check(lib().sa_seed_index_create(ref.h, ctypes.byref(h)))
        self.h = h

    def info(self) -> dict:
        L, b = _U64(0), _U64(0)
        _check(lib().sa_seed_index_info(self.h, ctypes.byref(L), ctypes.byref(b)))
        return {"ref_len": L.value, "device_bytes": b.value}

    def candidates(self, reads: np.ndarray, read_off: np.ndarray, read_len: np.ndarray,
                   params: sa_seed_params | None = None, cap: int | None = None):
        """Host buffers: (candidate jobs, support, read_first)."""
        params = params or make_seed_params()
        reads = np.ascontiguousarray(reads, np.uint8)
        off = np.ascontiguousarray(read_off, np.uint64)
        ln = np.ascontiguousarray(read_len, np.uint32)
        n_reads = len(ln)
        first = np.zeros(n_reads + 1, np.uint32)
        n = _U64(0)
        if cap is None:
            # size by a first call that only counts
            rc = lib().sa_seed_candidates(self.h, ctypes.byref(params), _ptr(reads), reads.size, _ptr(off),
                                          _ptr(ln), n_reads, None, None, _ptr(first), 0, ctypes.byref(n))
            if rc not in (SA_OK, SA_EOVERFLOW):
                _check(rc)
            cap = n.value
        jobs = np.zeros(max(1, cap), JOB_DTYPE)
        sup = np.zeros(max(1, cap), np.uint32)
        _check(lib().sa_seed_candidates(self.h, ctypes.byref(params), _ptr(reads), reads.size, _ptr(off),
                                        _ptr(ln), n_reads, _ptr(jobs), _ptr(sup), _ptr(first), cap,
                                        ctypes.byref(n)))
        return jobs[:n.value], sup[:n.value], first

    def candidates_dev(self, reads, read_off, read_len, cand, support, read_first,
                       params: sa_seed_params | None = None, stream=None) -> int:
        """Device tensors (torch); returns the number of candidates (SAError
        SA_EOVERFLOW when they do not fit `cand`)."""
        params = params or make_seed_params()
        st = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
        n = _U64(0)
        _check(lib().sa_seed_candidates_dev(self.h, ctypes.byref(params), ctypes.c_void_p(reads.data_ptr()),
                                            reads.numel(), ctypes.c_void_p(read_off.data_ptr()),
                                            ctypes.c_void_p(read_len.data_ptr()), read_len.numel(),
                                            ctypes.c_void_p(cand.data_ptr()), ctypes.c_void_p(support.data_ptr()),
                                            ctypes.c_void_p(read_first.data_ptr()), cand.numel() // 32,
                                            ctypes.byref(n), st))
        return n.value

    def close(self):
        if self.h:
            lib().sa_seed_index_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving loop (sa_server_create / sa_submit / sa_poll)."""

    def __init__(self, ref: Reference, params: sa_params | None = None, hbm_budget: int = 0,
                 max_inflight: int = 0):
        self.ref = ref
        self.h = sa_server_create(ref.h, params or make_params(), hbm_budget, max_inflight)

    def submit(self, jobs: np.ndarray, reads: np.ndarray) -> int:
        jobs = np.ascontiguousarray(jobs, JOB_DTYPE)
        reads = np.ascontiguousarray(reads, np.uint8)
        return sa_submit(self.h, _ptr(jobs), len(jobs), _ptr(reads), reads.size)

    def poll(self, ticket: int, n_jobs: int, max_ops: int, timeout_ms: int = -1):
        """(rc, results, cigar) -- results/cigar are None unless rc == SA_OK."""
        out = np.zeros(n_jobs, RESULT_DTYPE)
        cigar = np.zeros(max(1, max_ops), np.uint32)
        rc, used = sa_poll(self.h, ticket, timeout_ms, _ptr(out), _ptr(cigar), cigar.size)
        if rc == SA_OK:
            return rc, out, cigar[:used]
        if rc in (SA_PENDING, SA_ETIMEOUT):
            return rc, None, None
        _check(rc)
        return rc, None, None

    def stats(self) -> dict:
        """sa_server_get_stats: request, batch and admission counters."""
        st = sa_server_stats()
        _check(lib().sa_server_get_stats(self.h, ctypes.byref(st)))
        return st.as_dict()

    def close(self):
        if self.h:
            sa_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
