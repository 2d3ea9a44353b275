"""Seeded synthetic workloads (shared input generator; no alignment arithmetic).

Both the CPU oracle and the CUDA library consume the arrays produced here, so
parity tests compare the two on identical bytes.  The generator is compiled
from ``synth.c`` (plain C, counter-based splitmix64 draws, integer-only
arithmetic, so x86-64 and aarch64 produce identical workloads).

The five workload recipes restate the shapes of the paper's experiments
(Illumina-like 100/150 bp reads, 500 bp inserts, reads of 50-250 bp; see the
paper's Experiments section and its Methods on paired-end alignment):

* ``plain``        10,000 windows of 400 bp, 100 bp reads, 2 % subs, 0.2 % indels U[1,5]
* ``mate_rescue``  100 Mbp genome (GC 41 % + 5 % repeats at 10 % divergence), 150 bp
                   mates, insert ~ N(500, 50), 800 bp windows from the mate position
* ``uneven``       n ~ U[50,250], m ~ U[ceil(1.5 n), 6 n] from the mate-rescue genome
* ``lowsim``       n = 250, m = 1000, divergence {0,5,10,20,30,40} %, geometric indels <= 30
* ``serving``      3.1 Gbp i.i.d. genome, requests of U[1, 50000] jobs, m ~ U[2n, 6n]
* ``pairs``        paired 150 bp reads (insert ~ N(500, 50)) on the mate-rescue genome, each
                   read with its source window, decoy windows and (for some pairs) a planted
                   copy of end 2's source; per-candidate seed-support counts
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, f"libsynth.{platform.machine()}.so")
_lib = None

# workload ids (part of the stream keys)
W_PLAIN, W_MATE, W_UNEVEN, W_LOWSIM, W_SERVE, W_PAIRS = 1, 2, 3, 4, 5, 6
# job recipe kinds in synth.c
_J_PLAIN, _J_MATE, _J_UNEVEN, _J_LOWSIM, _J_SERVE = 1, 2, 3, 4, 5
FLAG_RC = 1  # job flag: align the reverse complement of the read


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "synth.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"       # per process: concurrent builds never share a file
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               src, "-o", tmp])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        u32, u64, i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        p = ctypes.c_void_p
        lib.synth_reference.argtypes = [u32, u64, u64, u32, p, i32]
        lib.synth_paste_repeats.argtypes = [u32, u64, p, u64, u32, u32, u32]
        lib.synth_job_read_lens.argtypes = [u32, u32, u64, u64, u32, u32, u32, u32, u32, u32,
                                            u64, u64, p]
        lib.synth_jobs.argtypes = [u32, u32, u64, p, u64, u32, u32, u32, u32, u32, u32,
                                   u32, u32, u32, u32, u32, u64, u64,
                                   p, p, p, p, p, p, p, i32]
        lib.synth_uniform.argtypes = [u32, u64, u32, u64, u64, u64, p, p]
        lib.synth_pairs_plant.argtypes = [u32, u64, p, u64, u32, u32, u32, u32, u64, u64]
        lib.synth_pairs_counts.argtypes = [u32, u64, u64, u32, u32, u32, u64, u64, p]
        lib.synth_pairs.argtypes = [u32, u64, p, u64, u32, u32, u32, u32, u32, u64, u64, p,
                                    p, p, p, p, p, p, p, p, i32]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def _threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


@dataclass
class Workload:
    """A batch of alignment jobs over one reference (all arrays host numpy)."""
    name: str
    ref: np.ndarray            # uint8 ASCII 'ACGT'
    reads: np.ndarray          # uint8 ASCII, reads concatenated
    read_off: np.ndarray       # uint64 offset of each read in ``reads``
    read_len: np.ndarray       # uint32 n
    flags: np.ndarray          # uint32 (FLAG_RC)
    ref_pos: np.ndarray        # uint64 window start in ``ref``
    win_len: np.ndarray        # uint32 m
    truth: np.ndarray          # uint64 source position the read was drawn from
    meta: dict = field(default_factory=dict)

    @property
    def n_jobs(self) -> int:
        return int(self.read_len.shape[0])

    @property
    def cells(self) -> int:
        return int(np.dot(self.read_len.astype(np.int64), self.win_len.astype(np.int64)))

    def subset(self, idx) -> "Workload":
        """Jobs ``idx`` (an index array or slice) sharing the same reference."""
        idx = np.arange(self.n_jobs)[idx] if isinstance(idx, slice) else np.asarray(idx)
        n = self.read_len[idx]
        off = np.zeros(len(idx), np.uint64)
        if len(idx):
            off[1:] = np.cumsum(n[:-1].astype(np.uint64))
        total = int(n.astype(np.int64).sum())
        reads = np.empty(total, np.uint8)
        for k, j in enumerate(idx):
            o = int(self.read_off[j])
            reads[int(off[k]):int(off[k]) + int(n[k])] = self.reads[o:o + int(n[k])]
        return Workload(self.name, self.ref, reads, off, n.copy(), self.flags[idx].copy(),
                        self.ref_pos[idx].copy(), self.win_len[idx].copy(),
                        self.truth[idx].copy(), dict(self.meta))


def reference(workload: int, seed: int, length: int, gc: float = 0.5,
              repeats: tuple | None = None) -> np.ndarray:
    """i.i.d. reference with GC fraction ``gc``; ``repeats`` = (copies, seg_len, divergence)."""
    lib = _load()
    out = np.empty(length, np.uint8)
    lib.synth_reference(workload, seed, length, int(round(gc * 1e6)), _ptr(out), _threads())
    if repeats:
        copies, seg, div = repeats
        lib.synth_paste_repeats(workload, seed, _ptr(out), length, copies, seg,
                                int(round(div * 1e6)))
    return out


def _jobs(name, kind, workload, seed, ref, n_jobs, *, win_len=0, rlen=0, n_lo=0, n_hi=0,
          m_lo_x10=0, m_hi_x=0, insert=(0, 0), win_before=0, win_total=0, flip_rc=0,
          first_item=0) -> Workload:
    lib = _load()
    n = np.empty(n_jobs, np.uint32)
    lib.synth_job_read_lens(kind, workload, seed, len(ref), win_len, rlen, n_lo, n_hi,
                            m_lo_x10, m_hi_x, first_item, n_jobs, _ptr(n))
    off = np.zeros(n_jobs, np.uint64)
    if n_jobs:
        off[1:] = np.cumsum(n[:-1].astype(np.uint64))
    reads = np.empty(int(n.astype(np.int64).sum()), np.uint8)
    read_len = np.empty(n_jobs, np.uint32)
    flags = np.empty(n_jobs, np.uint32)
    ref_pos = np.empty(n_jobs, np.uint64)
    wl = np.empty(n_jobs, np.uint32)
    truth = np.empty(n_jobs, np.uint64)
    lib.synth_jobs(kind, workload, seed, _ptr(ref), len(ref), win_len, rlen,
                   n_lo, n_hi, m_lo_x10, m_hi_x, insert[0], insert[1], win_before, win_total,
                   flip_rc, first_item, n_jobs, _ptr(off), _ptr(read_len), _ptr(flags),
                   _ptr(ref_pos), _ptr(wl), _ptr(reads), _ptr(truth), _threads())
    return Workload(name, ref, reads, off, read_len, flags, ref_pos, wl, truth,
                    {"seed": seed, "workload": workload})


# ---------------------------------------------------------------------------
# the five recipes

def plain(seed: int = 1, n_jobs: int = 10_000, win: int = 400, read: int = 100) -> Workload:
    """10,000 independent 400 bp uniform windows (concatenated), 100 bp reads."""
    ref = reference(W_PLAIN, seed, n_jobs * win, 0.5)
    return _jobs("plain", _J_PLAIN, W_PLAIN, seed, ref, n_jobs, win_len=win, rlen=read)


_GENOME_CACHE: dict = {}


def genome(seed: int = 1, length: int = 100_000_000) -> np.ndarray:
    """Mate-rescue genome: GC 41 % i.i.d. plus 5 % of its length as 300 bp repeats
    copied from uniform sources with 10 % substitutions."""
    key = (seed, length)
    if key not in _GENOME_CACHE:
        copies = (length // 20) // 300
        _GENOME_CACHE.clear()
        _GENOME_CACHE[key] = reference(W_MATE, seed, length, 0.41, (copies, 300, 0.10))
    return _GENOME_CACHE[key]


def mate_rescue(seed: int = 1, n_pairs: int = 1_000_000, genome_len: int = 100_000_000,
                read: int = 150, first_item: int = 0) -> Workload:
    """Unaligned mate (150 bp, reverse-complemented, flagged RC) against an 800 bp
    window starting 400 bp before the expected mate position (mate + 500)."""
    ref = genome(seed, genome_len)
    return _jobs("mate_rescue", _J_MATE, W_MATE, seed, ref, n_pairs, win_len=800, rlen=read,
                 insert=(500, 50), win_before=400, win_total=800, flip_rc=FLAG_RC,
                 first_item=first_item)


def uneven(seed: int = 1, n_jobs: int = 4_000_000, genome_len: int = 100_000_000,
           n_range=(50, 250), first_item: int = 0) -> Workload:
    ref = genome(seed, genome_len)
    return _jobs("uneven", _J_UNEVEN, W_UNEVEN, seed, ref, n_jobs, n_lo=n_range[0],
                 n_hi=n_range[1], m_lo_x10=15, m_hi_x=6, first_item=first_item)


def lowsim(seed: int = 1, n_jobs: int = 500_000, genome_len: int = 100_000_000,
           first_item: int = 0) -> Workload:
    ref = genome(seed, genome_len)
    return _jobs("lowsim", _J_LOWSIM, W_LOWSIM, seed, ref, n_jobs, win_len=1000, rlen=250,
                 first_item=first_item)


def serving_reference(seed: int = 1, length: int = 3_100_000_000) -> np.ndarray:
    return reference(W_SERVE, seed, length, 0.5)


def serving_request(ref: np.ndarray, seed: int, request: int, n_jobs: int) -> Workload:
    """Jobs of one serving request; job items are keyed by (request, index)."""
    return _jobs("serving", _J_SERVE, W_SERVE, seed, ref, n_jobs, n_lo=50, n_hi=250,
                 m_lo_x10=20, m_hi_x=6, first_item=(request << 20))


def serving_arrivals(seed: int, n_requests: int, max_jobs: int = 50_000):
    """(jobs per request ~ U[1, max_jobs], uniform ppm for exponential gaps)."""
    lib = _load()
    sizes = np.empty(n_requests, np.uint64)
    ppm = np.empty(n_requests, np.uint32)
    lib.synth_uniform(W_SERVE, seed, 7, n_requests, 1, max_jobs, _ptr(sizes), _ptr(ppm))
    return sizes, ppm


def small(seed: int, n_jobs: int, n_range=(1, 40), m_range=(1, 90), ref_len: int = 20_000,
          alphabet: int = 4) -> Workload:
    """Small random jobs for parity tests: arbitrary n, m (including m < n), optional
    reduced alphabet (alphabet=2 draws only A/C, which makes ties frequent)."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    letters = np.frombuffer(b"ACGT", np.uint8)[:alphabet]
    ref = letters[rng.integers(0, alphabet, ref_len)]
    n = rng.integers(n_range[0], n_range[1] + 1, n_jobs).astype(np.uint32)
    m = rng.integers(m_range[0], m_range[1] + 1, n_jobs).astype(np.uint32)
    m = np.minimum(m, ref_len).astype(np.uint32)
    pos = np.array([rng.integers(0, ref_len - int(mm) + 1) for mm in m], np.uint64)
    off = np.zeros(n_jobs, np.uint64)
    if n_jobs:
        off[1:] = np.cumsum(n[:-1].astype(np.uint64))
    reads = np.empty(int(n.astype(np.int64).sum()), np.uint8)
    for j in range(n_jobs):
        o, nn = int(off[j]), int(n[j])
        if rng.random() < 0.6 and int(m[j]) >= nn:
            # a mutated copy of a piece of the window, so alignments are non-trivial
            s = int(pos[j]) + int(rng.integers(0, int(m[j]) - nn + 1))
            seg = ref[s:s + nn].copy()
            flips = rng.random(nn) < 0.1
            seg[flips] = letters[rng.integers(0, alphabet, int(flips.sum()))]
            reads[o:o + nn] = seg
        else:
            reads[o:o + nn] = letters[rng.integers(0, alphabet, nn)]
    flags = (rng.random(n_jobs) < 0.25).astype(np.uint32) * FLAG_RC
    return Workload("small", ref, reads, off, n, flags, pos, m, pos.copy(), {"seed": seed})


@dataclass
class PairedWorkload(Workload):
    """Candidate jobs of paired reads: the jobs of read r are read_first[r] ..
    read_first[r+1]-1 (reads 2p and 2p+1 are the ends of pair p); every
    candidate carries its seed support."""
    read_first: np.ndarray = None      # uint64, n_reads + 1
    support: np.ndarray = None         # uint32 per job
    read_truth: np.ndarray = None      # uint64 source position per read

    @property
    def n_reads(self) -> int:
        return int(self.read_first.shape[0]) - 1


def pairs(seed: int = 1, n_pairs: int = 100_000, genome_len: int = 100_000_000, read: int = 150,
          decoy_max: int = 40, dup: float = 0.1, first_item: int = 0) -> PairedWorkload:
    """Paired reads with several candidate windows each (source window, a shifted
    copy of it for 20 % of reads, U[0, decoy_max] uniform decoys, and for a
    fraction ``dup`` of pairs a window on a planted copy of end 2's source).
    The planted copies go into a private copy of the mate-rescue genome."""
    lib = _load()
    ref = genome(seed, genome_len).copy()
    dup_ppm = int(round(dup * 1e6))
    lib.synth_pairs_plant(W_PAIRS, seed, _ptr(ref), len(ref), read, 500, 50, dup_ppm, first_item,
                          n_pairs)
    counts = np.empty(2 * n_pairs, np.uint32)
    lib.synth_pairs_counts(W_PAIRS, seed, len(ref), read, min(decoy_max, 61), dup_ppm, first_item,
                           n_pairs, _ptr(counts))
    read_first = np.zeros(2 * n_pairs + 1, np.uint64)
    read_first[1:] = np.cumsum(counts.astype(np.uint64))
    n_jobs = int(read_first[-1])
    reads = np.empty(2 * n_pairs * read, np.uint8)
    read_truth = np.empty(2 * n_pairs, np.uint64)
    off = np.empty(n_jobs, np.uint64)
    rl = np.empty(n_jobs, np.uint32)
    fl = np.empty(n_jobs, np.uint32)
    pos = np.empty(n_jobs, np.uint64)
    wl = np.empty(n_jobs, np.uint32)
    sup = np.empty(n_jobs, np.uint32)
    lib.synth_pairs(W_PAIRS, seed, _ptr(ref), len(ref), read, 500, 50, min(decoy_max, 61), dup_ppm,
                    first_item, n_pairs, _ptr(read_first), _ptr(reads), _ptr(read_truth), _ptr(off),
                    _ptr(rl), _ptr(fl), _ptr(pos), _ptr(wl), _ptr(sup), _threads())
    truth = np.repeat(read_truth, counts.astype(np.int64))
    return PairedWorkload("pairs", ref, reads, off, rl, fl, pos, wl, truth,
                          {"seed": seed, "workload": W_PAIRS}, read_first=read_first, support=sup,
                          read_truth=read_truth)
