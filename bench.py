"""Benchmark: GCUPS of batched affine-gap alignment (score + traceback + CIGAR)
on one GB300.  The headline line is the uneven-length batch: 4M jobs, reads of
50-250 bp against windows of 1.5-6x their length on a synthetic 100 Mbp genome,
16-bit packed scores with exact overflow detection and a 32-bit rerun, the
length-bucket plan picked by the library's autotuner (sa_tune), and the score
segment replayed as a CUDA graph.  The same line carries the mate-rescue batch
(1M 150 bp mates against 800 bp windows) in 32-bit scores, with its 16-bit
figure beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

One step = one call of the library on the whole batch: staging (read packing,
bucketing), the score pass, the overflow rerun, the reduced direction pass,
traceback, CIGAR compaction and results.  `value` times steps whose inputs
already sit in device memory (sa_align_batch_dev); `e2e` times sa_align_batch
from pinned host buffers, host<->device copies included.  Cells = sum of n*m
(full matrices).  With --impl reference the CPU oracle is timed instead, on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GCUPS (affine DP incl. traceback) at 1 GB300 vs plain form; p50/p99 request latency"
WORKLOADS = {
    "c3": "uneven (C3): 4M jobs, n U[50,250], m U[1.5n,6n], windows in a 100 Mbp GC41 genome + 5% repeats; "
          "int16 packed + exact int32 rerun, autotuned plan, score segment replayed as a CUDA graph",
    "c2": "mate_rescue (C2): 1M jobs, 150 bp mate (reverse-complemented) vs 800 bp window, 100 Mbp GC41 genome "
          "+ 5% repeats; int32 scores",
}
DEFAULT_JOBS = {"c3": 4_000_000, "c2": 1_000_000}
OPS_PER_CELL = 6          # lane-ops per cell of the roofline formula: 1 add H+GO, 2 add-max (E, F), 1 add diag+delta, 1 max3, 1 column-max update
# issue-aware bound: the half-rate instructions (DPX maxima on the ALU pipe, integer
# multiply-adds on the FMA pipe) the recurrence needs per register of two 16-bit
# cells (or one 32-bit cell): the add-maxima of G (with the zero floor), E and F, the
# three-way maximum of H, the add forming H + S_GO, and half a maximum for the
# column maximum (three-way maxima over a lane's rows).  The probe shows the two
# pipes share their issue (add-max alone 63.7, multiply-add alone 62.0, the two
# interleaved 69.6 lane-ops per SM per clock), so they are counted together at the
# interleaved rate.
ISSUE_OPS_PER_REG = 5.5
PROBE_S16X2, PROBE_S32, PROBE_IMAD, PROBE_MIX = 6, 0, 5, 11   # operation codes of the throughput probe


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--jobs", type=int, default=None,
                    help="jobs per GPU (default: the configuration's size, 4M for c3, 1M for c2)")
    ap.add_argument("--no-tune", action="store_true", help="keep the default plan (skip sa_tune)")
    ap.add_argument("--width", type=int, default=None, choices=[0, 16, 32],
                    help="score width of the line's batches (default: 32 for c2, as its spec says; "
                         "0 = 16-bit pairs where no job of a bucket can overflow, for c3)")
    ap.add_argument("--no-c2", action="store_true", help="skip the mate-rescue object of the headline line")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-form comparison")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving latency run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--slots", type=int, default=2, help="in-flight slots of the serving runs")
    ap.add_argument("--probe-ops", action="store_true",
                    help="print the measured issue rate (lane-ops per SM per clock) of every "
                         "operation of the throughput probe and exit")
    ap.add_argument("--config", default="c3", choices=["c1", "c2", "c3", "c3-detail", "c4", "c5", "pairs", "seeds"],
                    help="c3 (default): the headline line on the uneven 4M-job batch; c2: the same "
                         "line on the mate-rescue batch; c1 plain windows (plain and batched forms, "
                         "both modes) plus mate rescue in GLOCAL; c3-detail: the uneven batch per "
                         "width and plan; c4 low similarity, c5 serving sweep, pairs: paired reads "
                         "with several candidate windows each (effort limit, alignment, selection): "
                         "one extra JSON line each (1 GPU)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,utilization.gpu,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            try:
                rows.append(dict(sm=float(f[1]), max=float(f[2]), util=float(f[3]), hw=f[6], hwt=f[7],
                                 swt=f[8], swp=f[9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}
        load = [r for r in rows if r["util"] >= 50] or rows
        reasons = sorted({name for r in load for name, key in
                          (("hw_slowdown", "hw"), ("hw_thermal_slowdown", "hwt"),
                           ("sw_thermal_slowdown", "swt"), ("sw_power_cap", "swp"))
                          if r[key].lower() == "active"})
        return {"sm_mhz": statistics.median(r["sm"] for r in load), "sm_max_mhz": max(r["max"] for r in rows),
                "reasons": reasons, "samples": len(load)}


# ---------------------------------------------------------------------------

def kernel_source_sha():
    """sha1 (12 hex digits) of the score-pass kernel sources (fill.cuh + fill16.cuh)."""
    h = hashlib.sha1()
    for f in ("fill.cuh", "fill16.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1302_5507_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:12]


TRAFFIC_CSV = os.path.join(ROOT, "profiles", "score_pass_traffic.csv")


def traffic_per_step(config: str, jobs: int):
    """DRAM read + write bytes of the score-pass kernels in one step of `config`
    with `jobs` jobs, from the committed ncu figures (profiles/score_pass_traffic.csv:
    bytes of the captured step scaled by jobs), if they were taken on the current
    kernel sources; else None."""
    if not os.path.exists(TRAFFIC_CSV):
        return None
    with open(TRAFFIC_CSV) as f:
        for row in csv.DictReader(f):
            if row["config"] == config and row["kernel_sources_sha1"] == kernel_source_sha():
                return float(row["dram_bytes"]) * jobs / float(row["jobs"])
    return None


def direction_bound(stats, wl):
    """HBM roofline of the traceback's direction data: GCUPS (over all cells of the
    batch) if only writing its band heights / rectangle nibbles limited the step."""
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        gbs, basis = float(peaks["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        gbs, basis = 6800.0, "fallback"
    return {"hbm_gbs": gbs, "hbm_basis": basis,
            "full_matrix_nibbles_gcups": gbs / 0.5,
            "note": "the band passes write bytes only for cells on the diagonals an optimal path "
                    "can use, so their data is a small fraction of 0.5 B per cell of the batch"}


PROBE_OPS = ("viaddmax_s32", "vimax3_s32", "vimax3_s32_relu", "iadd_s32", "imax_s32", "imad_s32",
             "viaddmax_s16x2", "vimax3_s16x2", "prmt", "vmaxs4 (s8x4)", "vaddss4 (s8x4)",
             "viaddmax_s16x2 + imad (half the chains each)", "viaddmax_s16x2 + prmt (half the chains each)",
             "lop3", "iadd3", "ffma (fp32)", "hmax2 (fp16x2)",
             "viaddmax_s16x2 + lop3", "viaddmax_s16x2 + iadd3", "viaddmax_s16x2 + ffma",
             "viaddmax_s16x2 + hmax2", "viaddmax_s16x2 + funnel shift")


def probe_all_ops():
    """Issue rate of every probe operation, lane-ops per SM per clock (median of 5,
    at the median SM clock sampled meanwhile)."""
    import ctypes
    import torch
    from paper_1302_5507_gb300 import build as sa_build
    torch.cuda.set_device(0)
    sa_build.build()
    lib = ctypes.CDLL(sa_build.PROBE)
    lib.sa_probe_ops_per_sm_clk.restype = ctypes.c_double
    lib.sa_probe_ops_per_sm_clk.argtypes = [ctypes.c_int, ctypes.c_double]
    rates = {op: [] for op in range(len(PROBE_OPS))}
    with ClockSampler(0) as clk:
        for _ in range(5):
            for op in rates:
                rates[op].append(lib.sa_probe_ops_per_sm_clk(op, 1e-6))
    mhz = clk.summary()["sm_mhz"] or 2070.0
    out = {"sm_mhz": mhz, "unit": "lane-ops per SM per clock"}
    for op, name in enumerate(PROBE_OPS):
        if name in ("iadd_s32", "imax_s32"):
            continue                   # their chains are folded by the compiler: not a rate
        good = [r for r in rates[op] if r > 0]
        out[name] = round(statistics.median(good) / (mhz * 1e6), 2) if good else None
    print(json.dumps(out), flush=True)


def dpx_lane_ops_per_sm_clk(local_rank: int):
    """Measured issue rate of the packed 16-bit and the 32-bit add-max (DPX)
    instructions and of the integer multiply-add, lane-operations per SM per
    clock, from the probe library; the clock is the median SM clock sampled
    while the probe runs."""
    import ctypes
    from paper_1302_5507_gb300 import build as sa_build
    lib = ctypes.CDLL(sa_build.PROBE)
    lib.sa_probe_ops_per_sm_clk.restype = ctypes.c_double
    lib.sa_probe_ops_per_sm_clk.argtypes = [ctypes.c_int, ctypes.c_double]
    rates = {PROBE_S16X2: [], PROBE_S32: [], PROBE_IMAD: [], PROBE_MIX: []}
    with ClockSampler(local_rank) as clk:
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 1.5:
            for op in rates:
                rates[op].append(lib.sa_probe_ops_per_sm_clk(op, 1e-6))   # ops per second per SM
    mhz = clk.summary()["sm_mhz"] or 2070.0
    out = {"sm_mhz": mhz}
    for op, key in ((PROBE_S16X2, "viaddmax_s16x2"), (PROBE_S32, "viaddmax_s32"), (PROBE_IMAD, "imad_s32"),
                    (PROBE_MIX, "viaddmax_s16x2+imad")):
        good = [r for r in rates[op] if r > 0]
        out[key] = statistics.median(good) / (mhz * 1e6) if good else None
    return out


def cpu_baseline(wl, target_s: float = 8.0):
    import oracle
    nthreads = oracle.threads()
    probe = wl.subset(np.arange(min(2000, wl.n_jobs)))
    t0 = time.perf_counter()
    oracle.align(probe, n_threads=nthreads)
    rate = probe.cells / (time.perf_counter() - t0)
    n = int(min(wl.n_jobs, max(2000, target_s * rate / (wl.cells / wl.n_jobs))))
    sample = wl.subset(np.arange(n))
    t0 = time.perf_counter()
    oracle.align(sample, n_threads=nthreads)
    dt = time.perf_counter() - t0
    # one thread on a small sample (about 2 s)
    n1 = int(min(wl.n_jobs, max(50, 2.0 * rate / nthreads / (wl.cells / wl.n_jobs))))
    one = wl.subset(np.arange(n1))
    t0 = time.perf_counter()
    oracle.align(one, n_threads=1)
    dt1 = time.perf_counter() - t0
    return {"value": sample.cells / dt / 1e9, "unit": "GCUPS", "cores": nthreads, "kind": "oracle",
            "sample": f"first {n} of {wl.n_jobs} jobs ({sample.cells:.3g} cells, {dt:.1f} s, LOCAL + CIGAR)",
            "single_thread": {"value": one.cells / dt1 / 1e9, "unit": "GCUPS",
                              "sample": f"first {n1} jobs ({one.cells:.3g} cells, {dt1:.1f} s)"}}


def make_workload(config: str, rank: int, n_jobs: int, genome_len: int = 100_000_000):
    """This rank's shard of `config`: jobs rank*n_jobs .. (rank+1)*n_jobs-1 of the
    workload's stream on the shared genome (independent jobs, no exchange between
    ranks)."""
    import workloads
    if config == "c2":
        return workloads.mate_rescue(seed=1, n_pairs=n_jobs, genome_len=genome_len, first_item=rank * n_jobs)
    return workloads.uneven(seed=1, n_jobs=n_jobs, genome_len=genome_len, first_item=rank * n_jobs)


def tune_sample():
    """The autotuner's sample: 200k jobs of the uneven distribution, drawn from
    another part of its stream than the timed batch."""
    import workloads
    return workloads.uneven(seed=1, n_jobs=200_000, first_item=1 << 28)


def max_over_ranks(x: float, dist, device) -> float:
    """The largest value of `x` over all ranks (the timed region of the slowest rank)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, rank, world):
    import workloads  # noqa: F401
    if rank != 0:
        return
    config = args.config if args.config in WORKLOADS else "c3"
    wl = make_workload(config, 0, args.jobs or DEFAULT_JOBS[config])
    import oracle
    nthreads = oracle.threads()
    # each step: a bounded sample (about 2 s of oracle work), same workload and metric
    probe = wl.subset(np.arange(1000))
    t0 = time.perf_counter()
    oracle.align(probe, n_threads=nthreads)
    rate = probe.cells / (time.perf_counter() - t0)
    n = int(max(1000, 2.0 * rate / (wl.cells / wl.n_jobs)))
    times, cells = [], 0
    for step in range(args.warmup + args.steps):
        lo = step * 997 % max(1, wl.n_jobs - n)
        sub = wl.subset(np.arange(lo, lo + n))
        t0 = time.perf_counter()
        oracle.align(sub, n_threads=nthreads)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            cells += sub.cells
    value = cells / sum(times) / 1e9
    line = {"metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOADS[config], "jobs_per_step": n, "mode": "LOCAL", "scoring": "1/2/2/1",
                       "cache": "oracle on host cores"},
            "cpu_baseline": {"value": value, "unit": "GCUPS", "cores": nthreads, "kind": "oracle",
                             "sample": f"{n} consecutive jobs per step of {wl.n_jobs}"},
            "e2e": {"value": value, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def roofline_of(cells, fill_ms, packed, dpx, sm_mhz, n_sm, config, jobs):
    """Roofline of the score pass (the dominant kernel family): achieved cells per
    second over the score-pass phase, against (1) a cell-count formula, 6 DPX
    lane-ops per cell at the measured DPX rate, and (2) an issue-aware bound: the
    half-rate instructions the recurrence needs per register of cells (5.5), at the
    measured rate of add-maxima and multiply-adds interleaved (the two pipes share
    their issue)."""
    lanes = dpx["viaddmax_s16x2" if packed else "viaddmax_s32"] or 64.0
    mixed = dpx.get("viaddmax_s16x2+imad") or lanes
    cells_per_op = 2 if packed else 1
    clk = n_sm * sm_mhz * 1e6
    peak = clk * lanes * cells_per_op / OPS_PER_CELL / 1e9
    issue_peak = clk * mixed * cells_per_op / ISSUE_OPS_PER_REG / 1e9
    achieved = cells / (fill_ms / 1e3) / 1e9 if fill_ms > 0 else None
    traffic = traffic_per_step(config, jobs)
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GCUPS",
            "frac": (achieved / peak) if achieved else None, "traffic": traffic,
            "kernel": ("k_fill16 packed 16-bit score pass" if packed else "k_fill32 score pass")
                      + " (score, ends, colbest, second best), all length buckets of one step; "
                        "CUDA events around the score-pass phase on the launching stream",
            "peak_basis": f"{n_sm} SMs x {lanes:.1f} DPX lane-ops/SM/clk (measured, probe) x "
                          f"{sm_mhz:.0f} MHz (median under load) x {cells_per_op} cells per lane-op "
                          f"/ {OPS_PER_CELL} lane-ops per cell",
            "issue_aware": {"peak": issue_peak, "frac": (achieved / issue_peak) if achieved else None,
                            "basis": f"{ISSUE_OPS_PER_REG} half-rate instructions per register of {cells_per_op} "
                                     f"cell(s) (add-max G with the floor, E, F; max3 H; H + S_GO; half a "
                                     f"column maximum) at {mixed:.1f} lane-ops/SM/clk, the measured rate of "
                                     f"add-maxima and multiply-adds interleaved (ALU and FMA pipes share their "
                                     f"issue: {lanes:.1f} and {dpx.get('imad_s32') or 0:.1f} alone)"},
            "traffic_basis": "DRAM read+write bytes per step of the score-pass kernels from one ncu capture "
                             "of a smaller batch of the same workload, scaled by jobs "
                             "(profiles/score_pass_traffic.csv); null when the kernel sources changed since",
            "dpx_probe": dpx, "kernel_sources_sha1": kernel_source_sha()}


def run_ours(args, rank, world, dist):
    import torch
    import paper_1302_5507_gb300 as sa
    import __graft_entry__
    config = args.config
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    __graft_entry__.build()
    wl = make_workload(config, rank, args.jobs or DEFAULT_JOBS[config])
    jobs = sa.jobs_array(wl.read_off, wl.read_len, wl.flags, wl.ref_pos, wl.win_len)
    ref = sa.Reference(wl.ref, device=local_rank)
    # C2's scores are int32; C3 packs 16-bit pairs
    width = args.width if args.width is not None else (32 if config == "c2" else 0)
    tuned = None
    if config == "c3" and not args.no_tune:
        # the plan (configuration per read length, width per configuration) from the
        # library's autotuner on a separate sample of the same distribution
        smp = tune_sample()
        t0 = time.perf_counter()
        classes = ref.tune(sa.jobs_array(smp.read_off, smp.read_len, smp.flags, smp.ref_pos, smp.win_len),
                           smp.reads)
        plan = np.frombuffer(ref.plan()[8:], np.uint8)
        tuned = {"classes_tuned": int(classes), "seconds": time.perf_counter() - t0,
                 "sample": "200k jobs of the same distribution (another part of its stream)",
                 "cfg_of_length": {str(n): int(plan[n]) for n in (50, 100, 150, 200, 250)}}
    params = sa.make_params(width=width)                    # no phase events: the score segment replays as a graph
    params_prof = sa.make_params(width=width, profile=True)  # phase timing (CUDA events per phase)
    cap = sa.cigar_max_ops(wl.read_len)
    stream = torch.cuda.Stream(device=dev)
    d_jobs = torch.from_numpy(jobs.view(np.uint8)).to(dev)
    d_reads = torch.from_numpy(wl.reads).to(dev)
    d_out = torch.empty(len(jobs) * 56, dtype=torch.uint8, device=dev)
    d_cig = torch.empty(cap, dtype=torch.int32, device=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    # --- device-resident steps
    for _ in range(args.warmup):
        ref.align_dev(d_jobs, d_reads, d_out, d_cig, params, stream=stream)
    barrier()
    fill_ms, stats = [], None
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            ref.align_dev(d_jobs, d_reads, d_out, d_cig, params, stream=stream)
        ev1.record(stream)
        barrier()
        stats = ref.stats()
        # the same steps again with per-phase CUDA events (score-pass time for the roofline)
        step_stats = []
        for _ in range(args.steps):
            ref.align_dev(d_jobs, d_reads, d_out, d_cig, params_prof, stream=stream)
            st_ = ref.stats()
            step_stats.append(st_)
            fill_ms.append(st_["ms_fill"])
        barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist, dev)
    ms_per_step = ms / args.steps
    cells_rank = wl.cells
    cells_all = cells_rank * world
    value = cells_all * args.steps / (ms / 1e3) / 1e9
    launches = int(stats["kernel_launches"]) * args.steps

    # --- end to end from pinned host memory (sa_align_batch)
    h_jobs = torch.from_numpy(jobs.view(np.uint8)).pin_memory()
    h_reads = torch.from_numpy(wl.reads).pin_memory()
    h_out = torch.empty(len(jobs) * 56, dtype=torch.uint8).pin_memory()
    h_cig = torch.empty(cap, dtype=torch.int32).pin_memory()
    out_np = h_out.numpy().view(sa.RESULT_DTYPE)
    cig_np = h_cig.numpy().view(np.uint32)
    jobs_np = h_jobs.numpy().view(sa.JOB_DTYPE)
    reads_np = h_reads.numpy()
    e2e_params = sa.make_params(width=width)
    for _ in range(max(1, args.warmup - 1)):
        ref.align(jobs_np, reads_np, e2e_params, out=out_np, cigar=cig_np, stream=None)
    barrier()
    t0 = time.perf_counter()
    used = 0
    for _ in range(args.steps):
        _, c = ref.align(jobs_np, reads_np, e2e_params, out=out_np, cigar=cig_np, stream=None)
        used = len(c)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)
    e2e_value = cells_all * args.steps / e2e_s / 1e9

    # --- plain form on the same workload (comparison form)
    plain = None
    if not args.no_plain:
        pp = sa.make_params(form=sa.SA_FORM_PLAIN, profile=True)
        ref.align_dev(d_jobs, d_reads, d_out, d_cig, pp, stream=stream)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        nplain = max(1, min(args.steps, 2))
        for _ in range(nplain):
            ref.align_dev(d_jobs, d_reads, d_out, d_cig, pp, stream=stream)
        e1.record(stream)
        barrier()
        pms = e0.elapsed_time(e1) / nplain
        plain = {"value": cells_rank / (pms / 1e3) / 1e9, "unit": "GCUPS", "ms_per_step": pms,
                 "form": "plain: 65,536-job batches in input order, one configuration for the longest "
                         "read, one whole-window direction fill + one traceback launch each (int32)"}

    phases = {k: float(np.mean([st[k] for st in step_stats]))
              for k in ("ms_stage", "ms_fill", "ms_rerun", "ms_rect", "ms_traceback", "ms_finalize", "ms_total")}
    clocks = clk.summary()
    sm_mhz = clocks["sm_mhz"] or 2070.0
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    # roofline of the score pass: the packed 16-bit kernel when every job ran in it
    packed = int(stats["jobs16"]) == wl.n_jobs
    graph_replays = int(stats["graph_replays"])
    dpx = dpx_lane_ops_per_sm_clk(local_rank)
    fill_avg = float(np.mean(fill_ms)) if fill_ms else 0.0
    roofline = roofline_of(cells_rank, fill_avg, packed, dpx, sm_mhz, n_sm, config, wl.n_jobs)
    # the traceback's own bound: its direction data against the measured copy bandwidth
    roofline["direction_data_bound"] = direction_bound(stats, wl)

    line = None
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "s16x2" if packed else "int32",
                "data": "synthetic",
                "config": {"workload": WORKLOADS[config] + ("" if args.width is None else
                                                            f" (run at width {width or 'auto'})"),
                           "jobs_per_gpu": wl.n_jobs, "cells_per_gpu": cells_rank,
                           "mode": "LOCAL", "scoring": "match 1, mismatch 2, gap open 2, gap extend 1",
                           "width": width or "auto (16-bit pairs where no job of a bucket can overflow)",
                           "plan": "autotuned (sa_tune)" if tuned else "default",
                           "form": "batched", "cache": "inputs, lane-key scratch and direction data larger "
                                                       "than L2 (no flush)",
                           "parallelism": f"independent shards x{world}"},
                "e2e": {"value": e2e_value, "unit": "GCUPS",
                        "h2d_bytes_per_step": int(jobs.nbytes + wl.reads.nbytes),
                        "d2h_bytes_per_step": int(len(jobs) * 56 + used * 4)},
                "gpu_launches": launches,
                "score_segment_graph_replayed": bool(graph_replays),
                "overflow_reruns": int(stats["overflow_reruns"]),
                "autotune": tuned,
                "roofline": roofline,
                "clocks": clocks,
                "phases_ms": phases,
                "traceback_classes": {"diagonal": int(stats["diag_jobs"]), "band": int(stats["band_jobs"]),
                                      "rectangle": int(stats["rect_jobs"])},
                "plain_form": plain}

    # --- the mate-rescue batch (C2) at its own width (int32), 16-bit beside it
    if rank == 0 and config == "c3" and not args.no_c2:
        mate = make_workload("c2", 0, DEFAULT_JOBS["c2"])
        with sa.Reference(mate.ref, device=local_rank) as mref:
            c2 = device_line(sa, mref, mate, args, WORKLOADS["c2"], widths=(32, 0), cigar=(True,))
        r32, r16 = c2["rows"]
        line["c2_mate_rescue"] = {
            "value": r32["gcups"], "unit": "GCUPS", "dtype": "int32", "ms_per_step": r32["ms_per_step"],
            "score_pass_gcups": r32["score_pass_gcups"], "jobs": c2["jobs"], "cells": c2["cells"],
            "phases_ms": r32["phases_ms"],
            "note_s16x2": {"value": r16["gcups"], "score_pass_gcups": r16["score_pass_gcups"],
                           "ms_per_step": r16["ms_per_step"],
                           "what": "the same batch with the default width (16-bit packed pairs, exact)"},
            "timing": "CUDA events around the steps (phase events on)"}

    # --- serving latency (coalescing server), rank 0 only: a short run on this genome
    # (with the default plan, whose coarser buckets suit the server's smaller batches)
    if rank == 0 and not args.no_serving:
        import workloads
        if tuned:
            ref.set_plan(None)
        sizes, ppm = workloads.serving_arrivals(seed=3, n_requests=40)
        reqs = [workloads.serving_request(wl.ref, 3, k, int(sizes[k])) for k in range(40)]
        line["serving"] = serving_run(sa, ref, reqs, ppm, (0.8,), genome="the uneven batch's genome (100 Mbp)",
                                      slots=args.slots)
    ref.close()
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(wl)
    if rank == 0:
        print(json.dumps(line), flush=True)


def concat(reqs):
    """One workload holding the jobs of `reqs` (read offsets rebased), same reference."""
    import workloads
    off = np.cumsum([0] + [r.reads.size for r in reqs[:-1]]).astype(np.uint64)
    return workloads.Workload(
        "concat", reqs[0].ref, np.concatenate([r.reads for r in reqs]),
        np.concatenate([r.read_off + o for r, o in zip(reqs, off)]),
        np.concatenate([r.read_len for r in reqs]), np.concatenate([r.flags for r in reqs]),
        np.concatenate([r.ref_pos for r in reqs]), np.concatenate([r.win_len for r in reqs]),
        np.concatenate([r.truth for r in reqs]), dict(reqs[0].meta))


def serving_run(sa, ref, reqs, ppm, loads, genome: str, plain: bool = False, slots: int = 2,
                check: bool = False):
    """Open-loop Poisson arrivals of `reqs` at each offered load (a fraction of the
    offline batched throughput of the same jobs); p50/p99 submit -> result.
    check: every served result (all fields and the CIGAR) must equal the offline
    batched result of the same job, and a seeded sample of the offline results
    must equal the oracle's."""
    allj = concat(reqs)
    jobs_all = sa.jobs_array(allj.read_off, allj.read_len, allj.flags, allj.ref_pos, allj.win_len)
    ref.align(jobs_all, allj.reads)                       # warm-up (workspace growth)
    # median of three calls: one call from pageable host buffers varies with the host's
    # copy rate (one box measured a third of the usual rate in a single call)
    off_t = []
    for _ in range(3):
        t0 = time.perf_counter()
        off_res, off_cig = ref.align(jobs_all, allj.reads)
        off_t.append(time.perf_counter() - t0)
    offline = allj.cells / float(np.median(off_t))
    first_job = np.cumsum([0] + [r.n_jobs for r in reqs])
    out = {"requests": len(reqs), "jobs": int(allj.n_jobs), "cells": int(allj.cells), "genome": genome,
           "offline_batched_gcups": offline / 1e9,
           "offline_form": "all jobs of the requests in one sa_align_batch call (host buffers)",
           "server": f"{slots} slots; queued requests coalesce into one device batch (<= 1M jobs)",
           "poll": "one poller thread in submit order", "loads": []}
    if plain:
        pp = sa.make_params(form=sa.SA_FORM_PLAIN)
        t0 = time.perf_counter()
        ref.align(jobs_all, allj.reads, pp)
        out["plain_gcups"] = allj.cells / (time.perf_counter() - t0) / 1e9
    mean_cells = allj.cells / len(reqs)
    warm_wl = allj.subset(np.arange(min(allj.n_jobs, 1 << 20)))
    warm_jobs = sa.jobs_array(warm_wl.read_off, warm_wl.read_len, warm_wl.flags, warm_wl.ref_pos, warm_wl.win_len)
    arrays = [sa.jobs_array(r.read_off, r.read_len, r.flags, r.ref_pos, r.win_len) for r in reqs]
    import queue as _queue
    for load in loads:
        rate = load * offline / mean_cells            # requests per second
        gaps = -np.log(np.maximum(ppm.astype(np.float64), 1.0) / 1e6) / rate
        lat, done_cells = [], 0
        served = {}
        pending = _queue.Queue()
        with sa.Server(ref, sa.make_params(), max_inflight=slots) as srv:
            # warm-up: each slot runs one batch as large as a coalesced batch can get
            # (device workspace and pinned staging reach their largest size before
            # the timed arrivals)
            warm = [srv.submit(warm_jobs, warm_wl.reads) for _ in range(2)]
            for tk in warm:
                srv.poll(tk, warm_wl.n_jobs, sa.cigar_max_ops(warm_wl.read_len), timeout_ms=-1)

            def poller():
                while True:
                    item = pending.get()
                    if item is None:
                        return
                    tk, ts, r, k = item
                    _, res, cig = srv.poll(tk, r.n_jobs, sa.cigar_max_ops(r.read_len), timeout_ms=-1)
                    lat.append(time.perf_counter() - ts)
                    if check:
                        served[k] = (res, cig)
            th = threading.Thread(target=poller)
            th.start()
            t_start = time.perf_counter()
            t_next = t_start
            for k, r in enumerate(reqs):
                t_next += gaps[k]
                while time.perf_counter() < t_next:
                    time.sleep(min(0.001, max(0.0, t_next - time.perf_counter())))
                pending.put((srv.submit(arrays[k], r.reads), time.perf_counter(), r, k))
                done_cells += r.cells
            pending.put(None)
            th.join()
            wall = time.perf_counter() - t_start
            sst = srv.stats()
        lat_ms = np.array(lat) * 1e3
        row = {"offered_load": load, "p50_ms": float(np.percentile(lat_ms, 50)),
               "p99_ms": float(np.percentile(lat_ms, 99)), "gcups": done_cells / wall / 1e9,
               "server": {k: int(sst[k]) for k in ("batches", "coalesced", "admission_stalls", "max_queue")}}
        row["vs_offline"] = row["gcups"] / out["offline_batched_gcups"]
        if plain:
            row["vs_plain"] = row["gcups"] / out["plain_gcups"]
        if check:
            bad = 0
            for k, r in enumerate(reqs):
                res, cig = served[k]
                exp = off_res[first_job[k]:first_job[k + 1]]
                c0 = int(exp["cigar_off"][0]) if r.n_jobs else 0
                c1 = int(exp["cigar_off"][-1]) + int(exp["cigar_len"][-1]) if r.n_jobs else 0
                same = all((res[f] == exp[f]).all() for f in ("score", "second", "read_begin", "read_end",
                                                              "ref_begin", "ref_end", "second_ref_end",
                                                              "cigar_len", "flags"))
                same = same and (res["cigar_off"].astype(np.int64) == exp["cigar_off"].astype(np.int64) - c0).all()
                if not (same and np.array_equal(cig, off_cig[c0:c1])):
                    bad += 1
            row["served_equal_offline"] = {"requests": len(reqs), "jobs": int(allj.n_jobs), "differing_requests": bad}
        out["loads"].append(row)
    if check:
        import oracle
        from oracle.compare import compare
        rng = np.random.default_rng(2024)
        idx = np.sort(rng.choice(allj.n_jobs, min(allj.n_jobs, 4000), replace=False))
        sub = allj.subset(idx)
        ores, oops = oracle.align(sub)
        sres = off_res[idx].copy()
        parts, o = [], 0
        for k, j in enumerate(idx):
            L = int(off_res["cigar_len"][j])
            parts.append(off_cig[int(off_res["cigar_off"][j]):int(off_res["cigar_off"][j]) + L])
            sres["cigar_off"][k] = o
            o += L
        bad = compare(sres, np.concatenate(parts), ores, oops)
        out["oracle_check"] = {"jobs": len(idx), "windows_past_2^31": int((sub.ref_pos >= 2 ** 31).sum()),
                               "mismatches": len(bad), "first": bad[:3]}
    return out


def device_line(sa, ref, wl, args, label, widths=(0,), cigar=(True, False), mode=0, form=0):
    """GCUPS of one workload through sa_align_batch_dev (inputs resident), per
    (width, CIGAR) setting, with the phase times of the library's CUDA events."""
    import torch
    dev = torch.device("cuda", 0)
    jobs = sa.jobs_array(wl.read_off, wl.read_len, wl.flags, wl.ref_pos, wl.win_len)
    d_jobs = torch.from_numpy(jobs.view(np.uint8)).to(dev)
    d_reads = torch.from_numpy(wl.reads).to(dev)
    d_out = torch.empty(len(jobs) * 56, dtype=torch.uint8, device=dev)
    d_cig = torch.empty(sa.cigar_max_ops(wl.read_len), dtype=torch.int32, device=dev)
    rows = []
    for width in widths:
        for cg in cigar:
            p = sa.make_params(width=width, want_cigar=cg, profile=True, mode=mode, form=form)
            for _ in range(max(3, args.warmup)):
                ref.align_dev(d_jobs, d_reads, d_out, d_cig if cg else None, p)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            sts = []
            e0.record()
            for _ in range(args.steps):
                ref.align_dev(d_jobs, d_reads, d_out, d_cig if cg else None, p)
                sts.append(ref.stats())
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.steps
            ph = {k: float(np.mean([st[k] for st in sts])) for k in
                  ("ms_stage", "ms_fill", "ms_rerun", "ms_rect", "ms_traceback", "ms_finalize")}
            st = sts[-1]
            rows.append({"mode": "GLOCAL" if mode else "LOCAL", "form": "plain" if form else "batched",
                         "width": width or "auto", "cigar": cg, "gcups": wl.cells / (ms / 1e3) / 1e9,
                         "ms_per_step": ms, "score_pass_gcups": wl.cells / (ph["ms_fill"] / 1e3) / 1e9,
                         "phases_ms": ph, "jobs16": int(st["jobs16"]), "overflow_reruns": int(st["overflow_reruns"]),
                         "diag_jobs": int(st["diag_jobs"]), "band_jobs": int(st["band_jobs"]),
                         "rect_jobs": int(st["rect_jobs"]), "rect_pairs": int(st["rect_pairs"]),
                         "kernel_launches": int(st["kernel_launches"])})
    return {"config": label, "jobs": int(wl.n_jobs), "cells": int(wl.cells), "steps": args.steps, "rows": rows}


def hbm_peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def pairs_line(sa, ref, w, args, ceiling=30, frag=(300, 700), min_score=None):
    """One step = effort limit + alignment (with CIGAR) + paired selection, all on
    device buffers, timed with CUDA events on the stream the library runs on.
    min_score: candidates scoring below it get no traceback and count as unaligned."""
    import torch
    dev = torch.device("cuda", 0)
    st = torch.cuda.current_stream()
    jobs = sa.jobs_array(w.read_off, w.read_len, w.flags, w.ref_pos, w.win_len)
    n_jobs, n_reads = len(jobs), w.n_reads
    dj = torch.from_numpy(jobs.view(np.uint8)).to(dev)
    ds = torch.from_numpy(w.support.view(np.int32)).to(dev)
    df = torch.from_numpy(w.read_first.astype(np.uint32).view(np.int32)).to(dev)
    dr = torch.from_numpy(w.reads).to(dev)
    dk = torch.empty(n_jobs * 32, dtype=torch.uint8, device=dev)
    dfrom = torch.empty(n_jobs, dtype=torch.int32, device=dev)
    dkf = torch.empty(n_reads + 1, dtype=torch.int32, device=dev)
    dres = torch.empty(n_jobs * 56, dtype=torch.uint8, device=dev)
    dcig = torch.empty(sa.cigar_max_ops(w.read_len), dtype=torch.int32, device=dev)
    dout = torch.empty(n_reads * 32, dtype=torch.uint8, device=dev)
    params = sa.make_params(min_score=sa.SA_NO_SCORE if min_score is None else min_score)
    sel = sa.make_select_params(paired=True, frag_min=frag[0], frag_max=frag[1])

    def step(ev=None):
        if ev: ev[0].record(st)
        n = ref.effort_limit_dev(dj, ds, df, ceiling, dk, dfrom, dkf, stream=st)
        if ev: ev[1].record(st)
        ref.align_dev(dk[: n * 32], dr, dres[: n * 56], dcig, params, stream=st)
        if ev: ev[2].record(st)
        ref.select_dev(dk[: n * 32], dres[: n * 56], dkf, dout, sel, stream=st)
        if ev: ev[3].record(st)
        return n
    for _ in range(max(3, args.warmup)):
        n_kept = step()
    torch.cuda.synchronize()
    kept_np = dk[: n_kept * 32].cpu().numpy().view(sa.JOB_DTYPE)
    cells = int(np.dot(kept_np["read_len"].astype(np.int64), kept_np["win_len"].astype(np.int64)))
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(st)
    for k in range(args.steps):
        step(evs[k])
    t1.record(st)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / args.steps
    ph = {name: float(np.mean([e[i].elapsed_time(e[i + 1]) for e in evs]))
          for i, name in enumerate(("ms_effort_limit", "ms_align", "ms_select"))}
    out = dout.cpu().numpy().view(sa.READ_RESULT_DTYPE)
    peak, basis = hbm_peak()
    # algorithmic bytes: effort limit reads every candidate (job 32 B + support 4 B) and
    # writes the kept ones (job 32 B + index 4 B) and the offsets; the selection reads
    # every kept job and result (32 + 56 B) once and writes 32 B a read
    b_lim = n_jobs * 36 + n_kept * 36 + (n_reads + 1) * 12
    b_sel = n_kept * 88 + n_reads * 36
    near = np.abs(kept_np["ref_pos"][np.minimum(out["job"], n_kept - 1)].astype(np.int64) -
                  w.read_truth.astype(np.int64)) < 100
    st_align = ref.stats()
    return {"min_score": min_score, "traced_jobs": int(st_align["diag_jobs"] + st_align["band_jobs"] +
                                                       st_align["rect_jobs"]),
            "reads": n_reads, "candidates": n_jobs, "kept_jobs": n_kept, "cells": cells, "steps": args.steps,
            "ms_per_step": ms, "gcups": cells / (ms / 1e3) / 1e9, "reads_per_s": n_reads / (ms / 1e3),
            "phases_ms": ph,
            "select_roofline": {"bound": "hbm", "achieved": b_sel / (ph["ms_select"] / 1e3) / 1e9,
                                "peak": peak, "peak_basis": basis, "unit": "GB/s",
                                "frac": b_sel / (ph["ms_select"] / 1e3) / 1e9 / peak, "bytes": b_sel,
                                "note": "phase time of the sa_select_dev call (check + selection "
                                        "kernels and the status read)"},
            "effort_limit_roofline": {"bound": "hbm", "achieved": b_lim / (ph["ms_effort_limit"] / 1e3) / 1e9,
                                      "peak": peak, "unit": "GB/s",
                                      "frac": b_lim / (ph["ms_effort_limit"] / 1e3) / 1e9 / peak,
                                      "bytes": b_lim},
            "proper_fraction": float((out["flags"] & sa.SA_READ_PROPER > 0).mean()),
            "chosen_at_source_fraction": float(near.mean()),
            "mapq_hist": {str(q): int((out["mapq"] == q).sum()) for q in (0, 20, 40, 60)}}


def seeds_line(sa, args, ceiling=30, frag=(300, 700)):
    """Paired reads from sequence to placement on the device: seeds and candidate
    windows (sa_seed_candidates_dev), effort limit, alignment with CIGAR, paired
    selection.  One step = the four calls on the whole batch, timed with CUDA
    events on the library's stream; the index is built once, before."""
    import torch
    import workloads
    n_pairs = args.jobs or 100_000
    w = workloads.pairs(seed=1, n_pairs=n_pairs)
    first = w.read_first.astype(np.int64)
    off = w.read_off[first[:-1]].astype(np.uint64)
    ln = w.read_len[first[:-1]].astype(np.uint32)
    n_reads = len(ln)
    dev = torch.device("cuda", 0)
    st = torch.cuda.current_stream()
    out = {"config": f"seeds: {n_pairs} read pairs (150 bp, insert N(500,50)) on the 100 Mbp genome with "
                     f"planted segmental duplicates; seeds of 20 bases every 10 on both strands, max_occ 256, "
                     f"pad 24, join 16; effort limit {ceiling}; FR fragment {frag[0]}-{frag[1]}",
           "reads": n_reads}
    with sa.Reference(w.ref) as ref:
        t0 = time.perf_counter()
        idx = sa.SeedIndex(ref)
        out["index_build_s"] = time.perf_counter() - t0
        out["index_device_bytes"] = idx.info()["device_bytes"]
        dr = torch.from_numpy(w.reads).to(dev)
        doff = torch.from_numpy(off.view(np.int64)).to(dev)
        dln = torch.from_numpy(ln.view(np.int32)).to(dev)
        cap = 64 * n_reads
        dc = torch.empty(cap * 32, dtype=torch.uint8, device=dev)
        ds = torch.empty(cap, dtype=torch.int32, device=dev)
        df = torch.empty(n_reads + 1, dtype=torch.int32, device=dev)
        dk = torch.empty(cap * 32, dtype=torch.uint8, device=dev)
        dfrom = torch.empty(cap, dtype=torch.int32, device=dev)
        dkf = torch.empty(n_reads + 1, dtype=torch.int32, device=dev)
        dres = torch.empty(cap * 56, dtype=torch.uint8, device=dev)
        dcig = torch.empty(sa.cigar_max_ops(ln) * ceiling, dtype=torch.int32, device=dev)
        dout = torch.empty(n_reads * 32, dtype=torch.uint8, device=dev)
        params = sa.make_params()
        selp = sa.make_select_params(paired=True, frag_min=frag[0], frag_max=frag[1])

        def step(ev=None):
            if ev: ev[0].record(st)
            nc = idx.candidates_dev(dr, doff, dln, dc, ds, df, stream=st)
            if ev: ev[1].record(st)
            nk = ref.effort_limit_dev(dc[: nc * 32], ds[:nc], df, ceiling, dk, dfrom, dkf, stream=st)
            if ev: ev[2].record(st)
            ref.align_dev(dk[: nk * 32], dr, dres[: nk * 56], dcig, params, stream=st)
            if ev: ev[3].record(st)
            ref.select_dev(dk[: nk * 32], dres[: nk * 56], dkf, dout, selp, stream=st)
            if ev: ev[4].record(st)
            return nc, nk
        for _ in range(max(3, args.warmup)):
            nc, nk = step()
        torch.cuda.synchronize()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
        for k in range(args.steps):
            step(evs[k])
        torch.cuda.synchronize()
        ms = float(np.mean([e[0].elapsed_time(e[4]) for e in evs]))
        ph = {name: float(np.mean([e[i].elapsed_time(e[i + 1]) for e in evs]))
              for i, name in enumerate(("ms_seed_candidates", "ms_effort_limit", "ms_align", "ms_select"))}
        kept = dk[: nk * 32].cpu().numpy().view(sa.JOB_DTYPE)
        cells = int(np.dot(kept["read_len"].astype(np.int64), kept["win_len"].astype(np.int64)))
        got = dout.cpu().numpy().view(sa.READ_RESULT_DTYPE)
        # reads that come out near the position they were drawn from
        jobs_np = kept
        chosen = np.minimum(got["job"], max(nk - 1, 0))
        near = np.abs(jobs_np["ref_pos"][chosen].astype(np.int64) - w.read_truth.astype(np.int64)) < 200
        near &= got["job"] != sa.SA_NO_JOB
        idx.close()
    seeds_per_strand = (150 - 20) // 10 + 1
    n_seeds = n_reads * 2 * seeds_per_strand
    out.update({"steps": args.steps, "ms_per_step": ms, "reads_per_s": n_reads / (ms / 1e3),
                "gcups": cells / (ms / 1e3) / 1e9, "candidates": int(nc), "kept": int(nk), "cells": cells,
                "seeds": n_seeds, "seeds_per_s": n_seeds / (ph["ms_seed_candidates"] / 1e3),
                "phases_ms": ph,
                "proper_fraction": float((got["flags"] & sa.SA_READ_PROPER > 0).mean()),
                "placed_at_source_fraction": float(near.mean()),
                "timing": "CUDA events on the library's stream around each call (the seeding call includes "
                          "its three host synchronisations: validation, hit total, candidate total)"})
    return out


def seeds_cpu_baseline(n_pairs_sample=1000, ceiling=30, frag=(300, 700)):
    """The oracle's chain (seeding, effort limit, alignment, paired selection) on
    the first pairs of the same workload; the lambda-mer table is built first
    and not timed (as the device index is built before the timed steps)."""
    import oracle
    import workloads
    from oracle import seed as OS
    from oracle import select as S
    w = workloads.pairs(seed=1, n_pairs=100_000)
    first = w.read_first.astype(np.int64)
    off = w.read_off[first[:-1]].astype(np.uint64)[: 2 * n_pairs_sample]
    ln = w.read_len[first[:-1]].astype(np.uint32)[: 2 * n_pairs_sample]
    t0 = time.perf_counter()
    table = OS.KmerTable(w.ref, 20)
    build_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    cand, cf = OS.seed_candidates(w.ref, w.reads, off, ln, table=table, lam=20, step=10, max_occ=256, pad=24,
                                  join=16)
    t_seed = time.perf_counter() - t0
    kept, kf = S.effort_limit(cand["support"].astype(np.int64), cf.astype(np.int64), ceiling)
    sub = workloads.Workload("seeded", w.ref, w.reads, cand["read_off"][kept], cand["read_len"][kept],
                             cand["flags"][kept], cand["ref_pos"][kept], cand["win_len"][kept],
                             cand["ref_pos"][kept])
    res, _ = oracle.align(sub)
    S.select(sub.flags, sub.read_len, res, kf, paired=True, frag_min=frag[0], frag_max=frag[1])
    dt = time.perf_counter() - t0
    return {"value": len(ln) / dt, "unit": "reads/s", "cores": oracle.threads(), "kind": "oracle",
            "sample": f"first {n_pairs_sample} pairs ({len(ln)} reads, {sub.n_jobs} kept candidates, "
                      f"{dt:.1f} s, of which seeding {t_seed:.1f} s); lambda-mer table built first in "
                      f"{build_s:.1f} s (not timed)"}


def pairs_cpu_baseline(w, ceiling=30, frag=(300, 700), budget_s=10.0):
    """The oracle's effort limit, alignment and paired selection on the first pairs
    (bounded sample), GCUPS over the kept cells."""
    import oracle
    from oracle import select as S
    n_pairs = 200
    while True:
        r_hi = 2 * n_pairs
        sub_first = w.read_first[: r_hi + 1].astype(np.int64)
        t0 = time.perf_counter()
        kept, kf = S.effort_limit(w.support.astype(np.int64), sub_first, ceiling)
        sub = w.subset(kept)
        res, _ = oracle.align(sub)
        S.select(sub.flags, sub.read_len, res, kf, paired=True, frag_min=frag[0], frag_max=frag[1])
        dt = time.perf_counter() - t0
        if dt > budget_s / 4 or 2 * n_pairs > w.n_reads // 2:
            return {"value": sub.cells / dt / 1e9, "unit": "GCUPS", "cores": oracle.threads(), "kind": "oracle",
                    "sample": f"first {n_pairs} pairs ({sub.n_jobs} kept jobs, {sub.cells:.3g} cells, {dt:.1f} s)"}
        n_pairs *= 4


def run_config(args):
    """Extra measurement lines of the uneven, low-similarity and serving configurations."""
    import torch
    import paper_1302_5507_gb300 as sa
    import __graft_entry__
    import workloads
    torch.cuda.set_device(0)
    __graft_entry__.build()
    if args.config == "c1":
        wl = workloads.plain(seed=1, n_jobs=args.jobs or 10_000)
        rows = []
        with sa.Reference(wl.ref) as ref:
            for mode in (0, 1):
                for form in (1, 0):
                    # int32 scores as the configuration states, the default width beside them
                    rows += device_line(sa, ref, wl, args, "", widths=(32, 0) if form == 0 else (0,),
                                        cigar=(True,), mode=mode, form=form)["rows"]
        mate = make_workload("c2", 0, 1_000_000)
        with sa.Reference(mate.ref) as ref:
            glocal = device_line(sa, ref, mate, args, "", cigar=(True, False), mode=1)["rows"]
        line = {"config": "c1 plain: 10k windows of 400 bp, 100 bp reads (plain and batched forms, both modes)",
                "jobs": int(wl.n_jobs), "cells": int(wl.cells), "steps": args.steps, "rows": rows,
                "mate_rescue_glocal": {"jobs": int(mate.n_jobs), "cells": int(mate.cells), "rows": glocal}}
    elif args.config == "c3-detail":
        wl = workloads.uneven(seed=1, n_jobs=args.jobs or 4_000_000)
        with sa.Reference(wl.ref) as ref:
            line = device_line(sa, ref, wl, args, "c3 uneven: 4M jobs, n U[50,250], m U[1.5n,6n]",
                               widths=(0, 32), cigar=(True,))
            # the tuned plan: sa_tune on a 200k-job sample of the same distribution
            sample = workloads.uneven(seed=1, n_jobs=200_000, first_item=1 << 28)
            t0 = time.perf_counter()
            classes = ref.tune(sa.jobs_array(sample.read_off, sample.read_len, sample.flags,
                                             sample.ref_pos, sample.win_len), sample.reads)
            tune_s = time.perf_counter() - t0
            tuned = device_line(sa, ref, wl, args, "tuned", widths=(0,), cigar=(True, False))
            plan = np.frombuffer(ref.plan()[8:], np.uint8)
            line["tuned_plan"] = {"classes_tuned": classes, "tune_seconds": tune_s,
                                  "cfg_of_length": {str(n): int(plan[n]) for n in (50, 100, 150, 200, 250)},
                                  "rows": tuned["rows"]}
    elif args.config == "pairs":
        w = workloads.pairs(seed=1, n_pairs=(args.jobs or 100_000))
        with sa.Reference(w.ref) as ref:
            rows = [pairs_line(sa, ref, w, args, min_score=ms) for ms in (None, 30)]
        line = {"config": f"pairs: {w.n_reads // 2} read pairs (150 bp, insert N(500,50)), {w.n_jobs} "
                          f"candidate windows, effort limit 30, FR fragment 300-700; rows without a score "
                          f"threshold and with min_score 30 (candidates below it are not traced and count "
                          f"as unaligned)", "rows": rows}
        if not args.no_cpu:
            line["cpu_baseline"] = pairs_cpu_baseline(w)
    elif args.config == "seeds":
        line = seeds_line(sa, args)
        if not args.no_cpu:
            line["cpu_baseline"] = seeds_cpu_baseline()
    elif args.config == "c4":
        wl = workloads.lowsim(seed=1, n_jobs=args.jobs or 500_000)
        with sa.Reference(wl.ref) as ref:
            # int32 scores as the configuration states, the default width (16-bit pairs with
            # the exact rerun) beside them; score-only and with traceback for each
            line = device_line(sa, ref, wl, args,
                               "c4 low similarity: 500k jobs, n 250, m 1000, divergence 0-40%",
                               widths=(32, 0))
    else:
        ref_acgt = workloads.serving_reference(seed=1)
        n_req = 200
        sizes, ppm = workloads.serving_arrivals(seed=3, n_requests=n_req)
        reqs = [workloads.serving_request(ref_acgt, 3, k, int(sizes[k])) for k in range(n_req)]
        with sa.Reference(ref_acgt) as ref:
            line = serving_run(sa, ref, reqs, ppm, (0.5, 0.8, 0.95), slots=args.slots,
                               genome="3.1 Gbp i.i.d. reference (775 MB packed, device-resident)", plain=True,
                               check=True)
        line["config"] = "c5 serving: requests of U[1,50000] jobs, n U[50,250], m U[2n,6n]"
    line["data"] = "synthetic"
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.probe_ops:
        if rank == 0:
            probe_all_ops()
        return
    if args.config not in WORKLOADS:
        if rank == 0:
            run_config(args)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    try:
        run_ours(args, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
