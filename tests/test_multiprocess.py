"""The N-GPU bench path on CPU ranks (gloo, world size 2): each rank takes its
own shard of jobs (no exchange), the timed region is the maximum over ranks, and
the whole-job value counts every rank's cells."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        wl = bench.make_workload("c3", rank, 300, genome_len=2_000_000)
        # each rank's own (fake) timed region; the reported one is the slowest
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist, "cpu")
        out[rank] = (wl.truth.copy(), int(wl.cells), ms)
    finally:
        dist.destroy_process_group()


def test_two_rank_shards_and_max_reduce():
    world, port = 2, _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn")
    truth0, cells0, ms0 = out[0]
    truth1, cells1, ms1 = out[1]
    # shards are disjoint job streams of the same distribution
    assert len(truth0) == len(truth1) == 300
    assert not np.array_equal(truth0, truth1)
    assert len(set(truth0.tolist()) & set(truth1.tolist())) < 5
    # every rank reports the slowest rank's time
    assert ms0 == ms1 == 15.0
    assert abs(cells0 - cells1) / cells0 < 0.2


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    called = []
    monkeypatch.setattr(bench, "make_workload", lambda *a, **k: called.append(a) or None)
    args = type("A", (), {"jobs": 10, "steps": 1, "warmup": 0, "gpus": 2})()
    bench.run_reference(args, rank=1, world=2)
    assert called == [] and capsys.readouterr().out == ""
