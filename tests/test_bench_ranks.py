"""Replica bookkeeping of bench.py on two gloo ranks (CPU): barrier, the
maximum of the timed region over ranks, the whole-job rate, and the
reference arm doing no work off rank 0."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r = bench.Ranks(world)
    r.barrier()
    ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
    out[rank] = (r.max(ms), bench.whole_job_glups(world, 1_000_000, 100, r.max(ms)))
    r.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        ms, value = out[rank]
        assert ms == 15.0
        # 2 ranks x 1e6 cells x 100 steps in 15 ms
        assert abs(value - 2 * 1e6 * 100 / 0.015 / 1e9) < 1e-9


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks(1)
    r.barrier()
    assert r.max(3.5) == 3.5
    assert abs(bench.whole_job_glups(1, 2_000_000, 10, 2.0) - 10.0) < 1e-12


def test_reference_arm_is_rank_zero_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    class A:
        workload, steps, warmup, gpus, storage = "prolate_turret", 1, 1, 2, None
    assert bench.run_reference(A()) is None
    assert capsys.readouterr().out == ""
