"""Multi-process host logic of bench.py on CPU (gloo, world size 2): the
replicas' timing reduction takes the slowest rank and the whole-job rate
counts every replica's pixels.  Rendering has no exchange step, so this is
the only cross-rank logic of the path."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [12.5, 40.0][rank]
    got = bench.max_over_ranks(local, world, torch.device("cpu"))
    rate = bench.whole_job_mpix_s(1024 * 1024, 20, world, got)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got, rate))


def test_two_rank_timing_reduction():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, rate in out:
        assert got == 40.0
        assert rate == pytest.approx(2 * 1024 * 1024 * 20 / 0.040 / 1e6)


def test_single_rank_is_identity():
    assert bench.max_over_ranks(3.25, 1, torch.device("cpu")) == 3.25
    assert bench.whole_job_mpix_s(100, 10, 1, 1000.0) == pytest.approx(100 * 10 / 1.0 / 1e6)
