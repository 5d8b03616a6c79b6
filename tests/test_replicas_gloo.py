"""Multi-GPU runs are replicas (each rank reconstructs its own realisation;
the path has no exchange step).  The host logic that turns per-rank timings
into the benchmark's whole-job number -- the barrier, the max over ranks and
the aggregate throughput -- runs here on CPU with the gloo backend,
world size 2."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 150.0][rank]
    dist.barrier()
    ms = bench.max_over_ranks(local_ms, dist, "cpu")
    value = bench.whole_job_throughput(1000, 4, world, ms)
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_two_rank_max_and_aggregate():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    assert out[0][0] == out[1][0] == 150.0
    # 2 ranks x 1000 units x 4 steps in 0.150 s
    assert out[0][1] == pytest.approx(2 * 1000 * 4 / 0.150)
    assert out[0][1] == out[1][1]


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.whole_job_throughput(10, 2, 1, 20.0) == pytest.approx(1000.0)
