"""World-size-2 test of the multi-rank (replicas) bookkeeping on CPU with gloo."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1511_04292_gb300 import replicas
    assert replicas.world() == (rank, world)
    replicas.barrier()
    # rank r "took" 100 (r + 1) ms for 1e9 (r + 1) updates
    g, mx, n = replicas.throughput(100.0 * (rank + 1), 1e9 * (rank + 1))
    out[rank] = (g, mx, n)
    replicas.barrier()
    dist.destroy_process_group()


def test_throughput_is_total_work_over_slowest_rank():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        g, mx, n = out[r]
        assert n == 2 and mx == 200.0
        assert abs(g - 3e9 / 0.2 / 1e9) < 1e-9


def test_single_process_is_identity():
    from paper_1511_04292_gb300 import replicas
    if dist.is_initialized():
        pytest.skip("process group already initialised")
    assert replicas.throughput(50.0, 5e9) == (100.0, 50.0, 1)
