"""The multi-GPU bench path runs independent replicas (no data-path
collective); its only exchange is the all-reduce MAX of the ranks' times.
Checked here with two gloo ranks on the CPU: every rank gets the slowest
rank's times and the whole-job throughput counts all ranks' edges."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

EDGES, STEPS = 2_135_630_032, 20


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = bench.aggregate_replicas(100.0 + 50.0 * rank, 120.0 + 10.0 * rank, EDGES, STEPS, world,
                                       torch.device("cpu"))
        out[rank] = torch.tensor(res, dtype=torch.float64)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replicas_take_the_slowest_rank(world):
    out = torch.zeros((world, 4), dtype=torch.float64).share_memory_()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    ms, e2e = 100.0 + 50.0 * (world - 1), 120.0 + 10.0 * (world - 1)
    want = torch.tensor([ms, e2e, world * EDGES * STEPS / (ms / 1e3) / 1e9,
                         world * EDGES * STEPS / (e2e / 1e3) / 1e9], dtype=torch.float64)
    for r in range(world):
        assert torch.allclose(out[r], want, rtol=0, atol=1e-9)


def test_single_replica_needs_no_process_group():
    import bench
    ms, e2e, v, ve = bench.aggregate_replicas(10.0, 12.0, EDGES, STEPS, 1, torch.device("cpu"))
    assert (ms, e2e) == (10.0, 12.0)
    assert v == EDGES * STEPS / 0.01 / 1e9 and ve == EDGES * STEPS / 0.012 / 1e9
