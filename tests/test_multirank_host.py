"""Multi-rank host logic of the benchmark on CPU with the gloo backend
(world_size 2): each rank solves its own field (weak scaling, no data-path
collective); only the timing is reduced, by the maximum over ranks."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local_ms = [12.5, 20.0][rank]
        mx = bench.max_over_ranks(local_ms, world, device="cpu")
        val = bench.weak_scaling_value(world, 256 ** 3, 10, mx / 1e3)
        seeds = [bench.field_seed(2409, rank, 2, f) for f in range(2)]
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)
        q.put((rank, mx, val, gathered))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_rank_max_time_weak_value_and_distinct_fields():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=100) for _ in range(world)]
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, mx, val, gathered in res:
        assert mx == 20.0  # the slowest rank's time, on every rank
        assert val == pytest.approx(2 * 256 ** 3 * 10 / 0.020)
        flat = [s for seeds in gathered for s in seeds]
        assert len(set(flat)) == 4  # every rank's fields differ


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.weak_scaling_value(1, 100, 5, 2.0) == 250.0
