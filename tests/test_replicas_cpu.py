"""Multi-rank host logic of bench.py (replicas, max-over-ranks timing) with
two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    try:
        ws, r, _ = bench.dist_env()
        assert (ws, r) == (world, rank)
        slowest = bench.reduce_max(1.5 + rank, "cpu")          # rank 1 is slower
        rate = bench.whole_job_rate(ws, 1000.0, slowest)
        dist.barrier()
        out.put((rank, slowest, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_slowest_and_sum_units():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate in res:
        assert slowest == 2.5
        assert rate == pytest.approx(2 * 1000.0 / 2.5)


def test_single_process_reduce_is_identity():
    import bench
    assert bench.reduce_max(3.25, "cpu") == 3.25
    assert bench.whole_job_rate(1, 10.0, 2.0) == 5.0
