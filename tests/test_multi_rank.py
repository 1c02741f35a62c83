"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas, one stream per rank)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_info() == (rank, rank, world)
        # rank r measured (10 + r) ms for its steps and (1 + 3 r) s end to end
        got = bench.max_over_ranks([10.0 + rank, 1.0 + 3.0 * rank], "cpu")
        out.put((rank, got, bench.job_throughput(200, world, got[0])))
        # the reference arm: only rank 0 runs (and prints) it; other ranks return at once
        if rank != 0:
            assert bench.run_reference(type("A", (), {"steps": 1, "warmup": 0})()) is None
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_sum_the_frames():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(out.get(timeout=5) for _ in range(2))
    for rank, got, value in res:
        assert got == [11.0, 4.0]                       # max over ranks, on every rank
        assert value == pytest.approx(400 / 11e-3)      # both ranks' frames over the slowest time


def test_single_process_reduction_is_the_identity():
    assert not dist.is_initialized()
    assert bench.max_over_ranks([3.0, 5.0], "cpu") == [3.0, 5.0]
    assert bench.job_throughput(100, 1, 50.0) == pytest.approx(2000.0)
