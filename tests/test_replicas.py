"""Multi-GPU runs are replicas (pairs are independent units, no collective in the path): the
bench's replica arithmetic, max-over-ranks step time and whole-job throughput, checked with
two gloo ranks on the CPU."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, results):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        step_ms = [2.0, 3.5][rank]                       # rank 1 is the slow one
        results[rank] = (bench.max_over_ranks(step_ms, "cpu"),
                         bench.replica_throughput(1280 * 384 * 128, world, bench.max_over_ranks(step_ms, "cpu") * 1e-3))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_step():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        results = m.dict()
        mp.spawn(_rank_main, args=(world, port, results), nprocs=world, join=True)
        got = dict(results)
    assert got[0] == got[1]
    ms, value = got[0]
    assert ms == 3.5
    assert value == pytest.approx(2 * 1280 * 384 * 128 / 3.5e-3 / 1e9)


def test_single_process_is_the_identity():
    assert bench.max_over_ranks(1.25, "cpu") == 1.25
    assert bench.replica_throughput(1000, 1, 1e-3) == pytest.approx(1e-3)
