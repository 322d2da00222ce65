"""The multi-rank bookkeeping of bench.py (replicas on N GPUs) on CPU with the gloo backend:
the job time is the slowest rank's and the job value adds the ranks' work."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [3.0, 7.5][rank]
        out[rank] = bench.max_over_ranks(mine, world, device="cpu")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_on_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    assert dict(out) == {0: 7.5, 1: 7.5}


def test_job_value_adds_the_replicas():
    import bench

    one = bench.job_value(6.4e6, 0.09, 1)
    assert abs(bench.job_value(6.4e6, 0.09, 4) - 4 * one) < 1e-9 * one
    assert bench.max_over_ranks(2.5, 1) == 2.5
