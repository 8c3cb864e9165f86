"""Host logic of the benchmark's multi-rank path, on the CPU: two `gloo` ranks
(one process each, rendezvous on 127.0.0.1) agree on the slowest rank's step
time, and the whole-job throughput counts the units of every rank.  One rank,
or no process group, returns the local time unchanged.  The workload override
used for small ncu captures keeps the crystal filling the slices."""

import math
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench.dist_env()[:2] == (rank, world)
        ms = bench.max_over_ranks(times[rank], "cpu")
        out[rank] = (ms, bench.aggregate_rate(1000.0, world, ms))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    world, times = 2, [12.5, 40.0]
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), times, out), nprocs=world, join=True)
    for r in range(world):
        ms, rate = out[r]
        assert ms == 40.0
        assert rate == pytest.approx(1000.0 * world / 40e-3)


def test_single_process_keeps_its_own_time():
    assert not dist.is_initialized()
    assert bench.max_over_ranks(7.25, "cpu") == 7.25
    assert bench.aggregate_rate(500.0, 1, 2.0) == pytest.approx(250000.0)


def test_slice_override_keeps_the_crystal_filling_the_slices():
    class A:
        workload, snapshots, slices = "paper_scale", 64, 12
    w = bench.workload(A)
    assert (w.grid.n_slices, w.n_t) == (12, 64)
    nz = w.ncell[2]
    assert nz == math.ceil(12 * w.grid.dz / w.a) and (nz - 1) * w.a < 12 * w.grid.dz <= nz * w.a
    assert w.ncell[:2] == (20, 20) and w.n_lo[2] == -(nz // 2) and w.n_hi[2] == nz // 2
