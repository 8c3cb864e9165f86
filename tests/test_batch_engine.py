"""The batched driver's default multislice engine (host logic, CPU): the work
queue for square grids from windows of QUEUE_MIN_WINDOW snapshots, per-slice
batch launches otherwise (non-square grids, or windows so small that a slice
of the queue has fewer items than its launch has blocks)."""

import workloads as W
from paper_2401_15599_gb300.batch import QUEUE_MIN_WINDOW, queue_by_default


def _grid(nx, ny):
    return W.GridSpec(nx, ny, nx * 0.158, ny * 0.158, 4, 2.0, 0.0, 200.0)


def test_square_grids_take_the_queue_from_the_minimum_window():
    grids = [_grid(128, 128), _grid(768, 768), _grid(512, 512)]
    assert queue_by_default(grids, QUEUE_MIN_WINDOW)
    assert queue_by_default(grids, 512)
    assert not queue_by_default(grids, QUEUE_MIN_WINDOW - 1)
    assert not queue_by_default(grids, 8)


def test_a_non_square_grid_takes_per_slice_launches():
    grids = [_grid(256, 256), _grid(512, 256)]
    assert not queue_by_default(grids, 512)
