"""The device trajectory synthesiser (used where a workload's positions do
not fit in memory for every snapshot at once) gives the numpy generator's
positions: same modes, same expansion (CPU)."""

import numpy as np

import workloads as W


def _close(a, b):
    """Within two float32 ulps of the coordinate (the FP32 mode sum and the
    final rounding) plus 1e-6 A."""
    return np.all(np.abs(a - b) <= 2 * np.spacing(np.abs(a)) + 1e-6)


def test_synth_matches_numpy_positions():
    for name in ("plain_small", "differentiation"):
        w = W.WORKLOADS[name].with_(n_t=40)
        inp = W.build_inputs(w)
        synth = inp.synth("cpu")
        for t0, t1 in ((0, 1), (0, 8), (7, 40)):
            a = inp.positions(list(range(t0, t1)))
            b = synth(t0, t1).numpy()
            assert a.shape == b.shape and a.dtype == b.dtype
            assert _close(a, b)


def test_synth_of_a_batched_job_into_a_buffer():
    import torch
    w = W.batching_jobs(n_jobs=3)[2].with_(n_t=16)
    inp = W.build_inputs(w)
    out = torch.empty((8, inp.crystal.n_atoms, 3), dtype=torch.float32)
    got = inp.synth("cpu")(8, 16, out=out)
    assert got is out
    assert _close(inp.positions(list(range(8, 16))), out.numpy())
