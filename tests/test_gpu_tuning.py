"""The native snapshot-batch tuner (tacaw_tune_multislice through the C-ABI)
on a GB300: positive timings for every candidate, the best is one of them,
and a pipeline with batch="auto" gives the same exit waves, bit for bit, as
an explicit batch (the multislice result does not depend on batching)."""

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_15599_gb300 import build
    build.build()
    from paper_2401_15599_gb300 import _lib
    return _lib.load()


def test_measure_candidates(lib):
    from paper_2401_15599_gb300 import tuning
    g = W.GridSpec(256, 256, 40.5, 40.5, 10, 2.0, 0.0, 200.0)
    timings, best = tuning.measure_multislice_batches(g, candidates=(2, 4, 8), reps=2)
    assert set(timings) == {2, 4, 8} and all(t > 0 for t in timings.values())
    assert best in timings and timings[best] == min(timings.values())


def test_auto_batch_pipeline(lib, tmp_path, monkeypatch):
    monkeypatch.setenv("TACAW_TUNE_CACHE", str(tmp_path / "tune.json"))
    from paper_2401_15599_gb300.pipeline import TimeToSpectrum
    w = W.WORKLOADS["plain_small"]
    inp = W.build_inputs(w)
    pos = torch.from_numpy(inp.positions(snapshots=list(range(48)))).cuda()
    sp = torch.from_numpy(inp.species).cuda()
    a = TimeToSpectrum(w.grid, 48, pos.shape[1], inp.amp_sigma, w.dt_fs, batch="auto")
    a.prepare(None, None)
    a.exit_waves(pos, sp)
    b = TimeToSpectrum(w.grid, 48, pos.shape[1], inp.amp_sigma, w.dt_fs, batch=5)
    b.prepare(None, None)
    b.exit_waves(pos, sp)
    torch.cuda.synchronize()
    assert a.batch in (8, 16, 32, 48)
    assert torch.equal(a.psi, b.psi)
    assert (tmp_path / "tune.json").exists()
