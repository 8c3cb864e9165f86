"""The whole path in one library call with host buffers
(tacaw_time_to_spectrum_host): positions in host memory -> I(q, E) and I_el in
host memory.  Same kernels and batches as the device-input pipeline, so the
results are bit-identical to it, and within the spectrum bound of the FP64
oracle; page-locked and pageable host memory both work, and back-to-back calls
into the same host buffers give the same bits."""

import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_15599_gb300 import build
    build.build()
    from paper_2401_15599_gb300 import api as A
    return A


@pytest.mark.parametrize("precision", ["fft32", "bf16x6"])
def test_host_path_matches_device_pipeline_and_oracle(api, precision):
    from paper_2401_15599_gb300.pipeline import TimeToSpectrum
    w = W.WORKLOADS["plain_small"].with_(n_t=64)
    inp = W.build_inputs(w)
    pos = inp.positions()
    sp = torch.from_numpy(inp.species).cuda()
    tts = TimeToSpectrum(w.grid, w.n_t, pos.shape[1], inp.amp_sigma, w.dt_fs, batch=24, precision=precision)
    tts.prepare(None, None)
    ref_i, ref_el = tts.run(torch.from_numpy(pos).cuda(), sp)
    pinned = torch.from_numpy(pos).pin_memory()
    ws = api.time_to_spectrum_host_workspace(w.grid, w.n_t, pos.shape[1], 24, precision)
    out, out_el = api.time_to_spectrum_host(w.grid, pinned, sp, inp.amp_sigma, w.dt_fs, 24, precision=precision,
                                            workspace=ws)
    torch.cuda.synchronize()
    api.status()
    assert torch.equal(out, ref_i.cpu()) and torch.equal(out_el, ref_el.cpu())
    out2, out_el2 = api.time_to_spectrum_host(w.grid, torch.from_numpy(pos), sp, inp.amp_sigma, w.dt_fs, 24,
                                              precision=precision, out=out.clone(), out_el=out_el.clone())
    torch.cuda.synchronize()
    assert torch.equal(out2, out) and torch.equal(out_el2, out_el)
    g = O.grid_from_spec(w.grid)
    psi = O.exit_waves(g, pos.astype(np.float64), inp.species, inp.amp_sigma.astype(np.float64))
    ref, ref_e, _ = O.spectrum(psi, w.dt_fs)
    assert np.linalg.norm(out.numpy() - ref) / np.linalg.norm(ref) < 2e-5
    assert np.linalg.norm(out_el.numpy() - ref_e) / np.linalg.norm(ref_e) < 1e-6


def test_host_path_with_the_work_queue(api):
    """ms_flags = TACAW_MS_QUEUE: the one-call path runs each batch through the
    work-queue multislice; the spectrum equals the per-slice path's bit for bit."""
    from paper_2401_15599_gb300 import _lib as L
    w = W.WORKLOADS["plain_small"].with_(n_t=64)
    inp = W.build_inputs(w)
    pos = torch.from_numpy(inp.positions())
    sp = torch.from_numpy(inp.species).cuda()
    a, a_el = api.time_to_spectrum_host(w.grid, pos, sp, inp.amp_sigma, w.dt_fs, 24, precision="fft32")
    b, b_el = api.time_to_spectrum_host(w.grid, pos, sp, inp.amp_sigma, w.dt_fs, 24, ms_flags=L.TACAW_MS_QUEUE,
                                        precision="fft32")
    torch.cuda.synchronize()
    api.status()
    assert torch.equal(a, b) and torch.equal(a_el, b_el)
