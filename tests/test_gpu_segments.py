"""GPU parity of spectra averaged over sets of consecutive snapshots
(tacaw_spectrum_segments, through the C-ABI) against the FP64 oracle.

Same bound as the single-trajectory spectrum: relative L2 below 2e-5 on
I(q, E); the FP64 set sums of the elastic part agree to 1e-12.
"""

import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPEC_TOL = 2e-5


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_15599_gb300 import build
    build.build()
    from paper_2401_15599_gb300 import api as A
    return A


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _waves(rng, t, nq):
    z = 1.0 + 0.05 * (rng.standard_normal((t, nq)) + 1j * rng.standard_normal((t, nq)))
    return z.astype(np.complex64)


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to("cuda")


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
@pytest.mark.parametrize("n_t,nq,seg,hop,n_sets", [(256, 2048, 64, 32, 0), (200, 777, 50, 25, 0),
                                                    (97, 300, 33, 16, 3), (64, 129, 64, 5, 0)])
def test_segments_natural_grid(api, precision, n_t, nq, seg, hop, n_sets):
    rng = np.random.default_rng(n_t * 7 + nq)
    psi = _waves(rng, n_t, nq)
    inten, iel = api.spectrum_segments(_dev(psi), 5.0, seg, hop, n_sets=n_sets, precision=precision)
    ref, ref_el, _ = O.segment_spectrum(psi.astype(np.complex128), 5.0, seg, hop,
                                        n_sets=None if n_sets == 0 else n_sets)
    assert inten.shape == (nq, seg)
    assert rel_l2(inten.cpu().numpy(), ref) < SPEC_TOL
    assert rel_l2(iel.cpu().numpy(), ref_el) < 1e-12


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_segments_explicit_grid_kubo_normalise(api, precision):
    rng = np.random.default_rng(21)
    n_t, nq, seg, hop = 300, 513, 100, 50           # the paper's Si averaging shape (5 sets here)
    psi = _waves(rng, n_t, nq)
    omega = np.linspace(-200.0, 200.0, 256, endpoint=False)
    inten, iel = api.spectrum_segments(_dev(psi), 25.0, seg, hop, omega_meV=omega, kubo=True,
                                       temperature_K=300.0, normalize=True, precision=precision)
    ref, ref_el, _ = O.segment_spectrum(psi.astype(np.complex128), 25.0, seg, hop, omega_meV=omega,
                                        kubo=True, temperature_K=300.0, normalize=True)
    assert rel_l2(inten.cpu().numpy(), ref) < SPEC_TOL
    assert rel_l2(iel.cpu().numpy(), ref_el) < 1e-6
    assert float(inten.double().sum() + iel.sum()) == pytest.approx(1.0, abs=1e-6)


def test_segments_one_set_equals_spectrum(api):
    rng = np.random.default_rng(22)
    psi = _dev(_waves(rng, 128, 1000))
    a, ael = api.spectrum_segments(psi, 5.0, 128, 1)
    b, bel = api.spectrum(psi, 5.0)
    assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) < 1e-7
    assert torch.equal(ael, bel)


def test_segments_exit_waves_of_a_trajectory(api):
    # exit waves of the seeded simple-cubic trajectory (GPU potential + multislice),
    # averaged over sets of 64 snapshots offset by 32
    from paper_2401_15599_gb300.pipeline import TimeToSpectrum
    w = W.WORKLOADS["plain_small"]
    inp = W.build_inputs(w)
    pos = inp.positions()
    tts = TimeToSpectrum(w.grid, pos.shape[0], pos.shape[1], inp.amp_sigma, w.dt_fs, batch=64)
    tts.prepare(None, None)
    tts.run(_dev(pos), _dev(inp.species))
    torch.cuda.synchronize()
    psi = tts.psi.reshape(pos.shape[0], -1)
    inten, iel = api.spectrum_segments(psi, w.dt_fs, 64, 32)
    ref, ref_el, _ = O.segment_spectrum(psi.cpu().numpy().astype(np.complex128), w.dt_fs, 64, 32)
    assert rel_l2(inten.cpu().numpy(), ref) < SPEC_TOL
    assert rel_l2(iel.cpu().numpy(), ref_el) < 1e-12


def test_segments_errors(api):
    psi = _dev(_waves(np.random.default_rng(1), 32, 16))
    with pytest.raises(RuntimeError):
        api.spectrum_segments(psi, 5.0, 40, 8)               # set longer than the trajectory
    with pytest.raises(RuntimeError):
        api.spectrum_segments(psi, 5.0, 16, 8, n_sets=4)     # only 3 sets fit
    with pytest.raises(RuntimeError):
        api.spectrum_segments(psi, 5.0, 16, 0)               # hop must be positive
