"""GPU parity of the natural-grid temporal transform as an FFT over time
(precision "fft32", through the C-ABI) against the FP64 oracle spectrum.

FP32 FFT rounding grows like log2(T) ulps of the spectrum's norm, well under
the 2e-5 relative-L2 bound of the spectra; the time mean is kept as a sum of
two floats (about 48 bits), so I_el agrees with the FP64 oracle to 1e-12.
"""

import numpy as np
import pytest

import oracle as O

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


@pytest.mark.parametrize("n_t,nq", [(64, 333), (128, 1000), (256, 4097), (384, 700), (512, 1024), (768, 129),
                                    (1024, 515), (2048, 257), (4096, 300)])
def test_time_fft_natural_grid(api, n_t, nq):
    rng = np.random.default_rng(n_t + 3 * nq)
    psi = _waves(rng, n_t, nq)
    inten, iel = api.spectrum(_dev(psi), 5.0, precision="fft32")
    ref, ref_el, _ = O.spectrum(psi.astype(np.complex128), 5.0)
    assert rel_l2(inten.cpu().numpy(), ref) < SPEC_TOL
    assert rel_l2(iel.cpu().numpy(), ref_el) < 1e-12      # two-float mean, about 48 bits
    # the E = 0 bin of the mean-free signal is (numerically) empty
    assert float(inten[:, n_t // 2].abs().max()) < 1e-10 * float(inten.max())


def test_time_fft_kubo_normalise_and_given_sum(api):
    rng = np.random.default_rng(51)
    psi = _waves(rng, 1024, 2000)
    d = _dev(psi)
    inten, iel = api.spectrum(d, 5.0, kubo=True, temperature_K=300.0, normalize=True, precision="fft32")
    ref, ref_el, _ = O.spectrum(psi.astype(np.complex128), 5.0, kubo=True, temperature_K=300.0, normalize=True)
    assert rel_l2(inten.cpu().numpy(), ref) < SPEC_TOL
    assert rel_l2(iel.cpu().numpy(), ref_el) < 1e-6
    s = d.to(torch.complex128).sum(dim=0)
    a, _ = api.spectrum(d, 5.0, precision="fft32")
    b, _ = api.spectrum(d, 5.0, psi_sum=s, precision="fft32")
    assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) < 1e-6


def test_time_fft_matches_gemm_paths(api):
    rng = np.random.default_rng(52)
    d = _dev(_waves(rng, 512, 3000))
    a, _ = api.spectrum(d, 5.0, precision="fft32")
    b, _ = api.spectrum(d, 5.0, precision="fp32")
    assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) < SPEC_TOL


def test_time_fft_segments(api):
    rng = np.random.default_rng(53)
    psi = _waves(rng, 1000, 600)
    inten, iel = api.spectrum_segments(_dev(psi), 5.0, 256, 128, precision="fft32")
    ref, ref_el, _ = O.segment_spectrum(psi.astype(np.complex128), 5.0, 256, 128)
    assert rel_l2(inten.cpu().numpy(), ref) < SPEC_TOL
    assert rel_l2(iel.cpu().numpy(), ref_el) < 1e-12


def test_time_fft_errors(api):
    d = _dev(_waves(np.random.default_rng(1), 100, 16))
    with pytest.raises(RuntimeError):
        api.spectrum(d, 5.0, precision="fft32")                       # T = 100 has no plan
    d = _dev(_waves(np.random.default_rng(1), 128, 16))
    with pytest.raises(RuntimeError):
        api.spectrum(d, 5.0, omega_meV=np.linspace(-10, 10, 8), precision="fft32")   # natural grid only
