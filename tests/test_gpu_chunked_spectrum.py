"""Time-chunked spectra against the FP64 oracle.

tacaw_spectrum_accumulate sums the transform of (psi - m_ref) chunk by chunk
and tacaw_spectrum_finish removes (m - m_ref) S(E) in FP64, so the result must
be the plain spectrum of the whole trajectory (Eq. (9) with the elastic part
removed), whatever the chunks and the reference mean: here the mean of the
first chunk (a trajectory that is never resident at once) or the exact mean
(the sharded form, where the mean is all-reduced first).  Bound: relative L2
of I(q, E) below 2e-5 (FP32 SIMT and three-term split BF16), per 50 meV band
on exit-wave-like series with strong beams.
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


def _chunked(api, z, dt, omega, chunks, precision, exact_mean=False, **kw):
    psi = torch.from_numpy(z).cuda()
    n_t, nq = psi.shape
    psum = torch.zeros(nq, dtype=torch.complex128, device="cuda")
    psum += psi.to(torch.complex128).sum(0)          # the running sum the multislice keeps (test input)
    phi = torch.zeros((nq, len(omega)), dtype=torch.complex64, device="cuda")
    if exact_mean:
        m_ref = api.time_mean(psum, n_t)
    else:
        first = torch.zeros(nq, dtype=torch.complex128, device="cuda")
        first += psi[: chunks[0]].to(torch.complex128).sum(0)
        m_ref = api.time_mean(first, chunks[0])
    t0 = 0
    for c in chunks:
        api.spectrum_accumulate(psi[t0:t0 + c], t0, dt, omega, m_ref, phi, precision=precision)
        t0 += c
    assert t0 == n_t
    inten, iel = api.spectrum_finish(phi, n_t, dt, omega, m_ref, psum, **kw)
    api.status()
    return inten.cpu().numpy().astype(np.float64), iel.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp32", "bf16x6"])
@pytest.mark.parametrize("exact_mean", [False, True])
def test_chunked_equals_whole_trajectory(api, precision, exact_mean):
    rng = np.random.default_rng(17)
    n_t, nq = 300, 777
    z = (1.0 + 0.05 * (rng.standard_normal((n_t, nq)) + 1j * rng.standard_normal((n_t, nq)))).astype(np.complex64)
    z += (0.3 * np.exp(1j * rng.uniform(0, 2 * np.pi, nq))).astype(np.complex64)
    omega = np.linspace(-150.0, 150.0, 256, endpoint=False)
    got, got_el = _chunked(api, z, 5.0, omega, [64, 100, 136], precision, exact_mean)
    ref, ref_el, _ = O.spectrum(z.astype(np.complex128), 5.0, omega)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < SPEC_TOL
    assert np.linalg.norm(got_el - ref_el) / np.linalg.norm(ref_el) < 1e-12


def test_chunked_natural_grid_kubo_normalize(api):
    rng = np.random.default_rng(23)
    n_t, nq = 256, 300
    z = (1.0 + 0.05 * (rng.standard_normal((n_t, nq)) + 1j * rng.standard_normal((n_t, nq)))).astype(np.complex64)
    e = O.natural_energies(n_t, 5.0)
    got, got_el = _chunked(api, z, 5.0, e, [32] * 8, "fp32", kubo=True, temperature_K=300.0, normalize=True)
    ref, ref_el, _ = O.spectrum(z.astype(np.complex128), 5.0, kubo=True, temperature_K=300.0, normalize=True)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < SPEC_TOL
    assert np.linalg.norm(got_el - ref_el) / np.linalg.norm(ref_el) < 1e-6
    assert abs(got.sum() + got_el.sum() - 1.0) < 1e-5


@pytest.mark.parametrize("precision", ["bf16x6", "fp32"])
def test_chunked_per_band_on_strong_beams(api, precision):
    # seeded exit-wave-like series (4096 snapshots, strong beams with weak phase
    # modulation): eight chunks of 512, reference mean from the first chunk
    z = W.modulated_waves(4096, 1024, 5.0, n_strong=48, seed=77)
    omega = np.arange(1024) * (400.0 / 1024) - 200.0
    got, got_el = _chunked(api, z, 5.0, omega, [512] * 8, precision)
    ref, ref_el, _ = O.spectrum(z.astype(np.complex128), 5.0, omega)
    rows = []
    for lo in range(-200, 200, 50):
        sel = (omega >= lo) & (omega < lo + 50)
        rows.append(np.linalg.norm(got[:, sel] - ref[:, sel]) / np.linalg.norm(ref[:, sel]))
    print(f"\nchunked {precision}: per band " + ", ".join(f"{x:.2e}" for x in rows))
    assert max(rows) < SPEC_TOL
    assert np.linalg.norm(got_el - ref_el) / np.linalg.norm(ref_el) < 1e-12


def test_accumulate_argument_errors(api):
    from paper_2401_15599_gb300 import _lib as L
    psi = torch.zeros((4, 8), dtype=torch.complex64, device="cuda")
    phi = torch.zeros((8, 16), dtype=torch.complex64, device="cuda")
    m = torch.zeros(8, dtype=torch.complex128, device="cuda")
    with pytest.raises(L.TacawError) as exc:
        api.spectrum_accumulate(psi, -1, 5.0, np.zeros(16), m, phi)
    assert exc.value.code == L.TACAW_EINVAL
    with pytest.raises(ValueError):
        api.spectrum_accumulate(psi, 0, 5.0, np.zeros(15), m, phi)
