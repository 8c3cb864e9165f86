"""GPU parity of the QEP by-products (through the C-ABI) against the oracle:
QEP patterns of snapshot subsets, energy integrals of spectra, line and
azimuthal profiles in theta = lambda q, relative differences.  All GPU sums
are FP64, so the bounds are FP64 rounding of float32 inputs (1e-12 relative),
and bin membership and counts must match exactly.
"""

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


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to("cuda")


def _waves(rng, t, nq):
    z = 1.0 + 0.05 * (rng.standard_normal((t, nq)) + 1j * rng.standard_normal((t, nq)))
    return z.astype(np.complex64)


@pytest.mark.parametrize("t0,stride,n", [(0, 1, 0), (0, 40, 0), (7, 13, 5), (399, 1, 1)])
def test_qep_intensity(api, t0, stride, n):
    rng = np.random.default_rng(t0 + stride)
    psi = _waves(rng, 400, 1500)
    got = api.qep_intensity(_dev(psi), t0, stride, n).cpu().numpy()
    ref = O.qep_intensity(psi.astype(np.complex128), t0, stride, None if n == 0 else n)
    assert np.allclose(got, ref, rtol=1e-12, atol=0)


def test_energy_integral_of_gpu_spectrum_is_the_qep_pattern(api):
    rng = np.random.default_rng(31)
    psi = _dev(_waves(rng, 256, 3000))
    inten, iel = api.spectrum(psi, 5.0)
    got = api.energy_integral(inten, iel).cpu().numpy()
    ref = O.energy_integral(inten.cpu().numpy(), iel.cpu().numpy())
    assert np.allclose(got, ref, rtol=1e-12)
    qep = api.qep_intensity(psi).cpu().numpy()
    assert np.allclose(got, qep, rtol=2e-5)          # Parseval through the FP32 spectrum


@pytest.mark.parametrize("nx,ny,lx,ly", [(64, 64, 32.0, 32.0), (96, 40, 30.0, 11.0), (512, 512, 81.0, 81.0)])
def test_line_and_azimuthal_profiles(api, nx, ny, lx, ly):
    rng = np.random.default_rng(nx + ny)
    values = rng.random((ny, nx))
    lam = 0.025079                                   # Angstrom (200 keV), given to both sides
    line, theta = api.line_profile(_dev(values), lx, lam)
    ref_line, ref_theta = O.line_profile(values, lx, lam)
    assert np.array_equal(line.cpu().numpy(), ref_line)
    assert np.allclose(theta.cpu().numpy(), ref_theta, rtol=1e-15, atol=1e-15)
    dth, nb = 0.37, 40
    prof, counts = api.azimuthal_profile(_dev(values), lx, ly, lam, dth, nb)
    ref_prof, ref_counts = O.azimuthal_profile(values, lx, ly, lam, dth, nb)
    assert np.array_equal(counts.cpu().numpy(), ref_counts)
    assert np.allclose(prof.cpu().numpy(), ref_prof, rtol=1e-12)


def test_relative_difference(api):
    rng = np.random.default_rng(33)
    a = rng.random(1000)
    b = rng.random(1000)
    a[:3] = 0.0
    b[:3] = 0.0
    got = api.relative_difference(_dev(a), _dev(b)).cpu().numpy()
    assert np.allclose(got, O.relative_difference(a, b), rtol=1e-15, atol=0)


def test_qep_line_of_a_static_crystal(api):
    # GPU potential + multislice of a static crystal: the QEP pattern along
    # theta_y = 0 sits on the Bragg positions theta_x = lambda h / a
    from paper_2401_15599_gb300.pipeline import TimeToSpectrum
    spec = W.GridSpec(64, 64, 32.0, 32.0, 2, 4.0, 0.0, 100.0)
    cr = W.simple_cubic((8, 8, 2), 4.0)
    pos = np.repeat(cr.positions[None].astype(np.float32), 4, axis=0)
    tts = TimeToSpectrum(spec, 4, pos.shape[1], np.array([[20.0, 0.3]], np.float32), 5.0, batch=4)
    tts.prepare(None, None)
    tts.run(_dev(pos), _dev(cr.species.astype(np.int32)))
    torch.cuda.synchronize()
    qep = api.qep_intensity(tts.psi.reshape(4, -1)).reshape(64, 64)
    line, theta = api.line_profile(qep, 32.0, 0.037014)
    line = line.cpu().numpy()
    k = np.arange(64) - 32
    assert np.max(line[(k % 8) != 0]) < 1e-9 * np.max(line)
    assert np.all(line[np.isin(k, [-16, -8, 0, 8, 16])] > 1e-8 * np.max(line))


def test_errors(api):
    psi = _dev(_waves(np.random.default_rng(1), 10, 8))
    with pytest.raises(RuntimeError):
        api.qep_intensity(psi, 0, 3, 5)              # only 4 snapshots every 3rd
    with pytest.raises(RuntimeError):
        api.qep_intensity(psi, 10, 1, 0)             # t0 beyond the trajectory
