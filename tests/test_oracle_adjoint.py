"""Pins of the FP64 oracle adjoint: every stage against central finite
differences of the oracle's forward, and the full chain (loss -> spectrum ->
multislice -> potential) against finite differences in the per-species
amplitude and width."""

import numpy as np
import pytest

import oracle as O
import oracle.adjoint as A


def _grid(nx=12, ny=10, lx=6.0, ly=5.0, n_slices=3, dz=2.0, z0=0.0, kev=100.0):
    return O.Grid(nx, ny, lx, ly, n_slices, dz, z0, kev, 2.0 / 3.0)


def _fd(f, x, h):
    return (f(x + h) - f(x - h)) / (2 * h)


@pytest.mark.parametrize("n_t,omega", [(8, None), (9, None), (8, np.array([-50.0, -3.0, 0.0, 7.5, 120.0]))])
def test_spectrum_backward_finite_differences(n_t, omega):
    rng = np.random.default_rng(n_t)
    nq = 3
    psi = 1 + 0.1 * (rng.standard_normal((n_t, nq)) + 1j * rng.standard_normal((n_t, nq)))
    n_w = n_t if omega is None else len(omega)
    dl_di = rng.standard_normal((nq, n_w))

    def loss(p):
        inten, _, _ = O.spectrum(p, 5.0, omega)
        return float(np.sum(dl_di * inten))

    g = A.spectrum_backward(psi, 5.0, dl_di, omega)
    for (n, q) in [(0, 0), (n_t - 1, 2), (n_t // 2, 1)]:
        e = np.zeros_like(psi)
        e[n, q] = 1.0
        d_re = _fd(lambda h: loss(psi + h * e), 0.0, 1e-6)
        d_im = _fd(lambda h: loss(psi + 1j * h * e), 0.0, 1e-6)
        assert g[n, q].real == pytest.approx(d_re, rel=1e-6, abs=1e-9)
        assert g[n, q].imag == pytest.approx(d_im, rel=1e-6, abs=1e-9)


def test_multislice_backward_finite_differences():
    rng = np.random.default_rng(3)
    g = _grid()
    v = rng.uniform(0.0, 40.0, (g.n_slices, g.ny, g.nx))
    psi_in = 1 + 0.2 * (rng.standard_normal((g.ny, g.nx)) + 1j * rng.standard_normal((g.ny, g.nx)))
    g_exit = rng.standard_normal((g.ny, g.nx)) + 1j * rng.standard_normal((g.ny, g.nx))

    def lin(vv, pin):
        return float(np.real(np.sum(np.conj(g_exit) * O.multislice(g, vv, pin))))

    g_v, g_psi = A.multislice_backward(g, v, g_exit, psi_in)
    for (s, j, i) in [(0, 0, 0), (1, 3, 7), (2, 9, 11), (2, 4, 5)]:
        e = np.zeros_like(v)
        e[s, j, i] = 1.0
        d = _fd(lambda h: lin(v + h * e, psi_in), 0.0, 1e-4)
        assert g_v[s, j, i] == pytest.approx(d, rel=1e-6, abs=1e-12)
    for (j, i) in [(0, 0), (5, 6)]:
        e = np.zeros((g.ny, g.nx))
        e[j, i] = 1.0
        d_re = _fd(lambda h: lin(v, psi_in + h * e), 0.0, 1e-6)
        d_im = _fd(lambda h: lin(v, psi_in + 1j * h * e), 0.0, 1e-6)
        assert g_psi[j, i].real == pytest.approx(d_re, rel=1e-6, abs=1e-12)
        assert g_psi[j, i].imag == pytest.approx(d_im, rel=1e-6, abs=1e-12)


def test_potential_backward_finite_differences():
    rng = np.random.default_rng(4)
    g = _grid(nx=40, ny=36, lx=8.0, ly=7.2, n_slices=4, dz=1.5, z0=0.3)
    n = 9
    pos = np.stack([rng.uniform(0, g.lx, n), rng.uniform(0, g.ly, n), rng.uniform(-0.5, 6.5, n)], axis=1)
    species = rng.integers(0, 2, n)
    amp_sigma = np.array([[20.0, 0.3], [12.0, 0.45]])
    g_v = rng.standard_normal((g.n_slices, g.ny, g.nx))

    def lin(asg):
        return float(np.sum(g_v * O.projected_potential(g, pos, species, asg)))

    grad = A.potential_backward(g, pos, species, amp_sigma, g_v)
    for sp in range(2):
        for c, h in ((0, 1e-4), (1, 1e-7)):
            e = np.zeros_like(amp_sigma)
            e[sp, c] = 1.0
            d = _fd(lambda hh: lin(amp_sigma + hh * e), 0.0, h)
            assert grad[sp, c] == pytest.approx(d, rel=2e-6, abs=1e-9)


def test_full_chain_gradient_of_fitting_loss():
    # loss between spectra of the same trajectory with amplitudes scaled by 1.05
    rng = np.random.default_rng(5)
    g = _grid(nx=16, ny=16, lx=8.0, ly=8.0, n_slices=2, dz=4.0, kev=200.0)
    n_t, dt = 8, 5.0
    base = np.array([[2.0, 2.0, 1.0], [6.0, 2.0, 5.0], [2.0, 6.0, 5.0], [6.0, 6.0, 1.0]])
    pos = base[None] + 0.15 * rng.standard_normal((n_t, 4, 3))
    species = np.array([0, 1, 0, 1])
    amp_sigma = np.array([[20.0, 0.35], [14.0, 0.4]])

    def spectra(asg):
        psi = O.exit_waves(g, pos, species, asg)
        inten, _, e = O.spectrum(psi, dt)
        return psi, inten, e

    _, target, e = spectra(amp_sigma * np.array([[1.05, 1.0]]))
    w = A.loss_weights(g, n_t, e)

    def total(asg):
        return A.loss(spectra(asg)[1], target, w)

    psi, inten, _ = spectra(amp_sigma)
    dl_di = A.loss_grad(inten, target, w)
    g_psi = A.spectrum_backward(psi, dt, dl_di).reshape(n_t, g.ny, g.nx)
    grad = np.zeros_like(amp_sigma)
    for t in range(n_t):
        v = O.projected_potential(g, pos[t], species, amp_sigma)
        g_v, _ = A.multislice_backward(g, v, g_psi[t])
        grad += A.potential_backward(g, pos[t], species, amp_sigma, g_v)
    for sp in range(2):
        for c, h in ((0, 1e-4), (1, 1e-6)):
            ee = np.zeros_like(amp_sigma)
            ee[sp, c] = 1.0
            d = _fd(lambda hh: total(amp_sigma + hh * ee), 0.0, h)
            assert grad[sp, c] == pytest.approx(d, rel=1e-5)
