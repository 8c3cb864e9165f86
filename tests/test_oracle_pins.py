"""Pins of the FP64 oracle to facts fixed by the paper and the mathematics.

Each test checks one oracle function against something other than itself:
printed values (tests/golden), closed forms, brute-force sums on tiny
inputs, or invariants.  They run on the CPU (no GPU marker).
"""

import os

import numpy as np
import pytest
from scipy import integrate

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    return np.array(rows)


def _grid(nx=16, ny=16, lx=8.0, ly=8.0, n_slices=4, dz=2.0, z0=0.0, kev=100.0, bl=2.0 / 3.0):
    return O.Grid(nx, ny, lx, ly, n_slices, dz, z0, kev, bl)


# ---------------------------------------------------------------------------
# Beam constants
# ---------------------------------------------------------------------------
def test_beam_constants_textbook_values():
    for kev, lam, sig in _golden("beam_constants.txt"):
        assert O.wavelength(kev) == pytest.approx(lam, rel=2e-4)
        assert O.interaction_constant(kev) == pytest.approx(sig, rel=2e-4)


def test_beam_constants_energy_momentum_route():
    # lambda = hc / sqrt(E_k (E_k + 2 m c^2)) and the interaction parameter in
    # the form 2 pi / (lambda U) * (m c^2 + eU) / (2 m c^2 + eU), with hc and
    # m c^2 taken as CODATA energies rather than SI constants.
    hc_kev_a = 12.398419843320026
    mc2_kev = 510.99895000
    for kev in (60.0, 100.0, 200.0, 300.0):
        lam = hc_kev_a / np.sqrt(kev * (kev + 2.0 * mc2_kev))
        sig = 2.0 * np.pi / (lam * kev * 1e3) * (mc2_kev + kev) / (2.0 * mc2_kev + kev)
        assert O.wavelength(kev) == pytest.approx(lam, rel=1e-9)
        assert O.interaction_constant(kev) == pytest.approx(sig, rel=1e-9)


# ---------------------------------------------------------------------------
# Energy grid of the time-to-energy transform
# ---------------------------------------------------------------------------
def test_energy_limits_match_paper_footnotes():
    for dt, thz, mev, digits in _golden("paper_energy_limits.txt"):
        e = O.natural_energies(1000, dt)
        e_max = np.max(np.abs(e))                      # Nyquist bin, labelled -E_max
        assert e_max == pytest.approx(O.H_MEV_FS / (2 * dt), rel=1e-12)
        f_thz = e_max / O.H_MEV_FS * 1e3               # E = h f
        tol = 0.5 * 10 ** (np.floor(np.log10(mev)) - digits + 1)
        assert abs(e_max - mev) <= tol + 0.5           # printed with "~"
        assert f_thz == pytest.approx(thz, rel=1e-3)


def test_energy_grid_resolution_and_order():
    t, dt = 256, 5.0
    e = O.natural_energies(t, dt)
    assert np.all(np.diff(e) > 0)
    assert np.allclose(np.diff(e), O.H_MEV_FS / (t * dt), rtol=1e-12)
    assert e[t // 2] == 0.0
    assert e[0] == pytest.approx(-O.H_MEV_FS / (2 * dt), rel=1e-12)
    # plain_small: E_min = 3.231 meV, E_max = 413.57 meV
    assert O.H_MEV_FS / (t * dt) == pytest.approx(3.2310, abs=1e-4)
    assert O.H_MEV_FS / (2 * dt) == pytest.approx(413.567, abs=1e-3)


# ---------------------------------------------------------------------------
# Transforms against brute-force DFTs
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("ny,nx", [(4, 4), (6, 6), (12, 12), (4, 6), (6, 12)])
def test_fft2_unitary_bruteforce(ny, nx):
    rng = np.random.default_rng(ny * 100 + nx)
    psi = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    ref = np.zeros((ny, nx), dtype=complex)
    inv = np.zeros((ny, nx), dtype=complex)
    for ky in range(ny):
        for kx in range(nx):
            for y in range(ny):
                for x in range(nx):
                    ph = 2 * np.pi * (kx * x / nx + ky * y / ny)
                    ref[ky, kx] += psi[y, x] * np.exp(-1j * ph)
                    inv[ky, kx] += psi[y, x] * np.exp(1j * ph)
    ref /= nx * ny
    assert np.allclose(O.fft2_unitary(psi), ref, atol=1e-13, rtol=0)
    assert np.allclose(O.ifft2_unitary(psi), inv, atol=1e-12, rtol=0)


@pytest.mark.parametrize("t", [8, 9, 12])
def test_temporal_transform_bruteforce(t):
    rng = np.random.default_rng(t)
    dt = 5.0
    a = rng.standard_normal((t, 3)) + 1j * rng.standard_normal((t, 3))
    e = O.natural_energies(t, dt)
    ref = np.zeros((3, t), dtype=complex)
    for q in range(3):
        for k in range(t):
            for n in range(t):
                ref[q, k] += a[n, q] * np.exp(-1j * e[k] * n * dt / O.HBAR_MEV_FS)
    assert np.allclose(O.temporal_transform(a, dt), ref, atol=1e-12, rtol=0)
    # the explicit DFT-matrix path at the natural energies gives the same result
    assert np.allclose(O.temporal_transform(a, dt, e), ref, atol=1e-12, rtol=0)
    # natural grid index k corresponds to integer frequency k - T//2
    kk = np.arange(t) - t // 2
    assert np.allclose(e, kk * O.H_MEV_FS / (t * dt), rtol=1e-13, atol=1e-12)


def test_energy_sign_loss_is_positive():
    # An exit-wave component oscillating as exp(+i E0 t / hbar) is a loss of E0
    # (Eq. (5): transitions n->m carry exp(i (E_m - E_n) t / hbar) and the
    # transform kernel is exp(-i E t / hbar)).
    t, dt = 64, 5.0
    e = O.natural_energies(t, dt)
    k0 = 5
    e0 = e[t // 2 + k0]
    n = np.arange(t)
    psi = 0.3 + 1e-2 * np.exp(1j * e0 * n * dt / O.HBAR_MEV_FS)
    inten, _, en = O.spectrum(psi[:, None], dt)
    assert en[np.argmax(inten[0])] == pytest.approx(e0)
    assert e0 > 0


# ---------------------------------------------------------------------------
# Slice potential
# ---------------------------------------------------------------------------
def test_slice_weights_quadrature_and_sum():
    g = _grid(n_slices=5, dz=2.0, z0=1.0)
    sig = 0.3
    for z in (0.2, 1.0, 1.3, 2.999, 3.0, 6.4, 9.0, 11.5, 12.0):
        w = O.slice_weights(z, sig, g)
        assert w.sum() == pytest.approx(1.0, abs=3e-9)
        pdf = lambda x: np.exp(-((x - z) ** 2) / (2 * sig**2)) / (np.sqrt(2 * np.pi) * sig)
        edges = g.z0 + g.dz * np.arange(g.n_slices + 1)
        lo = np.r_[z - 12 * sig, edges[1:-1]]
        hi = np.r_[edges[1:-1], z + 12 * sig]
        for s in range(g.n_slices):
            a, b = max(lo[s], z - 12 * sig), min(hi[s], z + 12 * sig)
            ref = integrate.quad(pdf, a, b, epsabs=1e-14)[0] if b > a else 0.0
            assert w[s] == pytest.approx(ref, abs=3e-9)


def test_slice_weights_boundary_split():
    g = _grid(n_slices=4, dz=4.0, z0=0.0)
    w = O.slice_weights(8.0, 0.3, g)                   # on the edge between slices 1 and 2
    assert w[1] == pytest.approx(0.5, abs=1e-12)
    assert w[2] == pytest.approx(0.5, abs=1e-12)
    assert w[0] == 0.0 and w[3] == 0.0


def _atoms_small(rng, n, g, n_species):
    pos = np.stack([rng.uniform(-0.5, g.lx + 0.5, n), rng.uniform(-0.5, g.ly + 0.5, n),
                    rng.uniform(g.z0 - 1, g.z0 + g.n_slices * g.dz + 1, n)], axis=1)
    species = rng.integers(0, n_species, n)
    return pos, species


def test_potential_window_equals_bruteforce():
    rng = np.random.default_rng(7)
    g = _grid(nx=24, ny=20, lx=9.0, ly=7.5, n_slices=3, dz=1.5, z0=0.5)
    pos, species = _atoms_small(rng, 30, g, 2)
    amp_sigma = np.array([[20.0, 0.3], [11.0, 0.41]])
    v = O.projected_potential(g, pos, species, amp_sigma)
    vb = O.projected_potential_bruteforce(g, pos, species, amp_sigma)
    assert np.allclose(v, vb, atol=1e-12, rtol=0)


def test_potential_integral_sum_rule():
    # sum_s sum_pixels v d^2 = sum_a amp 2 pi s^2 for a well-sampled Gaussian
    # (s/d = 3 makes the sampling error exp(-2 pi^2 s^2/d^2) negligible).
    rng = np.random.default_rng(3)
    g = _grid(nx=96, ny=80, lx=9.6, ly=8.0, n_slices=4, dz=2.0)
    pos, species = _atoms_small(rng, 12, g, 2)
    amp_sigma = np.array([[20.0, 0.3], [15.0, 0.35]])
    v = O.projected_potential(g, pos, species, amp_sigma)
    d2 = (g.lx / g.nx) * (g.ly / g.ny)
    ref = sum(amp_sigma[s, 0] * 2 * np.pi * amp_sigma[s, 1] ** 2 for s in species)
    # the 6-sigma square keeps erf(6/sqrt2)^2 of each Gaussian
    from scipy.special import erf as _erf
    assert v.sum() * d2 == pytest.approx(ref * _erf(6.0 / np.sqrt(2.0)) ** 2, rel=1e-9)


def test_potential_fourier_transform_analytic():
    # (1/N^2) sum_r v(r) e^{-2 pi i q.r} = (1/(lx ly)) sum_a amp 2 pi s^2
    #   exp(-2 pi^2 s^2 q^2) exp(-2 pi i q.R_a)   (atoms entirely in one slice)
    rng = np.random.default_rng(11)
    g = _grid(nx=96, ny=72, lx=9.6, ly=8.1, n_slices=1, dz=50.0, z0=-25.0)
    n = 5
    pos = np.stack([rng.uniform(0, g.lx, n), rng.uniform(0, g.ly, n), np.zeros(n)], axis=1)
    amp, s = 20.0, 0.3
    v = O.projected_potential(g, pos, np.zeros(n, int), [[amp, s]])[0]
    vq = O.fft2_unitary(v)
    qx, qy = O.spatial_frequencies(g)
    q2 = qx[None, :] ** 2 + qy[:, None] ** 2
    ph = sum(np.exp(-2j * np.pi * (qx[None, :] * p[0] + qy[:, None] * p[1])) for p in pos)
    ref = amp * 2 * np.pi * s * s * np.exp(-2 * np.pi**2 * s * s * q2) * ph / (g.lx * g.ly)
    assert np.max(np.abs(vq - ref)) < 1e-6 * np.max(np.abs(ref))


# ---------------------------------------------------------------------------
# Multislice
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(128, 128, 64.0, 64.0), (128, 96, 64.0, 60.0)])
def test_free_space_gaussian_beam_closed_form(shape):
    # V = 0: an elliptical Gaussian incident wave exp(-x^2/(2 wx^2) - y^2/(2 wy^2))
    # after a distance z is prod_c (w_c / w'_c) exp(-c^2 / (2 w'_c^2)) with
    # w'_c^2 = w_c^2 + i lambda z / (2 pi)  (paraxial Fresnel propagation).
    nx, ny, lx, ly = shape
    g = _grid(nx=nx, ny=ny, lx=lx, ly=ly, n_slices=20, dz=50.0, kev=100.0)
    wx, wy = 3.0, 2.5
    x = np.arange(g.nx) * g.lx / g.nx
    y = np.arange(g.ny) * g.ly / g.ny
    xc, yc = lx / 2, ly / 2
    ex2 = (x[None, :] - xc) ** 2
    ey2 = (y[:, None] - yc) ** 2
    psi_in = np.exp(-ex2 / (2 * wx * wx) - ey2 / (2 * wy * wy))
    out = O.multislice(g, np.zeros((g.n_slices, g.ny, g.nx)), psi_in)
    psi_r = O.ifft2_unitary(out)
    z = g.n_slices * g.dz
    c = 1j * O.wavelength(g.kev) * z / (2 * np.pi)

    def beam(cc):
        wx2, wy2 = wx * wx + cc, wy * wy + cc
        return np.sqrt(wx * wx / wx2) * np.sqrt(wy * wy / wy2) \
            * np.exp(-ex2 / (2 * wx2) - ey2 / (2 * wy2))

    ref = beam(c)
    assert np.max(np.abs(psi_r - ref)) < 1e-10
    # ... and with the propagator sign flipped the beam would differ by O(1)
    assert np.max(np.abs(psi_r - beam(np.conj(c)))) > 0.05


def test_uniform_potential_is_a_global_phase():
    g = _grid(nx=12, ny=12, n_slices=5, dz=2.0, kev=200.0)
    v0 = 7.5
    out = O.multislice(g, np.full((g.n_slices, g.ny, g.nx), v0))
    sig = O.interaction_constant(g.kev)
    assert out[0, 0] == pytest.approx(np.exp(1j * g.n_slices * sig * v0), abs=1e-14)
    out[0, 0] = 0
    assert np.max(np.abs(out)) < 1e-15


def test_weak_phase_single_slice_first_order():
    # One thin slice with one atom: Psi(q != 0) = i sigma v^(q) P(q) + O(sigma^2 v^2)
    g = _grid(nx=96, ny=96, lx=9.6, ly=9.6, n_slices=1, dz=1.0, z0=-0.5, kev=100.0)
    amp, s = 2.0, 0.3
    pos = np.array([[4.1, 5.3, 0.0]])
    v = O.projected_potential(g, pos, [0], [[amp, s]])
    out = O.multislice(g, v)
    sig = O.interaction_constant(g.kev)
    qx, qy = O.spatial_frequencies(g)
    q2 = qx[None, :] ** 2 + qy[:, None] ** 2
    vq = amp * 2 * np.pi * s * s * np.exp(-2 * np.pi**2 * s * s * q2) \
        * np.exp(-2j * np.pi * (qx[None, :] * pos[0, 0] + qy[:, None] * pos[0, 1])) / (g.lx * g.ly)
    ref = 1j * sig * vq * O.propagator(g)
    mask = (q2 > 0) & (O.bandlimit_mask(g) > 0)
    err = np.max(np.abs(out[mask] - ref[mask]))
    assert err < 2 * (sig * amp) ** 2 * np.max(np.abs(vq[mask])) / (sig * amp) + 1e-9
    # the wrong transmission sign, exp(-i sigma V), would be off by 2|ref|
    assert np.max(np.abs(out[mask] + ref[mask])) > 1.5 * np.max(np.abs(ref[mask]))


def test_norm_conserved_without_bandlimit_and_lost_outside_it():
    rng = np.random.default_rng(5)
    g = _grid(nx=32, ny=32, lx=16.0, ly=16.0, n_slices=6, dz=2.0, bl=10.0)
    v = rng.uniform(0, 30, (g.n_slices, g.ny, g.nx))
    out = O.multislice(g, v)
    assert np.sum(np.abs(out) ** 2) == pytest.approx(1.0, abs=1e-13)
    # with the 2/3 band limit one slice keeps exactly the power inside the disc
    g1 = _grid(nx=32, ny=32, lx=16.0, ly=16.0, n_slices=1, dz=2.0)
    chi_q = O.fft2_unitary(np.exp(1j * O.interaction_constant(g1.kev) * v[0]))
    inside = np.sum(np.abs(chi_q) ** 2 * O.bandlimit_mask(g1))
    out1 = O.multislice(g1, v[:1])
    assert np.sum(np.abs(out1) ** 2) == pytest.approx(inside, abs=1e-14)
    assert inside < 1.0 - 1e-6


def test_bandlimit_disc_radius():
    # plain_small: 64^2 over 32 A -> q_Nyq = 1/A, kept radius 2/3 1/A = 21.33 px
    g = O.grid_from_spec(W.WORKLOADS["plain_small"].grid)
    bl = O.bandlimit_mask(g)
    k = np.fft.fftfreq(64, 1.0 / 64)
    kk = k[None, :] ** 2 + k[:, None] ** 2
    assert np.array_equal(bl > 0, kk <= (64 / 3.0) ** 2)
    assert np.array_equal(bl > 0, 9 * kk <= 64 * 64)
    # non-square: 64 x 48 pixels over 32 x 32 A -> q_Nyq = min(1, 0.75) = 0.75 1/A,
    # kept radius 0.5 1/A, i.e. kx^2 + ky^2 <= 16^2 in units of 1/(32 A)
    g2 = _grid(nx=64, ny=48, lx=32.0, ly=32.0)
    kx = np.fft.fftfreq(64, 1.0 / 64)
    ky = np.fft.fftfreq(48, 1.0 / 48)
    k2 = kx[None, :] ** 2 + ky[:, None] ** 2
    assert np.array_equal(O.bandlimit_mask(g2) > 0, k2 <= 256)


# ---------------------------------------------------------------------------
# Spectrum
# ---------------------------------------------------------------------------
def _waves(rng, t, nq=6):
    return (1.0 + 0.05 * (rng.standard_normal((t, nq)) + 1j * rng.standard_normal((t, nq))))


def test_parseval_energy_integral_equals_qep():
    # I_el(q) + sum_k I(q, E_k) = mean_t |psi(q, t)|^2 on the natural grid:
    # the energy integral of the spectrum equals the QEP / frozen-phonon
    # intensity (Eq. (4) with Eq. (3)).
    rng = np.random.default_rng(1)
    psi = _waves(rng, 32)
    inten, iel, _ = O.spectrum(psi, 5.0)
    assert np.allclose(iel + inten.sum(axis=1), np.mean(np.abs(psi) ** 2, axis=0), rtol=1e-13)


def test_wiener_khinchin():
    # DFT of the circular autocorrelation (1/T) sum_t A*(t) A(t+tau) equals T I(q, E)
    rng = np.random.default_rng(2)
    t, dt = 16, 5.0
    psi = _waves(rng, t, 3)
    inten, _, e = O.spectrum(psi, dt)
    a = psi - psi.mean(axis=0)
    for q in range(3):
        c = np.array([np.sum(np.conj(a[:, q]) * np.roll(a[:, q], -tau)) / t for tau in range(t)])
        ck = np.array([np.sum(c * np.exp(-1j * ek * np.arange(t) * dt / O.HBAR_MEV_FS)) for ek in e])
        assert np.allclose(ck.real, t * inten[q], atol=1e-13)
        assert np.allclose(ck.imag, 0.0, atol=1e-13)


def test_elastic_bin_zero_and_static_lattice():
    rng = np.random.default_rng(3)
    psi = _waves(rng, 20)
    inten, iel, e = O.spectrum(psi, 5.0)
    assert np.all(inten[:, e == 0.0] < 1e-28)
    # identical snapshots: no inelastic intensity, elastic = |psi|^2
    static = np.repeat(psi[:1], 16, axis=0)
    inten, iel, _ = O.spectrum(static, 5.0)
    assert np.max(inten) < 1e-28
    assert np.allclose(iel, np.abs(psi[0]) ** 2, rtol=1e-14)


def test_kubo_factor_detailed_balance():
    e = np.array([-50.0, -1.0, -1e-9, 0.0, 1e-9, 1.0, 50.0])
    f = O.kubo_factor(e, 300.0)
    beta = 1.0 / (O.KB_MEV_PER_K * 300.0)
    assert f[3] == 1.0
    assert np.allclose(f / f[::-1], np.exp(beta * e), rtol=1e-12)
    assert np.allclose(f[2:5], 1.0 + beta * e[2:5] / 2, atol=1e-12)
    assert O.KB_MEV_PER_K * 300.0 == pytest.approx(25.852, abs=1e-3)


def test_normalisation_sums_to_one():
    rng = np.random.default_rng(4)
    psi = _waves(rng, 24)
    inten, iel, _ = O.spectrum(psi, 5.0, kubo=True, normalize=True)
    assert inten.sum() + iel.sum() == pytest.approx(1.0, abs=1e-14)


def _single_mode_run(standing, k_on_bin, t=64, dt=5.0):
    """Small crystal driven by one harmonic mode exactly on a DFT bin."""
    g = _grid(nx=32, ny=32, lx=8.0, ly=8.0, n_slices=2, dz=4.0, z0=0.0, kev=100.0)
    cr = W.simple_cubic((2, 2, 2), 4.0)
    e_mode = k_on_bin * O.H_MEV_FS / (t * dt)
    om = e_mode / O.HBAR_MEV_FS
    kvec = 2 * np.pi * np.array([1, 0, 0]) / cr.cell
    pol = np.array([0.6, 0.8, 0.0])
    tt = np.arange(t) * dt
    arg = cr.positions @ kvec + 0.4
    if standing:
        u = 0.15 * np.cos(arg)[None, :, None] * np.cos(om * tt)[:, None, None] * pol
    else:
        u = 0.15 * np.cos(arg[None, :] - om * tt[:, None])[:, :, None] * pol
    pos = cr.positions[None] + u
    psi = O.exit_waves(g, pos, cr.species, [[20.0, 0.3]])
    return psi, dt, e_mode


@pytest.mark.parametrize("standing", [False, True])
def test_single_mode_sidebands(standing):
    k0 = 4
    psi, dt, e_mode = _single_mode_run(standing, k0)
    t = psi.shape[0]
    inten, _, e = O.spectrum(psi.reshape(t, -1), dt)
    k = np.arange(t) - t // 2
    harm = (k % k0) == 0
    tot = inten.sum()
    assert tot > 1e-8
    assert inten[:, ~harm].sum() < 1e-12 * tot             # only at n * hbar Omega
    assert inten[:, k == k0].sum() > 1e-3 * tot             # first-order loss ...
    assert inten[:, k == -k0].sum() > 1e-3 * tot            # ... and gain sidebands
    if standing:
        # time-reversal symmetric trajectory: loss and gain sidebands equal
        for n in (1, 2):
            assert inten[:, k == n * k0] == pytest.approx(inten[:, k == -n * k0], rel=1e-9, abs=1e-30)
        # after the Kubo factor, gain / loss = exp(-beta hbar Omega)  (Eq. (8))
        ik, _, _ = O.spectrum(psi.reshape(t, -1), dt, kubo=True, temperature_K=300.0)
        beta = 1.0 / (O.KB_MEV_PER_K * 300.0)
        sel = inten[:, k == k0][:, 0] > 1e-6 * inten.max()
        ratio = ik[sel, k == -k0] / ik[sel, k == k0]
        assert np.allclose(ratio, np.exp(-beta * e_mode), rtol=1e-9)


def test_plain_small_inputs_are_seeded():
    w = W.WORKLOADS["plain_small"]
    a = W.build_inputs(w).positions(snapshots=[0, 17])
    b = W.build_inputs(w).positions(snapshots=[0, 17])
    assert np.array_equal(a, b)
    inp = W.build_inputs(w)
    u = inp.positions().astype(np.float64) - inp.crystal.positions[None]
    rms = np.sqrt(np.mean(np.sum(u**2, axis=-1)))
    assert rms == pytest.approx(0.05, rel=0.1)


# ---------------------------------------------------------------------------
# Spectra averaged over sets of consecutive snapshots
# ---------------------------------------------------------------------------
def test_segment_sets_match_paper():
    # set counts and durations the paper prints for its three trajectories
    for dt, n_t, seg, hop, n_sets, span_ps, all_fit in _golden("paper_segment_sets.txt"):
        n_t, seg, hop, n_sets = int(n_t), int(seg), int(hop), int(n_sets)
        most = O.segment_count(n_t, seg, hop)
        if all_fit:
            assert most == n_sets
        else:
            assert most >= n_sets
        assert seg * dt / 1000.0 == pytest.approx(span_ps, abs=0.006)
        starts = O.segment_starts(n_t, seg, hop, n_sets)
        assert len(starts) == n_sets and starts[-1] + seg <= n_t
    # Si: every snapshot is used twice except the first and the last 50
    use = np.zeros(4000, int)
    for s0 in O.segment_starts(4000, 100, 50):
        use[s0:s0 + 100] += 1
    assert np.all(use[50:-50] == 2) and np.all(use[:50] == 1) and np.all(use[-50:] == 1)


def test_segment_spectrum_one_set_is_the_spectrum():
    rng = np.random.default_rng(10)
    psi = _waves(rng, 24, 5)
    a = O.segment_spectrum(psi, 5.0, 24, 7)
    b = O.spectrum(psi, 5.0)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_segment_spectrum_bruteforce():
    # 12 snapshots, sets of 6 offset by 2 (starts 0, 2, 4, 6): per-set means and
    # DFT sums written out as plain loops
    rng = np.random.default_rng(11)
    t, seg, hop, dt = 12, 6, 2, 5.0
    psi = _waves(rng, t, 2)
    inten, iel, e = O.segment_spectrum(psi, dt, seg, hop)
    starts = [0, 2, 4, 6]
    for q in range(2):
        ref_i = np.zeros(seg)
        ref_el = 0.0
        for s0 in starts:
            m = sum(psi[s0 + n, q] for n in range(seg)) / seg
            ref_el += abs(m) ** 2 / len(starts)
            for k in range(seg):
                ek = (k - seg // 2) * O.H_MEV_FS / (seg * dt)
                phi = sum((psi[s0 + n, q] - m) * np.exp(-1j * ek * n * dt / O.HBAR_MEV_FS) for n in range(seg))
                ref_i[k] += abs(phi) ** 2 / seg ** 2 / len(starts)
        assert np.allclose(inten[q], ref_i, rtol=1e-12, atol=1e-18)
        assert iel[q] == pytest.approx(ref_el, rel=1e-13)


def test_segment_spectrum_parseval_over_tiling_sets():
    # sets that tile the trajectory: I_el + sum_k I = mean over all snapshots of |psi|^2
    rng = np.random.default_rng(12)
    psi = _waves(rng, 32, 4)
    inten, iel, _ = O.segment_spectrum(psi, 5.0, 8, 8)
    assert np.allclose(iel + inten.sum(axis=1), np.mean(np.abs(psi) ** 2, axis=0), rtol=1e-13)
    # with kubo and normalisation the averages still sum to one
    inten, iel, _ = O.segment_spectrum(psi, 5.0, 8, 4, kubo=True, normalize=True)
    assert inten.sum() + iel.sum() == pytest.approx(1.0, abs=1e-14)


def test_segment_spectrum_single_mode_on_bin():
    # a mode on bin 4 of 64 snapshots sits on bin 2 of every set of 32
    psi, dt, _ = _single_mode_run(False, 4)
    t = psi.shape[0]
    inten, _, e = O.segment_spectrum(psi.reshape(t, -1), dt, 32, 16)
    k = np.arange(32) - 16
    harm = (k % 2) == 0
    tot = inten.sum()
    assert inten[:, ~harm].sum() < 1e-12 * tot
    assert inten[:, k == 2].sum() > 1e-3 * tot and inten[:, k == -2].sum() > 1e-3 * tot


# ---------------------------------------------------------------------------
# QEP by-products: patterns, energy integrals, line and azimuthal profiles
# ---------------------------------------------------------------------------
def test_qep_subset_of_the_si_trajectory():
    # first figure: "QEP 100" takes 100 evenly spaced snapshots every 1 ps out of
    # the 4000 snapshots at 25 fs, i.e. every 40th; with |psi(t)|^2 = t the
    # pattern is the mean of 0, 40, ..., 3960 = 1980
    psi = np.sqrt(np.arange(4000.0))[:, None] * np.ones((1, 3))
    stride = int(round(1000.0 / 25.0))
    assert len(np.arange(0, 4000, stride)) == 100
    assert np.allclose(O.qep_intensity(psi, 0, stride), 1980.0, rtol=1e-15)
    assert np.allclose(O.qep_intensity(psi, 10, stride, n=3), (10 + 50 + 90) / 3.0, rtol=1e-15)


def test_energy_integral_equals_qep_of_all_snapshots():
    rng = np.random.default_rng(13)
    psi = _waves(rng, 40, 7)
    inten, iel, _ = O.spectrum(psi, 5.0)
    assert np.allclose(O.energy_integral(inten, iel), O.qep_intensity(psi), rtol=1e-13)


def test_line_profile_bragg_spots_of_a_static_crystal():
    # a crystal with period a = 8 pixels diffracts only into k_x = 8 h; along
    # theta_y = 0 the pattern sits at theta_x = lambda h / a
    g = _grid(nx=64, ny=64, lx=32.0, ly=32.0, n_slices=2, dz=4.0, z0=0.0, kev=100.0)
    cr = W.simple_cubic((8, 8, 2), 4.0)
    psi = O.exit_waves(g, cr.positions[None].astype(np.float64), cr.species, [[20.0, 0.3]], processes=1)
    lam = O.wavelength(g.kev)
    line, theta = O.line_profile(O.qep_intensity(psi), g.lx, lam)
    k = np.arange(64) - 32
    assert np.allclose(theta, lam * k / 32.0 * 1000.0, rtol=1e-14)
    bragg = (k % 8) == 0
    assert np.max(line[~bragg]) < 1e-20 * np.max(line)
    for h in (-2, -1, 0, 1, 2):                                    # inside the 2/3 band limit
        assert line[k == 8 * h][0] > 1e-8 * np.max(line)
        assert theta[k == 8 * h][0] == pytest.approx(lam * h / 4.0 * 1000.0, rel=1e-14, abs=1e-14)


def test_azimuthal_profile_bruteforce():
    import math
    rng = np.random.default_rng(14)
    nx, ny, lx, ly, lam, dth, nb = 6, 5, 3.0, 2.5, 0.037, 7.3, 4
    values = rng.random((ny, nx))
    prof, counts = O.azimuthal_profile(values, lx, ly, lam, dth, nb)
    ref_s, ref_c = np.zeros(nb), np.zeros(nb, int)
    for j in range(ny):
        for i in range(nx):
            ki = i if i < (nx + 1) // 2 else i - nx
            kj = j if j < (ny + 1) // 2 else j - ny
            th = lam * math.hypot(ki / lx, kj / ly) * 1000.0
            b = int(th // dth)
            if b < nb:
                ref_s[b] += values[j, i]
                ref_c[b] += 1
    assert np.array_equal(counts, ref_c) and counts.sum() > 0 and np.all(counts > 0)
    assert np.allclose(prof, ref_s / ref_c, rtol=1e-14)


def test_relative_difference_closed_forms():
    a = np.array([3.0, 1.0, 0.0, 2.0, -1.0])
    b = np.array([1.0, 3.0, 0.0, 2.0, 1.0])
    r = O.relative_difference(a, b)
    assert np.array_equal(r[:4], [0.5, -0.5, 0.0, 0.0])
    assert r[4] == 0.0                                   # a + b = 0
    assert np.array_equal(O.relative_difference(b, a)[:4], -r[:4])


# ---------------------------------------------------------------------------
# Convergent probe
# ---------------------------------------------------------------------------
def test_probe_aperture_and_normalisation():
    import math
    g = _grid(nx=48, ny=40, lx=30.0, ly=25.0, n_slices=1, dz=2.0, kev=200.0)
    lam = O.wavelength(g.kev)
    alpha = 6.3                                        # mrad
    psi = O.probe(g, alpha)
    assert np.mean(np.abs(psi) ** 2) == pytest.approx(1.0, abs=1e-13)
    psi_q = O.fft2_unitary(psi)
    n_ap = 0
    for j in range(g.ny):
        for i in range(g.nx):
            ki = i if i < (g.nx + 1) // 2 else i - g.nx
            kj = j if j < (g.ny + 1) // 2 else j - g.ny
            if lam * math.hypot(ki / g.lx, kj / g.ly) * 1000.0 <= alpha:
                n_ap += 1
                assert abs(psi_q[j, i]) == pytest.approx(1.0 / math.sqrt(n_ap_total(g, lam, alpha)), rel=1e-12)
            else:
                assert abs(psi_q[j, i]) < 1e-14
    assert n_ap == n_ap_total(g, lam, alpha) and n_ap > 10
    # an aperture that holds only q = 0 gives the unit plane wave
    assert np.allclose(O.probe(g, 1e-3), 1.0, atol=1e-14)


def n_ap_total(g, lam, alpha):
    qx = np.fft.fftfreq(g.nx, d=g.lx / g.nx)
    qy = np.fft.fftfreq(g.ny, d=g.ly / g.ny)
    return int(np.count_nonzero(lam * np.hypot(qx[None, :], qy[:, None]) * 1000.0 <= alpha))


def test_probe_position_is_a_circular_shift():
    g = _grid(nx=64, ny=48, lx=32.0, ly=24.0, n_slices=1, dz=2.0, kev=200.0)
    p0 = O.probe(g, 12.0, defocus_A=40.0)
    p1 = O.probe(g, 12.0, defocus_A=40.0, x0=3 * g.lx / g.nx, y0=5 * g.ly / g.ny)
    assert np.allclose(p1, np.roll(p0, (5, 3), axis=(0, 1)), atol=1e-12)
    assert np.argmax(np.abs(O.probe(g, 12.0, x0=3 * g.lx / g.nx, y0=5 * g.ly / g.ny))) == 5 * g.nx + 3


def test_probe_defocus_is_free_propagation():
    # a probe defocused by f equals the focused probe propagated through f of vacuum
    g = _grid(nx=64, ny=64, lx=32.0, ly=32.0, n_slices=2, dz=25.0, kev=200.0)
    focused = O.probe(g, 15.0)
    exit_q = O.multislice(g, np.zeros((2, 64, 64)), psi_in=focused)
    assert np.allclose(exit_q, O.fft2_unitary(O.probe(g, 15.0, defocus_A=50.0)), atol=1e-13)
