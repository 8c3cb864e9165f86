"""Plain FP64 CPU oracle of the TACAW hot path -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import this module.  It shares no code with the CUDA
path; both consume the same seeded inputs from ``workloads``.

What it computes (arXiv 2401.15599, the two-step procedure after Eq. (9)):

1. For each snapshot of a trajectory, propagate a plane wave through the
   snapshot by multislice (the paper defers to the standard multislice of
   Cowley and Moodie; the textbook form used here is written out below).
2. Stack the exit waves phi_MD(q, t), Fourier transform over time, take the
   squared modulus (Eq. (9) via the convolution theorem), optionally apply
   the Kubo detailed-balance factor (Eq. (8)) and the fractional-intensity
   normalisation (the unnumbered equation after Eq. (9)).

Readings taken where the paper is silent:

* Atoms are isotropic 3-D Gaussians; ``amp`` is the peak of the z-projection
  (V*A), so the projected profile is amp*exp(-rho^2/(2 s^2)).  Laterally the
  profile is truncated to the square |dx|, |dy| <= 6 s (so that it stays
  exactly separable in x and y) and summed with the minimum periodic image.
* An atom is split over slices by the fraction of its z-Gaussian inside each
  slice (differences of erf); the first slice reaches -inf and the last +inf;
  slices that do not meet [z - 6 s, z + 6 s] get weight 0.
* Unitary-scaled FFT: Psi(q) = (1/N^2) sum_r psi(r) exp(-2 pi i q.r); the
  inverse has no 1/N^2.
* Each slice: transmit by exp(i sigma_e V), forward FFT, multiply by the
  Fresnel propagator exp(-i pi lambda dz |q|^2) and the circular band limit
  |q| <= bandlimit * q_Nyquist, inverse FFT.  The last slice is propagated
  too and the exit wave is returned in q-space (FFT order).
* Elastic part = |time mean of psi|^2, reported separately; the inelastic
  spectrum transforms psi - mean.
* Energy sign: Phi(q, E) = sum_n A(q, t_n) exp(-i E t_n / hbar); E > 0 is
  energy loss.  Natural grid E_k = h k / (T dt), k = -T/2 .. T/2-1.

Parity of the whole C0/C1 pipeline is pinned only through the invariants in
``tests/test_oracle_pins.py`` (closed forms, brute-force DFTs, Parseval,
Wiener-Khinchin, static lattice, single-mode sidebands); beyond them the
end-to-end result is checked by agreement of two independent codes.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.special import erf

__all__ = [
    "H_MEV_FS", "HBAR_MEV_FS", "KB_MEV_PER_K",
    "Grid", "grid_from_spec", "wavelength", "interaction_constant",
    "slice_weights", "projected_potential", "projected_potential_bruteforce",
    "spatial_frequencies", "bandlimit_mask", "propagator",
    "fft2_unitary", "ifft2_unitary", "multislice", "exit_waves",
    "natural_energies", "time_mean", "temporal_transform", "kubo_factor",
    "spectrum", "segment_count", "segment_starts", "segment_spectrum",
    "qep_intensity", "energy_integral", "scattering_angles", "line_profile", "azimuthal_profile",
    "relative_difference", "probe",
]

# ---------------------------------------------------------------------------
# Physical constants (CODATA 2018, exact SI definitions where available).
# ---------------------------------------------------------------------------
PLANCK_J_S = 6.62607015e-34
C_M_S = 299792458.0
ME_KG = 9.1093837015e-31
E_C = 1.602176634e-19
H_MEV_FS = PLANCK_J_S / E_C * 1e3 * 1e15          # h in meV*fs
HBAR_MEV_FS = H_MEV_FS / (2.0 * np.pi)            # hbar in meV*fs
KB_MEV_PER_K = 1.380649e-23 / E_C * 1e3           # Boltzmann constant, meV/K


@dataclass(frozen=True)
class Grid:
    """Periodic simulation box and beam (lengths in Angstrom, energy in keV)."""

    nx: int
    ny: int
    lx: float
    ly: float
    n_slices: int
    dz: float
    z0: float
    kev: float
    bandlimit: float = 2.0 / 3.0


def grid_from_spec(spec) -> Grid:
    return Grid(spec.nx, spec.ny, spec.lx, spec.ly, spec.n_slices, spec.dz,
                spec.z0, spec.kev, spec.bandlimit)


# ---------------------------------------------------------------------------
# Beam constants: relativistic wavelength and interaction constant.
# ---------------------------------------------------------------------------
def wavelength(kev: float) -> float:
    """Relativistic electron wavelength in Angstrom.

    lambda = h / sqrt(2 m0 e U (1 + e U / (2 m0 c^2))).
    """
    eu = kev * 1e3 * E_C
    p = np.sqrt(2.0 * ME_KG * eu * (1.0 + eu / (2.0 * ME_KG * C_M_S**2)))
    return PLANCK_J_S / p * 1e10


def interaction_constant(kev: float) -> float:
    """sigma_e = 2 pi gamma m0 e lambda / h^2 in rad / (V * Angstrom)."""
    eu = kev * 1e3 * E_C
    gamma = 1.0 + eu / (ME_KG * C_M_S**2)
    lam_m = wavelength(kev) * 1e-10
    return 2.0 * np.pi * gamma * ME_KG * E_C * lam_m / PLANCK_J_S**2 * 1e-10


# ---------------------------------------------------------------------------
# Slice potential: Gaussian atoms projected onto the grid.
# ---------------------------------------------------------------------------
def slice_weights(z: float, sigma: float, g: Grid) -> np.ndarray:
    """Fraction of a z-Gaussian (centre z, width sigma) inside each slice.

    w_s = (erf(u_{s+1}) - erf(u_s)) / 2 with u = (edge - z) / (sqrt(2) sigma);
    the first lower edge is -inf and the last upper edge +inf, so the weights
    of an atom sum to one.  Slices that do not meet [z - 6 sigma, z + 6 sigma]
    get exactly 0.
    """
    n = g.n_slices
    edges = g.z0 + g.dz * np.arange(n + 1, dtype=np.float64)
    cdf = 0.5 * erf((edges - z) / (np.sqrt(2.0) * sigma))
    cdf[0] = -0.5
    cdf[n] = 0.5
    w = cdf[1:] - cdf[:-1]
    lo = edges[:-1].copy()
    hi = edges[1:].copy()
    lo[0] = -np.inf
    hi[n - 1] = np.inf
    rc = 6.0 * sigma
    touch = (hi > z - rc) & (lo < z + rc)
    w[~touch] = 0.0
    return w


def projected_potential(g: Grid, pos, species, amp_sigma) -> np.ndarray:
    """Slice potentials v_s(x_i, y_j) in V*Angstrom, shape (n_slices, ny, nx).

    v_s(r) = sum_a amp_a exp(-|r - R_a|^2 / (2 s_a^2)) w_s(z_a) over atoms
    whose minimum-image offsets satisfy |dx|, |dy| <= 6 s_a; pixel centres are
    x_i = i * lx / nx, y_j = j * ly / ny.  Each atom is evaluated on the
    small window of pixels that can lie within its cut-off.
    """
    pos = np.asarray(pos, dtype=np.float64)
    species = np.asarray(species)
    amp_sigma = np.asarray(amp_sigma, dtype=np.float64).reshape(-1, 2)
    dx, dy = g.lx / g.nx, g.ly / g.ny
    v = np.zeros((g.n_slices, g.ny * g.nx), dtype=np.float64)
    for sp in range(amp_sigma.shape[0]):
        amp, sig = amp_sigma[sp]
        rc = 6.0 * sig
        p = pos[species == sp]
        if p.shape[0] == 0:
            continue
        w = np.stack([slice_weights(z, sig, g) for z in p[:, 2]])      # (Na, n_s)
        wx = int(np.floor(2.0 * rc / dx)) + 2
        wy = int(np.floor(2.0 * rc / dy)) + 2
        i0 = np.ceil((p[:, 0] - rc) / dx).astype(np.int64)
        j0 = np.ceil((p[:, 1] - rc) / dy).astype(np.int64)
        ii = i0[:, None] + np.arange(wx)[None, :]                       # (Na, wx)
        jj = j0[:, None] + np.arange(wy)[None, :]
        ddx = ii * dx - p[:, 0:1]
        ddy = jj * dy - p[:, 1:2]
        r2 = ddx[:, None, :] ** 2 + ddy[:, :, None] ** 2               # (Na, wy, wx)
        inside = (np.abs(ddx)[:, None, :] <= rc) & (np.abs(ddy)[:, :, None] <= rc)
        gauss = amp * np.exp(-r2 / (2.0 * sig * sig)) * inside
        flat = (np.mod(jj, g.ny)[:, :, None] * g.nx + np.mod(ii, g.nx)[:, None, :])
        for s in np.nonzero(np.any(w != 0.0, axis=0))[0]:
            contrib = gauss * w[:, s][:, None, None]
            v[s] += np.bincount(flat.ravel(), weights=contrib.ravel(), minlength=g.nx * g.ny)
    return v.reshape(g.n_slices, g.ny, g.nx)


def projected_potential_bruteforce(g: Grid, pos, species, amp_sigma) -> np.ndarray:
    """Same definition evaluated on every pixel for every atom (tiny inputs only)."""
    pos = np.asarray(pos, dtype=np.float64)
    amp_sigma = np.asarray(amp_sigma, dtype=np.float64).reshape(-1, 2)
    x = np.arange(g.nx) * (g.lx / g.nx)
    y = np.arange(g.ny) * (g.ly / g.ny)
    v = np.zeros((g.n_slices, g.ny, g.nx))
    for a in range(pos.shape[0]):
        amp, sig = amp_sigma[int(species[a])]
        ddx = np.mod(x - pos[a, 0] + g.lx / 2.0, g.lx) - g.lx / 2.0
        ddy = np.mod(y - pos[a, 1] + g.ly / 2.0, g.ly) - g.ly / 2.0
        r2 = ddx[None, :] ** 2 + ddy[:, None] ** 2
        inside = (np.abs(ddx)[None, :] <= 6.0 * sig) & (np.abs(ddy)[:, None] <= 6.0 * sig)
        prof = amp * np.exp(-r2 / (2.0 * sig * sig)) * inside
        w = slice_weights(pos[a, 2], sig, g)
        v += w[:, None, None] * prof[None]
    return v


# ---------------------------------------------------------------------------
# Multislice.
# ---------------------------------------------------------------------------
def spatial_frequencies(g: Grid):
    """q_x (nx,), q_y (ny,) in 1/Angstrom, FFT order (numpy fftfreq)."""
    return np.fft.fftfreq(g.nx, d=g.lx / g.nx), np.fft.fftfreq(g.ny, d=g.ly / g.ny)


def bandlimit_mask(g: Grid) -> np.ndarray:
    """1 where |q| <= bandlimit * q_Nyquist, q_Nyquist = min(nx/2lx, ny/2ly)."""
    qx, qy = spatial_frequencies(g)
    q2 = qx[None, :] ** 2 + qy[:, None] ** 2
    qmax = g.bandlimit * min(g.nx / (2.0 * g.lx), g.ny / (2.0 * g.ly))
    return (q2 <= qmax * qmax).astype(np.float64)


def propagator(g: Grid) -> np.ndarray:
    """Band-limited Fresnel propagator exp(-i pi lambda dz |q|^2) * BL(q)."""
    qx, qy = spatial_frequencies(g)
    q2 = qx[None, :] ** 2 + qy[:, None] ** 2
    lam = wavelength(g.kev)
    return np.exp(-1j * np.pi * lam * g.dz * q2) * bandlimit_mask(g)


def fft2_unitary(psi: np.ndarray) -> np.ndarray:
    """Psi(q) = (1/(nx ny)) sum_r psi(r) exp(-2 pi i q.r) over the last two axes."""
    n = psi.shape[-1] * psi.shape[-2]
    return np.fft.fft2(psi) / n


def ifft2_unitary(psi_q: np.ndarray) -> np.ndarray:
    """psi(r) = sum_q Psi(q) exp(+2 pi i q.r) (no 1/N factor)."""
    n = psi_q.shape[-1] * psi_q.shape[-2]
    return np.fft.ifft2(psi_q) * n


def multislice(g: Grid, v: np.ndarray, psi_in=None) -> np.ndarray:
    """Exit wave in q-space (FFT order) of one snapshot with slice potentials v.

    psi_0 = psi_in (real space) or the unit plane wave; for every slice:
    chi = exp(i sigma_e v_s) psi_s; Chi = F2[chi]; Chi' = P BL Chi;
    psi_{s+1} = F2^-1[Chi'].  The exit wave is Chi' of the last slice.
    """
    sig = interaction_constant(g.kev)
    prop = propagator(g)
    psi = np.ones((g.ny, g.nx), dtype=np.complex128) if psi_in is None \
        else np.asarray(psi_in, dtype=np.complex128).copy()
    out = None
    for s in range(g.n_slices):
        chi = np.exp(1j * sig * v[s]) * psi
        out = prop * fft2_unitary(chi)
        if s + 1 < g.n_slices:
            psi = ifft2_unitary(out)
    return out


def _exit_wave_one(args):
    g, p, species, amp_sigma, psi_in = args
    return multislice(g, projected_potential(g, p, species, amp_sigma), psi_in)


def exit_waves(g: Grid, pos, species, amp_sigma, psi_in=None, processes=None) -> np.ndarray:
    """Exit waves psi(q, t) for every snapshot, shape (T, ny, nx) complex128.

    ``processes`` > 1 spreads snapshots over a spawn-started process pool
    (the computation per snapshot is unchanged).
    """
    pos = np.asarray(pos)
    jobs = [(g, pos[t], species, amp_sigma, psi_in) for t in range(pos.shape[0])]
    if processes is not None and processes > 1 and len(jobs) > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(processes) as pool:
            waves = pool.map(_exit_wave_one, jobs, chunksize=1)
    else:
        waves = [_exit_wave_one(j) for j in jobs]
    return np.stack(waves)


# ---------------------------------------------------------------------------
# Spectrum: elastic removal, temporal transform, power, Kubo, normalisation.
# ---------------------------------------------------------------------------
def natural_energies(n_t: int, dt_fs: float) -> np.ndarray:
    """E_k = h k / (T dt) in meV for k = -T/2 .. T/2-1 (fftshift order)."""
    return np.fft.fftshift(np.fft.fftfreq(n_t, d=dt_fs)) * H_MEV_FS


def time_mean(psi: np.ndarray) -> np.ndarray:
    """m_q = (1/T) sum_t psi(q, t); psi has shape (T, ...)."""
    return np.mean(np.asarray(psi, dtype=np.complex128), axis=0)


def temporal_transform(a: np.ndarray, dt_fs: float, omega_meV=None) -> np.ndarray:
    """Phi(q, E_k) = sum_n a(q, t_n) exp(-i E_k t_n / hbar), t_n = n dt.

    a has shape (T, nq); returns (nq, n_omega).  With omega_meV None the
    natural grid is used (FFT over time, reordered to ascending E);
    otherwise an explicit FP64 DFT matrix is applied.
    """
    a = np.asarray(a, dtype=np.complex128)
    n_t = a.shape[0]
    if omega_meV is None:
        return np.fft.fftshift(np.fft.fft(a, axis=0), axes=0).T.copy()
    e = np.asarray(omega_meV, dtype=np.float64)
    t = np.arange(n_t, dtype=np.float64) * dt_fs
    dft = np.exp(-1j * np.outer(t, e) / HBAR_MEV_FS)          # (T, n_omega)
    return a.T @ dft


def kubo_factor(e_meV, temperature_K: float) -> np.ndarray:
    """beta E / (1 - exp(-beta E)) (Eq. (8)); equals 1 at E = 0."""
    e = np.asarray(e_meV, dtype=np.float64)
    be = e / (KB_MEV_PER_K * temperature_K)
    out = np.ones_like(be)
    nz = be != 0.0
    out[nz] = be[nz] / (-np.expm1(-be[nz]))
    return out


def spectrum(psi, dt_fs: float, omega_meV=None, kubo=False, temperature_K=300.0,
             normalize=False):
    """I(q, E) and I_el(q) from exit waves psi of shape (T, nq) (or (T, ny, nx)).

    I(q, E_k) = |Phi(q, E_k)|^2 / T^2 with Phi the temporal transform of
    psi - mean_t psi; I_el(q) = |mean_t psi|^2.  ``kubo`` multiplies by the
    detailed-balance factor; ``normalize`` scales I and I_el together so that
    sum_{q,k} I + sum_q I_el = 1 on the numerical grid.
    Returns (I (nq, n_omega), I_el (nq,), E (n_omega,) in meV).
    """
    psi = np.asarray(psi, dtype=np.complex128)
    n_t = psi.shape[0]
    psi = psi.reshape(n_t, -1)
    m = time_mean(psi)
    i_el = np.abs(m) ** 2
    phi = temporal_transform(psi - m[None, :], dt_fs, omega_meV)
    inten = np.abs(phi) ** 2 / float(n_t) ** 2
    energies = natural_energies(n_t, dt_fs) if omega_meV is None \
        else np.asarray(omega_meV, dtype=np.float64)
    if kubo:
        inten = inten * kubo_factor(energies, temperature_K)[None, :]
    if normalize:
        total = inten.sum() + i_el.sum()
        inten = inten / total
        i_el = i_el / total
    return inten, i_el, energies


# ---------------------------------------------------------------- segments
def segment_count(n_t: int, seg_len: int, hop: int) -> int:
    """Largest number of sets of seg_len consecutive snapshots, starts 0, hop, 2 hop, ..."""
    if seg_len > n_t or seg_len < 1 or hop < 1:
        return 0
    return (n_t - seg_len) // hop + 1


def segment_starts(n_t: int, seg_len: int, hop: int, n_sets=None) -> np.ndarray:
    """First snapshot of each set: g * hop for g = 0 .. n_sets - 1 (all sets that fit
    when n_sets is None)."""
    most = segment_count(n_t, seg_len, hop)
    n = most if n_sets is None else int(n_sets)
    if n < 1 or n > most:
        raise ValueError("need 1 <= n_sets <= the number of complete sets")
    return np.arange(n) * hop


def segment_spectrum(psi, dt_fs: float, seg_len: int, hop: int, n_sets=None, omega_meV=None,
                     kubo=False, temperature_K=300.0, normalize=False):
    """Spectrum averaged over sets of consecutive snapshots (the averaging over
    trajectory segments the paper describes after Eq. (9) and applies with,
    e.g., 79 sets of 100 snapshots offset by 50).

    Set g holds snapshots g*hop .. g*hop + seg_len - 1 and is treated as a
    trajectory of its own: its time mean m_g, elastic part |m_g|^2 and
    I_g(q, E) = |sum_n (psi - m_g)(q, t_n) exp(-i E t_n / hbar)|^2 / seg_len^2
    with t_n measured from the start of the set (the start time only adds a
    phase).  I and I_el are the plain averages over the sets; the Kubo factor
    and the normalisation then act on the averages as in ``spectrum``.
    Natural grid (omega_meV None): E_k = h k / (seg_len dt).
    Returns (I (nq, n_omega), I_el (nq,), E (n_omega,) in meV).
    """
    psi = np.asarray(psi, dtype=np.complex128)
    n_t = psi.shape[0]
    psi = psi.reshape(n_t, -1)
    starts = segment_starts(n_t, seg_len, hop, n_sets)
    inten = 0.0
    i_el = 0.0
    for g0 in starts:
        i_g, iel_g, energies = spectrum(psi[g0:g0 + seg_len], dt_fs, omega_meV)
        inten = inten + i_g
        i_el = i_el + iel_g
    inten = inten / len(starts)
    i_el = i_el / len(starts)
    if kubo:
        inten = inten * kubo_factor(energies, temperature_K)[None, :]
    if normalize:
        total = inten.sum() + i_el.sum()
        inten = inten / total
        i_el = i_el / total
    return inten, i_el, energies


# ---------------------------------------------------------------- QEP by-products
def qep_intensity(psi, t0: int = 0, stride: int = 1, n=None) -> np.ndarray:
    """QEP diffraction pattern of a subset of snapshots (Eq. (4) with Eq. (3):
    |psi|^2 averaged over configurations): (1/n) sum_j |psi(q, t0 + j stride)|^2.
    psi has shape (T, ...); n None takes every snapshot t0, t0 + stride, ... < T."""
    psi = np.asarray(psi, dtype=np.complex128)
    idx = np.arange(t0, psi.shape[0], stride)
    if n is not None:
        if n < 1 or n > len(idx):
            raise ValueError("the snapshots do not fit")
        idx = idx[:n]
    return np.mean(np.abs(psi[idx]) ** 2, axis=0)


def energy_integral(inten, i_el=None) -> np.ndarray:
    """sum_k I(q, E_k) (+ I_el(q)): the energy integral of the spectrum."""
    out = np.sum(np.asarray(inten, dtype=np.float64), axis=1)
    return out if i_el is None else out + np.asarray(i_el, dtype=np.float64)


def scattering_angles(nx: int, ny: int, lx: float, ly: float, lam: float) -> np.ndarray:
    """theta = lambda |q| in mrad on the FFT-order grid (ny, nx)."""
    qx = np.fft.fftfreq(nx, d=lx / nx)
    qy = np.fft.fftfreq(ny, d=ly / ny)
    return lam * np.sqrt(qx[None, :] ** 2 + qy[:, None] ** 2) * 1000.0


def line_profile(values, lx: float, lam: float):
    """Profile of values (ny, nx) (FFT order) along q_y = 0, in ascending
    theta_x = lambda q_x; returns (line (nx,), theta_x (nx,) in mrad)."""
    values = np.asarray(values, dtype=np.float64)
    nx = values.shape[1]
    order = np.fft.fftshift(np.arange(nx))
    qx = np.fft.fftfreq(nx, d=lx / nx)
    return values[0, order], lam * qx[order] * 1000.0


def azimuthal_profile(values, lx: float, ly: float, lam: float, dtheta: float, n_bins: int):
    """Mean of values (ny, nx) (FFT order) over the q with theta in
    [b dtheta, (b+1) dtheta), b < n_bins (0 for an empty bin); returns
    (profile (n_bins,), counts (n_bins,))."""
    values = np.asarray(values, dtype=np.float64)
    ny, nx = values.shape
    b = np.floor(scattering_angles(nx, ny, lx, ly, lam) / dtheta).ravel()
    keep = b < n_bins
    counts = np.bincount(b[keep].astype(int), minlength=n_bins)
    sums = np.bincount(b[keep].astype(int), weights=values.ravel()[keep], minlength=n_bins)
    prof = np.where(counts > 0, sums / np.maximum(counts, 1), 0.0)
    return prof, counts


def relative_difference(a, b) -> np.ndarray:
    """(a - b) / (a + b), 0 where a + b = 0 (the paper's difference divided by sum)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    s = a + b
    return np.where(s != 0.0, (a - b) / np.where(s != 0.0, s, 1.0), 0.0)


# ---------------------------------------------------------------- convergent probe
def probe(g: Grid, alpha_mrad: float, defocus_A: float = 0.0, x0: float = 0.0, y0: float = 0.0) -> np.ndarray:
    """Real-space incident wave of a convergent probe (the 1 mrad convergence
    semi-angle set-up of the paper's Fe simulation), shape (ny, nx) complex128.

    Psi(q) = exp(-i pi lambda defocus |q|^2) exp(-2 pi i q.r_p) / sqrt(N_ap)
    for the N_ap grid points with theta = lambda |q| <= alpha (FP64, theta in
    mrad as lambda * sqrt(qx^2 + qy^2) * 1000), 0 elsewhere; psi(r) is its
    inverse transform without 1/N, so mean_r |psi|^2 = sum_q |Psi|^2 = 1 like
    the unit plane wave.  A positive defocus equals free propagation by that
    distance with the multislice propagator's sign.
    """
    qx, qy = spatial_frequencies(g)
    lam = wavelength(g.kev)
    theta = lam * np.sqrt(qx[None, :] ** 2 + qy[:, None] ** 2) * 1000.0
    inside = theta <= alpha_mrad
    n_ap = int(np.count_nonzero(inside))
    if n_ap == 0:
        raise ValueError("no grid point inside the aperture")
    q2 = qx[None, :] ** 2 + qy[:, None] ** 2
    phase = -np.pi * lam * defocus_A * q2 - 2.0 * np.pi * (qx[None, :] * x0 + qy[:, None] * y0)
    psi_q = np.where(inside, np.exp(1j * phase), 0.0) / np.sqrt(n_ap)
    return ifft2_unitary(psi_q)
