"""Crystals and classical harmonic trajectories (stand-in for the MD step).

The paper obtains its snapshots from molecular dynamics (Sec. "procedure",
first step) and notes that the time-correlation approach is exact for a
harmonic crystal.  Synthetic trajectories here are sums of plane-wave
harmonic modes, commensurate with the periodic supercell:

    u_a(t) = sum_j a_j e_j cos(k_j . R_a - Omega_j t + phi_j)

Every random number comes from ``numpy.random.default_rng(seed)`` in a fixed
draw order, so a seed fixes the trajectory bit for bit on any host.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# CODATA 2018 values used only to turn mode energies into angular
# frequencies and temperatures into classical amplitudes.
HBAR_MEV_FS = 658.2119569509067      # reduced Planck constant, meV*fs
KB_MEV_PER_K = 0.08617333262         # Boltzmann constant, meV/K
AMU_KG = 1.66053906660e-27           # atomic mass unit, kg
EV_J = 1.602176634e-19               # electron volt, J


@dataclass(frozen=True)
class Crystal:
    """Equilibrium structure of a periodic supercell.

    positions: (Na, 3) float64, Angstrom, inside [0, cell).
    species:   (Na,) int32 species index per atom.
    cell:      (3,) float64 supercell lengths (Lx, Ly, Lz), Angstrom.
    mass_u:    atomic mass in u (used only for classical amplitudes).
    """

    positions: np.ndarray
    species: np.ndarray
    cell: np.ndarray
    mass_u: float

    @property
    def n_atoms(self) -> int:
        return int(self.positions.shape[0])


def _lattice(ncell, a, basis) -> np.ndarray:
    nx, ny, nz = ncell
    basis = np.asarray(basis, dtype=np.float64)
    # x fastest, then basis, then y, then z: a stable, documented order.
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    origins = np.stack([i, j, k], axis=-1).reshape(-1, 3).astype(np.float64)
    pos = (origins[:, None, :] + basis[None, :, :]).reshape(-1, 3) * a
    return pos


def simple_cubic(ncell=(8, 8, 8), a=4.0, mass_u=26.98, n_species=1, rng=None) -> Crystal:
    """Simple-cubic supercell, one atom per cell at a*(i, j, k)."""
    pos = _lattice(ncell, a, [[0.0, 0.0, 0.0]])
    species = _assign_species(pos.shape[0], n_species, rng)
    return Crystal(pos, species, np.asarray(ncell, dtype=np.float64) * a, mass_u)


def fcc(ncell=(20, 20, 50), a=4.05, mass_u=26.98, n_species=1, rng=None) -> Crystal:
    """Face-centred-cubic supercell, four atoms per conventional cell."""
    basis = [[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]]
    pos = _lattice(ncell, a, basis)
    species = _assign_species(pos.shape[0], n_species, rng)
    return Crystal(pos, species, np.asarray(ncell, dtype=np.float64) * a, mass_u)


def _assign_species(n_atoms, n_species, rng) -> np.ndarray:
    if n_species <= 1:
        return np.zeros(n_atoms, dtype=np.int32)
    if rng is None:
        raise ValueError("several species need an rng to assign them")
    return rng.integers(0, n_species, size=n_atoms).astype(np.int32)


@dataclass(frozen=True)
class HarmonicModes:
    """A set of M plane-wave harmonic modes.

    n:        (M, 3) integer wave-vector indices, k = 2*pi*n/cell.
    k:        (M, 3) wave vectors, 1/Angstrom.
    e:        (M, 3) unit polarisation vectors.
    amp:      (M,) amplitudes a_j, Angstrom.
    energy:   (M,) mode energies hbar*Omega_j, meV.
    phase:    (M,) phases phi_j, rad.
    """

    n: np.ndarray
    k: np.ndarray
    e: np.ndarray
    amp: np.ndarray
    energy: np.ndarray
    phase: np.ndarray

    @property
    def omega(self) -> np.ndarray:
        """Angular frequencies Omega_j in rad/fs."""
        return self.energy / HBAR_MEV_FS


def draw_modes(rng, cell, energies_meV, amps, n_lo, n_hi) -> HarmonicModes:
    """Draw modes with integer indices n_c in [n_lo[c], n_hi[c]) (never all zero).

    Draw order (fixed): wave-vector indices, then polarisations, then phases.
    """
    energies = np.asarray(energies_meV, dtype=np.float64)
    m = energies.shape[0]
    amps = np.broadcast_to(np.asarray(amps, dtype=np.float64), (m,)).copy()
    n = np.zeros((m, 3), dtype=np.int64)
    for j in range(m):
        while True:
            cand = np.array([rng.integers(n_lo[c], n_hi[c]) for c in range(3)], dtype=np.int64)
            if np.any(cand != 0):
                n[j] = cand
                break
    e = rng.standard_normal((m, 3))
    e /= np.linalg.norm(e, axis=1, keepdims=True)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=m)
    k = 2.0 * np.pi * n / np.asarray(cell, dtype=np.float64)[None, :]
    return HarmonicModes(n, k, e, amps, energies, phase)


def classical_amplitudes(energies_meV, mass_u, temperature_K, n_modes=None) -> np.ndarray:
    """Classical equipartition amplitudes a_j = sqrt(2 kB T * 3 / (M Omega_j^2 n_modes)).

    With these, the per-atom mean-square displacement sum_j a_j^2/2 equals
    3 kB T / M * mean(1/Omega^2), as for a crystal with that frequency spread.
    """
    energies = np.asarray(energies_meV, dtype=np.float64)
    n_modes = energies.shape[0] if n_modes is None else n_modes
    kt_j = KB_MEV_PER_K * temperature_K * 1e-3 * EV_J
    omega_s = energies / HBAR_MEV_FS * 1e15
    mass = mass_u * AMU_KG
    a2_m2 = 2.0 * kt_j * 3.0 / (mass * omega_s**2 * n_modes)
    return np.sqrt(a2_m2) * 1e10


def positions(crystal: Crystal, modes: HarmonicModes, t_fs, dtype=np.float32,
              chunk_t=256, chunk_a=1 << 16) -> np.ndarray:
    """Positions R_a + u_a(t_n) for every time in t_fs, shape (T, Na, 3).

    cos(theta - Omega t) is expanded as cos(theta)cos(Omega t) +
    sin(theta)sin(Omega t), so each chunk is one real FP64 matrix product.
    """
    t = np.asarray(t_fs, dtype=np.float64)
    nt = t.shape[0]
    na = crystal.n_atoms
    out = np.empty((nt, na, 3), dtype=dtype)
    w = modes.omega
    for a0 in range(0, na, chunk_a):
        a1 = min(na, a0 + chunk_a)
        r = crystal.positions[a0:a1]
        theta = r @ modes.k.T + modes.phase[None, :]               # (na_c, M)
        ae = modes.amp[:, None] * modes.e                          # (M, 3)
        c = np.cos(theta).T[:, :, None] * ae[:, None, :]           # (M, na_c, 3)
        s = np.sin(theta).T[:, :, None] * ae[:, None, :]
        coef = np.concatenate([c, s], axis=0).reshape(2 * w.shape[0], -1)
        for t0 in range(0, nt, chunk_t):
            t1 = min(nt, t0 + chunk_t)
            wt = np.outer(t[t0:t1], w)
            z = np.concatenate([np.cos(wt), np.sin(wt)], axis=1)      # (Tc, 2M)
            u = (z @ coef).reshape(t1 - t0, a1 - a0, 3)
            out[t0:t1, a0:a1] = (r[None, :, :] + u).astype(dtype)
    return out


def static_positions(crystal: Crystal, n_t: int, dtype=np.float32) -> np.ndarray:
    """T identical snapshots of the equilibrium structure."""
    p = crystal.positions.astype(dtype)
    return np.broadcast_to(p[None], (n_t,) + p.shape).copy()


class TrajectorySynth:
    """Positions R_a + u_a(t_n) of a crystal and its harmonic modes synthesised
    with torch on a device, window by window, for trajectories too large to
    hold for every snapshot at once.  The per-atom mode coefficients are staged
    on the device once; a window needs only device work (so it can be recorded
    in a CUDA graph).  Same expansion of cos(theta - Omega t) as ``positions``:
    phases and cos/sin in FP64, the mode sum in FP32, the result float32
    (within two float32 ulps of ``positions``)."""

    def __init__(self, crystal: Crystal, modes: HarmonicModes, dt_fs: float, device="cpu"):
        import torch
        self.device = torch.device(device)
        self.dt = float(dt_fs)
        r = crystal.positions.astype(np.float64)
        theta = r @ modes.k.T + modes.phase[None, :]                       # (Na, M)
        ae = modes.amp[:, None] * modes.e                                  # (M, 3)
        coef = np.concatenate([np.cos(theta)[:, :, None] * ae[None], np.sin(theta)[:, :, None] * ae[None]],
                              axis=1)                                      # (Na, 2M, 3)
        self.coef = torch.as_tensor(coef.transpose(1, 0, 2).reshape(coef.shape[1], -1).astype(np.float32),
                                    device=self.device)                    # (2M, Na * 3)
        self.r = torch.as_tensor(r.reshape(-1), device=self.device)        # (Na * 3,) FP64
        self.w = torch.as_tensor(modes.omega.astype(np.float64), device=self.device)
        self.n_atoms = r.shape[0]

    def __call__(self, t0: int, t1: int, out=None):
        import torch
        t = torch.arange(t0, t1, dtype=torch.float64, device=self.device) * self.dt
        wt = torch.outer(t, self.w)
        z = torch.cat([torch.cos(wt), torch.sin(wt)], dim=1).to(torch.float32)   # (T, 2M)
        u = z @ self.coef                                                          # (T, Na * 3)
        res = (self.r[None, :] + u.to(torch.float64)).to(torch.float32).reshape(t1 - t0, self.n_atoms, 3)
        if out is not None:
            out.copy_(res)
            return out
        return res
