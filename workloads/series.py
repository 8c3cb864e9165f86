"""Seeded exit-wave-like time series for tests of the temporal transform.

Data only: a parametric signal, none of the method's arithmetic.  The series
mimic the structure of exit waves of a vibrating crystal: a few strong beams
(large constant amplitude, like q = 0 and the Bragg beams) and many weak
points, each carrying a small phase modulation by a handful of harmonic
vibrations (which puts loss and gain sidebands, and their multiples, into the
spectrum) plus a weak broadband floor.

    psi(q, t_n) = B_q exp(i theta_q) exp(i sum_j eps_qj cos(Omega_j t_n + phi_qj))
                  + floor_q (N(0, 1) + i N(0, 1)) / sqrt(2)

Draw order from default_rng(seed): beam amplitudes and phases, mode energies
(meV, U[e_lo, e_hi]), per-q depths and phases, then the floor.
"""

from __future__ import annotations

import numpy as np

HBAR_MEV_FS = 6.62607015e-34 / 1.602176634e-19 * 1e3 * 1e15 / (2.0 * np.pi)


def modulated_waves(n_t: int, n_q: int, dt_fs: float, n_strong: int, seed: int, n_modes: int = 12,
                    e_lo: float = 5.0, e_hi: float = 100.0, depth: float = 0.03,
                    floor: float = 2e-5) -> np.ndarray:
    """complex64 [n_t][n_q]: the first n_strong points are strong beams
    (|B| in [0.05, 1], the first one 1), the rest weak (|B| in 1e-4 .. 1e-2)."""
    rng = np.random.default_rng(seed)
    amp = 10.0 ** rng.uniform(-4.0, -2.0, n_q)
    amp[:n_strong] = rng.uniform(0.05, 1.0, n_strong)
    if n_strong > 0:
        amp[0] = 1.0
    theta = rng.uniform(0.0, 2.0 * np.pi, n_q)
    energies = rng.uniform(e_lo, e_hi, n_modes)
    eps = rng.uniform(0.0, depth, (n_q, n_modes))
    phi = rng.uniform(0.0, 2.0 * np.pi, (n_q, n_modes))
    noise = rng.standard_normal((n_t, n_q)) + 1j * rng.standard_normal((n_t, n_q))
    t = np.arange(n_t, dtype=np.float64) * dt_fs
    omega = energies / HBAR_MEV_FS                                  # rad / fs
    out = np.empty((n_t, n_q), dtype=np.complex64)
    for t0 in range(0, n_t, 256):
        t1 = min(n_t, t0 + 256)
        arg = np.cos(t[t0:t1, None, None] * omega[None, None, :] + phi[None, :, :])   # (Tc, q, M)
        mod = np.exp(1j * np.einsum("tqm,qm->tq", arg, eps))
        base = amp * np.exp(1j * theta)
        out[t0:t1] = (base[None, :] * mod + floor * amp[None, :] ** 0.5 * noise[t0:t1] / np.sqrt(2.0))
    return out
