"""FP64 adjoint of the TACAW hot path -- TEST INFRASTRUCTURE (see oracle/__init__).

Gradients follow PyTorch's convention for complex quantities: the gradient
of a real loss L with respect to z is dL/dRe z + i dL/dIm z, so that
dL = Re(conj(g_z) dz).  For a linear map y = M x the gradient is pulled back
as g_x = M^H g_y.

Step by step, reversing the forward of ``tacaw_oracle``:

* power: I = |Phi|^2 / T^2                 -> g_Phi = (2 / T^2) dL/dI Phi
* transform: Phi = sum_n A_n e^{-i E t_n / hbar} -> g_A(n) = sum_k g_Phi(k) e^{+i E_k t_n / hbar}
* centring: A = psi - mean_t psi           -> g_psi = g_A - mean_t g_A (self-adjoint)
* propagation: Y = P BL X                  -> g_X = conj(P BL) g_Y
* forward FFT: X = F chi / N^2             -> g_chi = F^H g_X / N^2
* transmission: chi = e^{i sigma v} psi    -> g_psi = e^{-i sigma v} g_chi,
                                              g_v = sigma Im(g_chi conj(chi))
* inverse FFT: psi_{s+1} = F^H Y_s         -> g_Y_s = F g_psi_{s+1}
* potential: v_s = sum_a amp_a G_a w_s(z_a) -> dL/d(amp, sigma) by the chain rule
  (the 6-sigma cut-offs are held fixed: their motion moves terms below e^-18).

The fitting loss of the differentiation workload is
L = sum w (I - I_tgt)^2 / sum w I_tgt^2, with w = 1 inside the band limit
and away from E = 0.
"""

from __future__ import annotations

import numpy as np
from scipy.special import erf

from .tacaw_oracle import (HBAR_MEV_FS, Grid, bandlimit_mask, fft2_unitary, ifft2_unitary,
                           interaction_constant, natural_energies, propagator, slice_weights,
                           temporal_transform, time_mean)

__all__ = ["spectrum_backward", "multislice_forward_states", "multislice_backward",
           "potential_backward", "loss", "loss_grad", "loss_weights"]


def _dft_matrix(n_t, dt_fs, omega_meV):
    e = natural_energies(n_t, dt_fs) if omega_meV is None else np.asarray(omega_meV, dtype=np.float64)
    t = np.arange(n_t, dtype=np.float64) * dt_fs
    return np.exp(-1j * np.outer(t, e) / HBAR_MEV_FS)        # (T, n_omega)


def spectrum_backward(psi, dt_fs, dl_di, omega_meV=None):
    """dL/dpsi (T, nq) given dL/dI (nq, n_omega) for I = |transform(psi - mean)|^2 / T^2."""
    psi = np.asarray(psi, dtype=np.complex128)
    n_t = psi.shape[0]
    psi = psi.reshape(n_t, -1)
    a = psi - time_mean(psi)[None, :]
    phi = temporal_transform(a, dt_fs, omega_meV)            # (nq, n_omega)
    g_phi = (2.0 / float(n_t) ** 2) * np.asarray(dl_di, dtype=np.float64) * phi
    e = _dft_matrix(n_t, dt_fs, omega_meV)
    g_a = (g_phi @ np.conj(e).T).T                           # (T, nq)
    return g_a - g_a.mean(axis=0, keepdims=True)


def multislice_forward_states(g: Grid, v, psi_in=None):
    """Real-space waves psi_s entering every slice, and the exit wave (q-space)."""
    sig = interaction_constant(g.kev)
    prop = propagator(g)
    psi = np.ones((g.ny, g.nx), dtype=np.complex128) if psi_in is None \
        else np.asarray(psi_in, dtype=np.complex128).copy()
    states = []
    out = None
    for s in range(g.n_slices):
        states.append(psi)
        out = prop * fft2_unitary(np.exp(1j * sig * v[s]) * psi)
        if s + 1 < g.n_slices:
            psi = ifft2_unitary(out)
    return states, out


def multislice_backward(g: Grid, v, g_exit, psi_in=None):
    """(dL/dv (n_slices, ny, nx), dL/dpsi_in (ny, nx)) given dL/d(exit wave)."""
    sig = interaction_constant(g.kev)
    prop = propagator(g)
    n = g.nx * g.ny
    states, _ = multislice_forward_states(g, v, psi_in)
    g_v = np.zeros((g.n_slices, g.ny, g.nx))
    g_y = np.asarray(g_exit, dtype=np.complex128)
    g_psi = None
    for s in reversed(range(g.n_slices)):
        g_x = np.conj(prop) * g_y
        g_chi = ifft2_unitary(g_x) / n
        t = np.exp(1j * sig * v[s])
        chi = t * states[s]
        g_v[s] = sig * np.imag(g_chi * np.conj(chi))
        g_psi = np.conj(t) * g_chi
        if s > 0:
            g_y = fft2_unitary(g_psi) * n
    return g_v, g_psi


def _dweight_dsigma(z, sigma, g: Grid):
    """d w_s / d sigma for every slice (0 on the open ends and outside the cut-off)."""
    n = g.n_slices
    edges = g.z0 + g.dz * np.arange(n + 1, dtype=np.float64)
    u = (edges - z) / (np.sqrt(2.0) * sigma)
    dcdf = -(u / sigma) * np.exp(-u * u) / np.sqrt(np.pi)     # d/dsigma of erf(u)/2
    dcdf[0] = 0.0
    dcdf[n] = 0.0
    dw = dcdf[1:] - dcdf[:-1]
    w = slice_weights(z, sigma, g)
    dw[w == 0.0] = 0.0
    return dw


def potential_backward(g: Grid, pos, species, amp_sigma, g_v):
    """dL/d(amp, sigma) per species (n_species, 2) given dL/dv (n_slices, ny, nx)."""
    pos = np.asarray(pos, dtype=np.float64)
    amp_sigma = np.asarray(amp_sigma, dtype=np.float64).reshape(-1, 2)
    x = np.arange(g.nx) * (g.lx / g.nx)
    y = np.arange(g.ny) * (g.ly / g.ny)
    out = np.zeros_like(amp_sigma)
    for a in range(pos.shape[0]):
        sp = int(species[a])
        amp, sig = amp_sigma[sp]
        ddx = np.mod(x - pos[a, 0] + g.lx / 2.0, g.lx) - g.lx / 2.0
        ddy = np.mod(y - pos[a, 1] + g.ly / 2.0, g.ly) - g.ly / 2.0
        r2 = ddx[None, :] ** 2 + ddy[:, None] ** 2
        inside = (np.abs(ddx)[None, :] <= 6.0 * sig) & (np.abs(ddy)[:, None] <= 6.0 * sig)
        prof = np.exp(-r2 / (2.0 * sig * sig)) * inside
        w = slice_weights(pos[a, 2], sig, g)
        dw = _dweight_dsigma(pos[a, 2], sig, g)
        gp = np.einsum("syx,yx->s", g_v, prof)                # sum_pixels g_v * profile
        gpr = np.einsum("syx,yx->s", g_v, prof * r2)
        out[sp, 0] += np.dot(gp, w)
        out[sp, 1] += amp * (np.dot(gpr, w) / sig ** 3 + np.dot(gp, dw))
    return out


def loss_weights(g: Grid, n_omega, e_meV):
    """w(q, E) = 1 inside the band limit and for E != 0, else 0; shape (nq, n_omega)."""
    bl = bandlimit_mask(g).reshape(-1)
    return np.outer(bl, (np.asarray(e_meV) != 0.0).astype(np.float64))


def loss(inten, target, w):
    return float(np.sum(w * (inten - target) ** 2) / np.sum(w * target ** 2))


def loss_grad(inten, target, w):
    return 2.0 * w * (inten - target) / np.sum(w * target ** 2)
