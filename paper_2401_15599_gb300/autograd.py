"""torch.autograd bindings of the hot path (gradient-based fitting).

``spectrum_from_potentials(V, grid, dt)``: I(q, E) from slice potentials
V [T, n_slices, ny, nx]; the backward gives dL/dV.

``spectrum_from_atoms(amp_sigma, pos, species, grid, dt)``: I(q, E) from
per-species Gaussian parameters; the backward gives dL/d(amp, sigma).

Forward and backward run entirely in libtacaw (FP32 multislice and
spectrum); the multislice adjoint recomputes forward waves from
checkpoints every ``ckpt_every`` slices (default ceil(sqrt(n_slices))).
Snapshots are processed in batches of ``batch`` to bound memory.
"""

from __future__ import annotations

import torch

from . import api


def _forward_waves(grid, V, batch):
    n_t = V.shape[0]
    psi = torch.empty((n_t, grid.ny, grid.nx), dtype=torch.complex64, device=V.device)
    for t0 in range(0, n_t, batch):
        api.multislice(grid, V[t0:t0 + batch], out=psi[t0:t0 + batch])
    return psi


class _FromPotentials(torch.autograd.Function):
    @staticmethod
    def forward(ctx, V, grid, dt_fs, omega_meV, batch, ckpt_every):
        V = V.detach().contiguous()
        psi = _forward_waves(grid, V, batch)
        inten, _ = api.spectrum(psi.reshape(psi.shape[0], -1), dt_fs, omega_meV=omega_meV)
        ctx.save_for_backward(V, psi)
        ctx.cfg = (grid, dt_fs, omega_meV, batch, ckpt_every)
        return inten

    @staticmethod
    def backward(ctx, dl_di):
        V, psi = ctx.saved_tensors
        grid, dt_fs, omega_meV, batch, ckpt_every = ctx.cfg
        g_psi = api.spectrum_backward(psi.reshape(psi.shape[0], -1), dt_fs, dl_di.contiguous().float(),
                                      omega_meV=omega_meV).reshape(psi.shape)
        dv = torch.empty_like(V)
        for t0 in range(0, V.shape[0], batch):
            api.multislice_backward(grid, V[t0:t0 + batch], g_psi[t0:t0 + batch].contiguous(),
                                    ckpt_every=ckpt_every, out=dv[t0:t0 + batch])
        return dv, None, None, None, None, None


class _FromAtoms(torch.autograd.Function):
    @staticmethod
    def forward(ctx, amp_sigma, pos, species, grid, dt_fs, omega_meV, batch, ckpt_every):
        asg = amp_sigma.detach().to("cpu", torch.float32)
        n_t = pos.shape[0]
        psi = torch.empty((n_t, grid.ny, grid.nx), dtype=torch.complex64, device=pos.device)
        for t0 in range(0, n_t, batch):
            v = api.potential(grid, pos[t0:t0 + batch], species, asg)
            api.multislice(grid, v, out=psi[t0:t0 + batch])
        inten, _ = api.spectrum(psi.reshape(n_t, -1), dt_fs, omega_meV=omega_meV)
        ctx.save_for_backward(pos, species, psi)
        ctx.cfg = (asg, grid, dt_fs, omega_meV, batch, ckpt_every, amp_sigma.dtype, amp_sigma.device)
        return inten

    @staticmethod
    def backward(ctx, dl_di):
        pos, species, psi = ctx.saved_tensors
        asg, grid, dt_fs, omega_meV, batch, ckpt_every, dtype, device = ctx.cfg
        n_t = pos.shape[0]
        g_psi = api.spectrum_backward(psi.reshape(n_t, -1), dt_fs, dl_di.contiguous().float(),
                                      omega_meV=omega_meV).reshape(psi.shape)
        grad = torch.zeros(asg.shape, dtype=torch.float64, device=pos.device)
        for t0 in range(0, n_t, batch):
            p = pos[t0:t0 + batch]
            v = api.potential(grid, p, species, asg)
            dv = api.multislice_backward(grid, v, g_psi[t0:t0 + batch].contiguous(), ckpt_every=ckpt_every)
            grad += api.potential_backward(grid, p, species, asg, dv)
        return grad.to(device=device, dtype=dtype), None, None, None, None, None, None, None


def spectrum_from_potentials(V, grid, dt_fs, omega_meV=None, batch=64, ckpt_every=0):
    return _FromPotentials.apply(V, grid, dt_fs, omega_meV, batch, ckpt_every)


def spectrum_from_atoms(amp_sigma, pos, species, grid, dt_fs, omega_meV=None, batch=64, ckpt_every=0):
    return _FromAtoms.apply(amp_sigma, pos, species, grid, dt_fs, omega_meV, batch, ckpt_every)
