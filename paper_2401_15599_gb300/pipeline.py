"""Time-to-spectrum driver: positions on the device -> I(q, E) on the device.

Chains the three C-ABI calls the way the paper's procedure does (after
Eq. (9)): for each batch of snapshots build the slice potentials and run
the multislice into the exit-wave set psi(q, t); then the temporal
transform.  All buffers and workspaces are allocated once in ``__init__``,
so ``run`` only enqueues kernels on the current stream.
"""

from __future__ import annotations

import torch

from . import api


class TimeToSpectrum:
    def __init__(self, grid, n_t, n_atoms, amp_sigma, dt_fs, batch=32, omega_meV=None,
                 precision="fp32", kubo=False, temperature_K=300.0, normalize=False,
                 device="cuda"):
        self.grid = grid
        self.n_t = int(n_t)
        self.n_atoms = int(n_atoms)
        self.amp_sigma = amp_sigma
        self.dt_fs = float(dt_fs)
        if batch == "auto":                     # tuned per grid and GPU, cached (tuning.py)
            from .tuning import best_multislice_batch
            batch = best_multislice_batch(grid, device=device)
        self.batch = max(1, min(int(batch), self.n_t))
        self.precision = precision
        self.kubo = kubo
        self.temperature_K = temperature_K
        self.normalize = normalize
        self.device = torch.device(device)
        g = grid
        self.omega = None if omega_meV is None else \
            torch.as_tensor(omega_meV, dtype=torch.float64, device=self.device)
        n_w = self.n_t if self.omega is None else self.omega.numel()
        nq = g.nx * g.ny
        self.psi = torch.empty((self.n_t, g.ny, g.nx), dtype=torch.complex64, device=self.device)
        self.psi_sum = torch.zeros((g.ny, g.nx), dtype=torch.complex128, device=self.device)
        self.V = torch.empty((self.batch, g.n_slices, g.ny, g.nx), dtype=torch.float32, device=self.device)
        self.I = torch.empty((nq, n_w), dtype=torch.float32, device=self.device)
        self.I_el = torch.empty(nq, dtype=torch.float64, device=self.device)
        self._ws = {}

    def _workspace(self, key, nbytes):
        ws = self._ws.get(key)
        if ws is None or ws.numel() < nbytes:
            ws = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=self.device)
            self._ws[key] = ws
        return ws

    def exit_waves(self, pos, species):
        """Potential + multislice for every snapshot of pos [T, Na, 3] into self.psi."""
        self.psi_sum.zero_()
        for t0 in range(0, self.n_t, self.batch):
            t1 = min(self.n_t, t0 + self.batch)
            v = self.V[: t1 - t0]
            api.potential(self.grid, pos[t0:t1], species, self.amp_sigma, out=v,
                          workspace=self._ws.get("pot"))
            api.multislice(self.grid, v, out=self.psi[t0:t1], psi_sum=self.psi_sum,
                           workspace=self._ws.get("ms"))
        return self.psi

    def spectrum(self):
        return api.spectrum(self.psi.reshape(self.n_t, -1), self.dt_fs, omega_meV=self.omega,
                            psi_sum=self.psi_sum.reshape(-1), precision=self.precision,
                            kubo=self.kubo, temperature_K=self.temperature_K,
                            normalize=self.normalize, out=self.I, i_el=self.I_el,
                            workspace=self._ws.get("spec"))

    def prepare(self, pos, species):
        """Size the workspaces once (one untimed run fills the cache)."""
        import ctypes
        from . import _lib as L
        lib = L.load()
        g = L.make_grid(self.grid)
        n = ctypes.c_size_t(0)
        amp = torch.as_tensor(self.amp_sigma, dtype=torch.float32).reshape(-1, 2)
        amp_c = (ctypes.c_float * amp.numel())(*amp.flatten().tolist())
        null = ctypes.c_void_p(0)
        L.check("tacaw_potential", lib.tacaw_potential(ctypes.byref(g), self.batch, self.n_atoms, null, null,
                                                       amp.shape[0], amp_c, null, null, ctypes.byref(n), null))
        self._workspace("pot", n.value)
        L.check("tacaw_multislice", lib.tacaw_multislice(ctypes.byref(g), self.batch, null, null, null, null, 0,
                                                         null, ctypes.byref(n), null))
        self._workspace("ms", n.value)
        n_w = self.n_t if self.omega is None else self.omega.numel()
        need = 0
        precs = [L.TACAW_FP32, L.TACAW_BF16X3]
        if self.omega is None and self.n_t in L.TIME_FFT_SIZES:
            precs.append(L.TACAW_FFT32)
        if self.precision == "bf16x6":
            precs.append(L.TACAW_BF16X6)
        for prec in precs:                               # one workspace serves every precision
            L.check("tacaw_spectrum", lib.tacaw_spectrum(self.grid.nx * self.grid.ny, self.n_t, self.dt_fs, n_w,
                                                         null, null, ctypes.c_void_p(1), null, ctypes.c_void_p(1),
                                                         prec, 0, 300.0, null, ctypes.byref(n), null))
            need = max(need, n.value)
        self._workspace("spec", need)

    def run(self, pos, species):
        self.exit_waves(pos, species)
        return self.spectrum()
