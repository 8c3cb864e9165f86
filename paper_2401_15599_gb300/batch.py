"""Time-to-spectrum for many independent trajectories of uneven size.

Each job has its own grid, slice count, snapshot count and atoms.  Snapshots
are processed in windows: for every window the slice potentials of each job
are built, then one ``tacaw_multislice_batch`` call advances all jobs
together (jobs of the same grid size share launches); finally each job's
spectrum is taken.  ``capture()`` records the whole run in a CUDA graph and
``replay()`` re-runs it with one launch from the host.
"""

from __future__ import annotations

from dataclasses import dataclass

import torch

from . import api


@dataclass
class Job:
    grid: object
    pos: torch.Tensor          # [T, Na, 3] float32, device
    species: torch.Tensor      # [Na] int32, device
    amp_sigma: object          # [n_species][2]
    dt_fs: float
    omega_meV: object = None


class BatchTimeToSpectrum:
    def __init__(self, jobs, window=8, precision="bf16x6", device="cuda"):
        self.jobs = list(jobs)
        if window == "auto":                    # tuned for the largest grid of the jobs (tuning.py)
            from .tuning import best_multislice_batch
            big = max(self.jobs, key=lambda j: j.grid.nx * j.grid.ny * j.grid.n_slices)
            window = best_multislice_batch(big.grid, device=device)
        self.window = int(window)
        self.precision = precision
        self.device = torch.device(device)
        self.state = []
        for j in self.jobs:
            g = j.grid
            n_t = j.pos.shape[0]
            n_w = n_t if j.omega_meV is None else len(j.omega_meV)
            st = {
                "psi": torch.empty((n_t, g.ny, g.nx), dtype=torch.complex64, device=self.device),
                "psi_sum": torch.zeros((g.ny, g.nx), dtype=torch.complex128, device=self.device),
                "V": torch.empty((min(self.window, n_t), g.n_slices, g.ny, g.nx), dtype=torch.float32,
                                 device=self.device),
                "I": torch.empty((g.nx * g.ny, n_w), dtype=torch.float32, device=self.device),
                "I_el": torch.empty(g.nx * g.ny, dtype=torch.float64, device=self.device),
                "omega": None if j.omega_meV is None else
                torch.as_tensor(j.omega_meV, dtype=torch.float64, device=self.device),
            }
            self.state.append(st)
        self.graph = None

    def run(self):
        for st in self.state:
            st["psi_sum"].zero_()
        t_max = max(j.pos.shape[0] for j in self.jobs)
        for t0 in range(0, t_max, self.window):
            batch = []
            for j, st in zip(self.jobs, self.state):
                n_t = j.pos.shape[0]
                if t0 >= n_t:
                    continue
                t1 = min(n_t, t0 + self.window)
                v = st["V"][: t1 - t0]
                api.potential(j.grid, j.pos[t0:t1], j.species, j.amp_sigma, out=v, workspace=st.get("ws_pot"))
                batch.append({"grid": j.grid, "V": v, "out": st["psi"][t0:t1], "psi_sum": st["psi_sum"]})
            api.multislice_batch(batch, workspace=getattr(self, "ws_batch", None))
        for j, st in zip(self.jobs, self.state):
            n_t = j.pos.shape[0]
            api.spectrum(st["psi"].reshape(n_t, -1), j.dt_fs, omega_meV=st["omega"],
                         psi_sum=st["psi_sum"].reshape(-1), precision=self.precision, out=st["I"],
                         i_el=st["I_el"], workspace=st.get("ws_spec"))
        return [(st["I"], st["I_el"]) for st in self.state]

    def prepare(self):
        """Allocate every workspace once (needed before capture)."""
        import ctypes
        from . import _lib as L
        lib = L.load()
        null = ctypes.c_void_p(0)
        for j, st in zip(self.jobs, self.state):
            g = L.make_grid(j.grid)
            n = ctypes.c_size_t(0)
            amp = torch.as_tensor(j.amp_sigma, dtype=torch.float32).reshape(-1, 2)
            amp_c = (ctypes.c_float * amp.numel())(*amp.flatten().tolist())
            L.check("tacaw_potential", lib.tacaw_potential(ctypes.byref(g), st["V"].shape[0], j.pos.shape[1], null,
                                                           null, amp.shape[0], amp_c, null, null, ctypes.byref(n),
                                                           null))
            st["ws_pot"] = torch.empty(max(n.value, 256), dtype=torch.uint8, device=self.device)
            n_t = j.pos.shape[0]
            n_w = st["I"].shape[1]
            prec = {"fp32": L.TACAW_FP32, "bf16x3": L.TACAW_BF16X3, "fft32": L.TACAW_FFT32,
                    "bf16x6": L.TACAW_BF16X6}[self.precision]
            L.check("tacaw_spectrum", lib.tacaw_spectrum(j.grid.nx * j.grid.ny, n_t, float(j.dt_fs), n_w,
                                                         ctypes.c_void_p(1) if st["omega"] is not None else null,
                                                         null, ctypes.c_void_p(1), null, ctypes.c_void_p(1), prec, 0,
                                                         300.0, null, ctypes.byref(n), null))
            st["ws_spec"] = torch.empty(max(n.value, 256), dtype=torch.uint8, device=self.device)
        arr = (L.TacawJob * len(self.jobs))()
        for i, j in enumerate(self.jobs):
            arr[i] = L.TacawJob(L.make_grid(j.grid), min(self.window, j.pos.shape[0]), 1, None, 1, None)
        n = ctypes.c_size_t(0)
        L.check("tacaw_multislice_batch", lib.tacaw_multislice_batch(arr, len(self.jobs), null, ctypes.byref(n),
                                                                     null))
        self.ws_batch = torch.empty(max(n.value, 256), dtype=torch.uint8, device=self.device)

    def capture(self):
        """Run once eagerly, then record the whole run into a CUDA graph."""
        self.prepare()
        self.run()
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run()
        return self.graph

    def replay(self):
        self.graph.replay()
        return [(st["I"], st["I_el"]) for st in self.state]
