"""Time-to-spectrum for many independent trajectories of uneven size.

Each job has its own grid, slice count, snapshot count and atoms.  Snapshots
are processed in windows: for every window the slice potentials of each job
are built, then one multislice call advances all jobs together: with square
grids and windows of at least QUEUE_MIN_WINDOW snapshots
``tacaw_multislice_queue`` (one persistent launch per grid size over a device
work queue; items of 32 rows or columns, which on uneven jobs of 128-768
points beat the queue's default of 16), else ``tacaw_multislice_batch`` (two
launches per slice, shared by the jobs of one grid size).  With windows of a
few snapshots a slice of the queue has fewer items than the launch has
blocks, so blocks wait on one another; per-slice launches are faster there.

Two forms of the spectrum (Eq. (9) with the elastic part removed):

* ``chunked=False``: every job keeps all of its exit waves and takes its
  spectrum at the end (``tacaw_spectrum``).
* ``chunked=True``: every job keeps the exit waves of one window only.  After
  each window its inelastic transform is added into Phi(q, E)
  (``tacaw_spectrum_accumulate``, centred on the mean of the job's first
  window), and ``tacaw_spectrum_finish`` removes the rest of the mean in FP64
  at the end.  Memory per job is one window of waves plus Phi, whatever the
  trajectory length.  Needs an explicit energy grid per job.

A job's positions are either a device tensor [T, Na, 3] or, for trajectories
too long to hold, a callable ``positions(t0, t1, out)`` that writes snapshots
t0 .. t1-1 into ``out`` on the device.  ``capture()`` records the whole run in
a CUDA graph and ``replay()`` re-runs it with one launch from the host.
"""

from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, Optional

import torch

from . import api


@dataclass
class Job:
    grid: object
    pos: Optional[torch.Tensor]   # [T, Na, 3] float32 on the device, or None with `positions`
    species: torch.Tensor         # [Na] int32, device
    amp_sigma: object             # [n_species][2]
    dt_fs: float
    omega_meV: object = None
    n_t: int = 0                  # with `positions`: the number of snapshots
    positions: Optional[Callable] = None   # positions(t0, t1, out) -> out [t1 - t0, Na, 3]

    def snapshots(self) -> int:
        return int(self.pos.shape[0]) if self.pos is not None else int(self.n_t)

    def atoms(self) -> int:
        return int(self.species.shape[0])


QUEUE_MIN_WINDOW = 32      # snapshots per window from which the work queue is the default


def queue_by_default(grids, window) -> bool:
    """The multislice engine ``queue="auto"`` picks: the work queue when every
    grid is square (the queue's tiles) and a window holds at least
    QUEUE_MIN_WINDOW snapshots, else per-slice batch launches."""
    return all(int(g.nx) == int(g.ny) for g in grids) and int(window) >= QUEUE_MIN_WINDOW


class BatchTimeToSpectrum:
    def __init__(self, jobs, window=8, precision="bf16x6", device="cuda", chunked=False, queue="auto", wave=0,
                 span=32):
        self.jobs = list(jobs)
        if window == "auto":                    # tuned for the largest grid of the jobs (tuning.py)
            from .tuning import best_multislice_batch
            big = max(self.jobs, key=lambda j: j.grid.nx * j.grid.ny * j.grid.n_slices)
            window = best_multislice_batch(big.grid, device=device)
        self.window = int(window)
        if queue == "auto":
            queue = queue_by_default([j.grid for j in self.jobs], self.window)
        self.queue, self.wave, self.span = bool(queue), int(wave), int(span)
        self.precision = precision
        self.chunked = bool(chunked)
        self.device = torch.device(device)
        self.state = []
        for j in self.jobs:
            g = j.grid
            n_t = j.snapshots()
            if self.chunked and j.omega_meV is None:
                raise ValueError("chunked spectra need an explicit energy grid per job (omega_meV)")
            n_w = n_t if j.omega_meV is None else len(j.omega_meV)
            nq = g.nx * g.ny
            w = min(self.window, n_t)
            st = {
                "psi": torch.empty((w if self.chunked else n_t, g.ny, g.nx), dtype=torch.complex64,
                                   device=self.device),
                "psi_sum": torch.zeros((g.ny, g.nx), dtype=torch.complex128, device=self.device),
                "V": torch.empty((w, g.n_slices, g.ny, g.nx), dtype=torch.float32, device=self.device),
                "I": torch.empty((nq, n_w), dtype=torch.float32, device=self.device),
                "I_el": torch.empty(nq, dtype=torch.float64, device=self.device),
                "omega": None if j.omega_meV is None else
                torch.as_tensor(j.omega_meV, dtype=torch.float64, device=self.device),
            }
            if j.pos is None:
                st["pos_buf"] = torch.empty((w, j.atoms(), 3), dtype=torch.float32, device=self.device)
            if self.chunked:
                st["phi"] = torch.zeros((nq, n_w), dtype=torch.complex64, device=self.device)
                st["m_ref"] = torch.zeros(nq, dtype=torch.complex128, device=self.device)
            self.state.append(st)
        self.graph = None

    def _positions(self, j, st, t0, t1):
        if j.pos is not None:
            return j.pos[t0:t1]
        out = st["pos_buf"][: t1 - t0]
        j.positions(t0, t1, out)
        return out

    def run(self):
        for st in self.state:
            st["psi_sum"].zero_()
            if self.chunked:
                st["phi"].zero_()
        t_max = max(j.snapshots() for j in self.jobs)
        for t0 in range(0, t_max, self.window):
            batch, live = [], []
            for j, st in zip(self.jobs, self.state):
                n_t = j.snapshots()
                if t0 >= n_t:
                    continue
                t1 = min(n_t, t0 + self.window)
                v = st["V"][: t1 - t0]
                api.potential(j.grid, self._positions(j, st, t0, t1), j.species, j.amp_sigma, out=v,
                              workspace=st.get("ws_pot"))
                out = st["psi"][: t1 - t0] if self.chunked else st["psi"][t0:t1]
                batch.append({"grid": j.grid, "V": v, "out": out, "psi_sum": st["psi_sum"]})
                live.append((j, st, t1))
            api.multislice_batch(batch, workspace=getattr(self, "ws_batch", None), queue=self.queue,
                                 wave=self.wave, span=self.span)
            if self.chunked:
                for j, st, t1 in live:
                    if t0 == 0:                 # reference mean: the job's first window
                        api.time_mean(st["psi_sum"].reshape(-1), t1 - t0, out=st["m_ref"])
                    api.spectrum_accumulate(st["psi"][: t1 - t0], t0, j.dt_fs, st["omega"], st["m_ref"],
                                            st["phi"], precision=self.precision, workspace=st.get("ws_acc"))
        for j, st in zip(self.jobs, self.state):
            n_t = j.snapshots()
            if self.chunked:
                api.spectrum_finish(st["phi"], n_t, j.dt_fs, st["omega"], st["m_ref"], st["psi_sum"].reshape(-1),
                                    out=st["I"], i_el=st["I_el"], workspace=st.get("ws_fin"))
            else:
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
        one = ctypes.c_void_p(1)
        prec = {"fp32": L.TACAW_FP32, "bf16x3": L.TACAW_BF16X3, "fft32": L.TACAW_FFT32,
                "bf16x6": L.TACAW_BF16X6}[self.precision]
        for j, st in zip(self.jobs, self.state):
            g = L.make_grid(j.grid)
            n = ctypes.c_size_t(0)
            amp = torch.as_tensor(j.amp_sigma, dtype=torch.float32).reshape(-1, 2)
            amp_c = (ctypes.c_float * amp.numel())(*amp.flatten().tolist())
            L.check("tacaw_potential", lib.tacaw_potential(ctypes.byref(g), st["V"].shape[0], j.atoms(), null,
                                                           null, amp.shape[0], amp_c, null, null, ctypes.byref(n),
                                                           null))
            st["ws_pot"] = torch.empty(max(n.value, 256), dtype=torch.uint8, device=self.device)
            n_t = j.snapshots()
            nq = j.grid.nx * j.grid.ny
            n_w = st["I"].shape[1]
            if self.chunked:
                L.check("tacaw_spectrum_accumulate",
                        lib.tacaw_spectrum_accumulate(nq, 0, st["psi"].shape[0], float(j.dt_fs), n_w, one, one, one,
                                                      one, prec, null, ctypes.byref(n), null))
                st["ws_acc"] = torch.empty(max(n.value, 256), dtype=torch.uint8, device=self.device)
                L.check("tacaw_spectrum_finish",
                        lib.tacaw_spectrum_finish(nq, n_t, float(j.dt_fs), n_w, one, one, one, one, one, one, 0,
                                                  300.0, null, ctypes.byref(n), null))
                st["ws_fin"] = torch.empty(max(n.value, 256), dtype=torch.uint8, device=self.device)
            else:
                L.check("tacaw_spectrum", lib.tacaw_spectrum(nq, n_t, float(j.dt_fs), n_w,
                                                             one if st["omega"] is not None else null,
                                                             null, one, null, one, prec, 0, 300.0, null,
                                                             ctypes.byref(n), null))
                st["ws_spec"] = torch.empty(max(n.value, 256), dtype=torch.uint8, device=self.device)
        arr = (L.TacawJob * len(self.jobs))()
        for i, j in enumerate(self.jobs):
            arr[i] = L.TacawJob(L.make_grid(j.grid), min(self.window, j.snapshots()), 1, None, 1, None)
        n = ctypes.c_size_t(0)
        if self.queue:
            L.check("tacaw_multislice_queue", lib.tacaw_multislice_queue(arr, len(self.jobs), self.wave, self.span,
                                                                         null, ctypes.byref(n), null))
        else:
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
