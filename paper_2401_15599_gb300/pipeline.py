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
                 device="cuda", ms_flags=0):
        self.grid = grid
        self.n_t = int(n_t)
        self.n_atoms = int(n_atoms)
        self.amp_sigma = amp_sigma
        self.dt_fs = float(dt_fs)
        self.ms_flags = int(ms_flags)           # variants of the passes (tacaw_multislice flags)
        if batch == "auto":                     # batch and row-pass variant tuned per grid and GPU, cached
            from .tuning import best_multislice_config
            batch, self.ms_flags = best_multislice_config(grid, device=device)
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
        self._copy_stream = None                # host-input path (run_host): H2D copies
        self._pos_stage = None                  # [2][batch][Na][3] device staging of host positions
        self._d2h_stream = None                 # run_host: D2H copies of I, I_el
        self._d2h_done = None                   # event: the last run_host's outputs are in host memory
        self._graph = None                      # CUDA graph of run() on self._graph_args
        self._graph_args = None

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
                           workspace=self._ws.get("ms"), ms_flags=self.ms_flags)
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

    def capture(self, pos, species):
        """Record run(pos, species) into a CUDA graph (after one eager run that
        fills the workspace cache); replay() then re-runs it on the same device
        buffers with one launch.  The buffers must stay alive and in place."""
        self.prepare(None, None)
        self.run(pos, species)
        torch.cuda.synchronize(self.device)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self.run(pos, species)
        self._graph, self._graph_args = graph, (pos, species)
        return graph

    def replay(self):
        """Re-run the captured run() (positions read from the captured buffer)."""
        if self._graph is None:
            raise RuntimeError("capture() first")
        self._graph.replay()
        return self.I, self.I_el

    def run_host(self, pos_host, species, out=None, out_el=None):
        """Host positions pos_host [T, Na, 3] (float32, CPU; pinned for asynchronous
        copies) -> I(q, E) and I_el in host memory.

        The positions travel to the device one snapshot batch at a time on a copy
        stream, into two staging buffers, so that the copy of batch b + 1 overlaps
        the potential and multislice of batch b; then the temporal transform, and
        I and I_el are copied into `out` / `out_el` (host tensors, allocated pinned
        if None) on a stream of their own, so that those copies overlap the next
        call's work (whose temporal transform waits for them).  Nothing blocks the
        host: call wait_host() and synchronize the current stream (or the device)
        before reading the outputs."""
        if pos_host.device.type != "cpu" or pos_host.dtype != torch.float32 or not pos_host.is_contiguous():
            raise ValueError("pos_host must be a contiguous float32 CPU tensor")
        if tuple(pos_host.shape) != (self.n_t, self.n_atoms, 3):
            raise ValueError(f"pos_host must be [{self.n_t}, {self.n_atoms}, 3]")
        comp = torch.cuda.current_stream(self.device)
        if self._copy_stream is None:
            self._copy_stream = torch.cuda.Stream(self.device)
        if self._pos_stage is None:
            self._pos_stage = torch.empty((2, self.batch, self.n_atoms, 3), dtype=torch.float32, device=self.device)
        cs = self._copy_stream
        ready = [torch.cuda.Event(), torch.cuda.Event()]
        free = [torch.cuda.Event(), torch.cuda.Event()]
        starts = list(range(0, self.n_t, self.batch))
        cs.wait_stream(comp)                    # earlier work may still read the staging buffers

        def issue(i):
            t0 = starts[i]
            t1 = min(self.n_t, t0 + self.batch)
            slot = i % 2
            with torch.cuda.stream(cs):
                if i >= 2:
                    cs.wait_event(free[slot])   # the potential of batch i - 2 has read it
                self._pos_stage[slot, : t1 - t0].copy_(pos_host[t0:t1], non_blocking=True)
                ready[slot].record(cs)

        issue(0)
        self.psi_sum.zero_()
        for i, t0 in enumerate(starts):
            if i + 1 < len(starts):
                issue(i + 1)
            t1 = min(self.n_t, t0 + self.batch)
            slot = i % 2
            comp.wait_event(ready[slot])
            v = self.V[: t1 - t0]
            api.potential(self.grid, self._pos_stage[slot, : t1 - t0], species, self.amp_sigma, out=v,
                          workspace=self._ws.get("pot"))
            free[slot].record(comp)
            api.multislice(self.grid, v, out=self.psi[t0:t1], psi_sum=self.psi_sum,
                           workspace=self._ws.get("ms"), ms_flags=self.ms_flags)
        if self._d2h_done is not None:
            comp.wait_event(self._d2h_done)     # the previous call's outputs have left I, I_el
        self.spectrum()
        if out is None:
            out = torch.empty(self.I.shape, dtype=self.I.dtype).pin_memory()
        if out_el is None:
            out_el = torch.empty(self.I_el.shape, dtype=self.I_el.dtype).pin_memory()
        if self._d2h_stream is None:
            self._d2h_stream = torch.cuda.Stream(self.device)
            self._d2h_done = torch.cuda.Event()
        d2h = self._d2h_stream
        d2h.wait_stream(comp)
        with torch.cuda.stream(d2h):
            out.copy_(self.I, non_blocking=True)
            out_el.copy_(self.I_el, non_blocking=True)
        self._d2h_done.record(d2h)
        return out, out_el

    def wait_host(self):
        """Make the current stream wait until the last run_host's outputs are in
        host memory."""
        if self._d2h_done is not None:
            torch.cuda.current_stream(self.device).wait_event(self._d2h_done)
