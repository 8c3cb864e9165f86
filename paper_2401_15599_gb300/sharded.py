"""One trajectory spread over several GPUs, one process per GPU.

The multislice of every snapshot is independent (the procedure after
Eq. (9) propagates the beam through each snapshot on its own), so rank r
takes the contiguous snapshots [t_lo, t_hi) of the trajectory.  The spectrum
needs every snapshot of a q, and the time mean in it, so it has one exchange:

  1. each rank: slice potentials and multislice of its snapshots; the FP64
     running sum of its exit waves;
  2. all-reduce of the FP64 sums -> the exact mean m of the whole trajectory;
  3. each rank: Phi_r(q, E) = sum_{n in its snapshots} (psi(q, t_n) - m_q)
     exp(-i E t_n / hbar) with the global times t_n (tacaw_spectrum_accumulate);
  4. reduce-scatter of Phi over q: rank r receives the sum over ranks of the
     rows [q_lo, q_hi);
  5. each rank: I = |Phi|^2 / T^2 and I_el = |m|^2 on its q rows
     (tacaw_spectrum_finish; with the exact mean the FP64 correction is 0).

Step 4 moves nq * n_omega complex numbers (less than the all-to-all of the
exit waves when n_omega < T).  Collectives go through torch.distributed
(NCCL: reduce_scatter_tensor; other backends: all_reduce, then each rank keeps
its rows).  The per-rank compute is the ``ops`` object: ``CudaOps`` (the
library's kernels) on GPUs; tests substitute their own.
"""

from __future__ import annotations

import torch
import torch.distributed as dist


def shard_bounds(n: int, world: int, rank: int):
    """Contiguous, balanced [lo, hi) of n items for `rank` of `world`."""
    base, extra = divmod(int(n), int(world))
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def _group_info(group):
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(group), dist.get_world_size(group)
    return 0, 1


class CudaOps:
    """Per-rank compute through the library (the GPU path)."""

    phi_dtype = torch.complex64

    def __init__(self, grid, n_atoms, amp_sigma, batch, precision, device, ms_flags=0):
        from .pipeline import TimeToSpectrum
        self.grid = grid
        self.amp_sigma = amp_sigma
        self.batch = batch
        self.precision = precision
        self.device = torch.device(device)
        self.ms_flags = ms_flags
        self.n_atoms = n_atoms
        self._tts = None
        self._TTS = TimeToSpectrum

    def exit_waves(self, pos, species):
        """pos [T_r, Na, 3] (device) -> psi [T_r, nq] complex64, FP64 sum [nq]."""
        n = int(pos.shape[0])
        if self._tts is None or self._tts.n_t != n:
            self._tts = self._TTS(self.grid, n, self.n_atoms, self.amp_sigma, 1.0, batch=self.batch,
                                  device=self.device, ms_flags=self.ms_flags)
            self._tts.prepare(None, None)
        psi = self._tts.exit_waves(pos, species)
        return psi.reshape(n, -1), self._tts.psi_sum.reshape(-1)

    def time_mean(self, psum, n_t):
        from . import api
        return api.time_mean(psum, n_t)

    def accumulate(self, psi, t0, dt_fs, omega, m, phi):
        from . import api
        api.spectrum_accumulate(psi, t0, dt_fs, omega, m, phi, precision=self.precision)

    def finish(self, phi, n_t, dt_fs, omega, m_ref, psum, kubo, temperature_K):
        from . import api
        return api.spectrum_finish(phi, n_t, dt_fs, omega, m_ref, psum, kubo=kubo, temperature_K=temperature_K)


class ShardedTimeToSpectrum:
    """I(q, E) of one trajectory whose snapshots are spread over the ranks of
    `group` (or one process without a group).  ``run(pos_local, species)``
    takes this rank's snapshots [t_lo, t_hi) and returns this rank's rows
    [q_lo, q_hi) of I and I_el, on the explicit energy grid omega_meV."""

    def __init__(self, grid, n_t, n_atoms, amp_sigma, dt_fs, omega_meV, group=None, batch=32,
                 precision="bf16x6", kubo=False, temperature_K=300.0, device="cuda", ops=None,
                 ms_flags=0):
        self.grid = grid
        self.n_t = int(n_t)
        self.dt_fs = float(dt_fs)
        self.group = group
        self.rank, self.world = _group_info(group)
        self.device = torch.device(device)
        self.omega = torch.as_tensor(omega_meV, dtype=torch.float64, device=self.device)
        self.kubo = kubo
        self.temperature_K = temperature_K
        self.nq = int(grid.nx) * int(grid.ny)
        self.t_lo, self.t_hi = shard_bounds(self.n_t, self.world, self.rank)
        self.rows = -(-self.nq // self.world)                   # q rows per rank (the last one padded)
        self.q_lo = min(self.nq, self.rank * self.rows)
        self.q_hi = min(self.nq, self.q_lo + self.rows)
        self.ops = ops if ops is not None else CudaOps(grid, n_atoms, amp_sigma, batch, precision, device,
                                                       ms_flags=ms_flags)

    def _all_reduce_sum(self, x):
        if self.world == 1:
            return x
        v = torch.view_as_real(x.contiguous())
        dist.all_reduce(v, op=dist.ReduceOp.SUM, group=self.group)
        return torch.view_as_complex(v)

    def _reduce_scatter_rows(self, phi):
        """Sum of phi over the ranks, rows [q_lo, q_hi) of it on this rank."""
        if self.world == 1:
            return phi
        n_w = phi.shape[1]
        padded = torch.zeros((self.rows * self.world, n_w), dtype=phi.dtype, device=phi.device)
        padded[: self.nq] = phi
        flat = torch.view_as_real(padded).reshape(-1)
        if dist.get_backend(self.group) == "nccl":
            out = torch.empty(flat.numel() // self.world, dtype=flat.dtype, device=flat.device)
            dist.reduce_scatter_tensor(out, flat, op=dist.ReduceOp.SUM, group=self.group)
        else:
            dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=self.group)
            out = flat.reshape(self.world, -1)[self.rank]
        mine = torch.view_as_complex(out.reshape(self.rows, n_w, 2))
        return mine[: self.q_hi - self.q_lo].contiguous()

    def run(self, pos_local, species):
        if int(pos_local.shape[0]) != self.t_hi - self.t_lo:
            raise ValueError(f"rank {self.rank} takes snapshots [{self.t_lo}, {self.t_hi})")
        n_w = self.omega.numel()
        if self.t_hi > self.t_lo:
            psi, psum_local = self.ops.exit_waves(pos_local, species)
            psum_local = psum_local.clone()
        else:
            psi = None
            psum_local = torch.zeros(self.nq, dtype=torch.complex128, device=self.device)
        psum = self._all_reduce_sum(psum_local)
        m = self.ops.time_mean(psum, self.n_t)
        phi = torch.zeros((self.nq, n_w), dtype=self.ops.phi_dtype, device=self.device)
        if psi is not None:
            self.ops.accumulate(psi, self.t_lo, self.dt_fs, self.omega, m, phi)
        mine = self._reduce_scatter_rows(phi)
        if self.q_hi == self.q_lo:
            return (torch.zeros((0, n_w), dtype=torch.float32, device=self.device),
                    torch.zeros(0, dtype=torch.float64, device=self.device))
        sl = slice(self.q_lo, self.q_hi)
        return self.ops.finish(mine, self.n_t, self.dt_fs, self.omega, m[sl].contiguous(), psum[sl].contiguous(),
                               self.kubo, self.temperature_K)
