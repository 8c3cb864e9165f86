"""The sharded multi-GPU path's host logic on CPU ranks (gloo): snapshots
split across 2 and 3 ranks, the FP64 all-reduce of the running sums, per-rank
partial transforms with global times, the reduce-scatter of Phi over q and
each rank's rows, against the single-process oracle spectrum of the whole
trajectory.  The per-rank compute is an FP64 stand-in built from the oracle's
steps (the library's kernels need a GPU); the orchestration is the product
code's."""

import os
import socket

import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")


class OracleOps:
    """FP64 per-rank compute from the oracle's steps (test stand-in)."""

    phi_dtype = torch.complex128

    def __init__(self, grid, amp_sigma):
        self.g = O.grid_from_spec(grid)
        self.amp_sigma = np.asarray(amp_sigma, np.float64)

    def exit_waves(self, pos, species):
        psi = O.exit_waves(self.g, pos.numpy().astype(np.float64), species.numpy(), self.amp_sigma)
        psi = torch.from_numpy(psi.reshape(psi.shape[0], -1))
        return psi, psi.sum(0)

    def time_mean(self, psum, n_t):
        return psum / n_t

    def accumulate(self, psi, t0, dt, omega, m, phi):
        a = (psi - m[None, :]).numpy()
        e = omega.numpy()
        shift = np.exp(-1j * e * (t0 * dt) / O.HBAR_MEV_FS)          # times of this rank's snapshots
        phi += torch.from_numpy(O.temporal_transform(a, dt, e) * shift[None, :])

    def finish(self, phi, n_t, dt, omega, m_ref, psum, kubo, temperature_K):
        inten = (phi.abs() ** 2 / float(n_t) ** 2).numpy()
        return torch.from_numpy(inten), (psum / n_t).abs() ** 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n_t, queue):
    import torch.distributed as dist
    from paper_2401_15599_gb300.sharded import ShardedTimeToSpectrum
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = W.WORKLOADS["plain_small"].with_(n_t=n_t)
        inp = W.build_inputs(w)
        omega = np.linspace(-120.0, 120.0, 48, endpoint=False)
        sh = ShardedTimeToSpectrum(w.grid, n_t, inp.crystal.n_atoms, inp.amp_sigma, w.dt_fs, omega, device="cpu",
                                   ops=OracleOps(w.grid, inp.amp_sigma))
        pos = torch.from_numpy(inp.positions(list(range(sh.t_lo, sh.t_hi))))
        inten, iel = sh.run(pos, torch.from_numpy(inp.species))
        queue.put((rank, sh.q_lo, sh.q_hi, sh.t_lo, sh.t_hi, inten.numpy(), iel.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n_t", [(2, 12), (3, 10)])
def test_sharded_spectrum_equals_single_process(world, n_t):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, n_t, queue)) for r in range(world)]
    for p in procs:
        p.start()
    parts = [queue.get(timeout=600) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    parts.sort()
    # snapshots: contiguous, covering, disjoint; q rows likewise
    assert [p[3] for p in parts][0] == 0 and parts[-1][4] == n_t
    assert all(parts[i][4] == parts[i + 1][3] for i in range(world - 1))
    nq = 64 * 64
    assert parts[0][1] == 0 and parts[-1][2] == nq
    assert all(parts[i][2] == parts[i + 1][1] for i in range(world - 1))
    inten = np.concatenate([p[5] for p in parts])
    iel = np.concatenate([p[6] for p in parts])
    w = W.WORKLOADS["plain_small"].with_(n_t=n_t)
    inp = W.build_inputs(w)
    g = O.grid_from_spec(w.grid)
    psi = O.exit_waves(g, inp.positions().astype(np.float64), inp.species, inp.amp_sigma.astype(np.float64))
    omega = np.linspace(-120.0, 120.0, 48, endpoint=False)
    ref, ref_el, _ = O.spectrum(psi, w.dt_fs, omega)
    assert np.linalg.norm(inten - ref) / np.linalg.norm(ref) < 1e-11
    assert np.linalg.norm(iel - ref_el) / np.linalg.norm(ref_el) < 1e-12


def test_shard_bounds_cover_every_item_once():
    from paper_2401_15599_gb300.sharded import shard_bounds
    for n in (0, 1, 7, 4096, 4097):
        for world in (1, 2, 3, 8):
            spans = [shard_bounds(n, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            assert max(b - a for a, b in spans) - min(b - a for a, b in spans) <= 1
