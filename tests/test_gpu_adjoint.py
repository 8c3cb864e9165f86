"""GPU adjoint: tacaw_spectrum_backward, tacaw_multislice_backward and
tacaw_potential_backward (through the C-ABI) against the FP64 oracle adjoint,
the autograd chain against the oracle chain, and -- at the full size of the
differentiation workload -- against central finite differences of the GPU's
own loss."""

import numpy as np
import pytest

import oracle as O
import oracle.adjoint as A
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_15599_gb300 import build
    build.build()
    from paper_2401_15599_gb300 import api as a
    return a


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def _grid(nx=64, ny=64, lx=16.0, ly=16.0, n_slices=5, dz=2.0, kev=200.0):
    return O.Grid(nx, ny, lx, ly, n_slices, dz, 0.0, kev, 2.0 / 3.0)


@pytest.mark.parametrize("n_t,nq,omega", [(64, 300, None), (37, 130, None),
                                          (50, 200, np.linspace(-100, 100, 96, endpoint=False))])
def test_spectrum_backward_matches_oracle(api, n_t, nq, omega):
    rng = np.random.default_rng(n_t + nq)
    psi = (1 + 0.05 * (rng.standard_normal((n_t, nq)) + 1j * rng.standard_normal((n_t, nq)))).astype(np.complex64)
    n_w = n_t if omega is None else len(omega)
    dl_di = rng.standard_normal((nq, n_w)).astype(np.float32)
    g = api.spectrum_backward(_dev(psi), 5.0, _dev(dl_di), omega_meV=omega).cpu().numpy()
    ref = A.spectrum_backward(psi.astype(np.complex128), 5.0, dl_di.astype(np.float64), omega)
    assert rel_l2(g, ref) < 1e-5


def _potentials(g, n_t, seed, n_atoms=40):
    rng = np.random.default_rng(seed)
    v = np.empty((n_t, g.n_slices, g.ny, g.nx), dtype=np.float32)
    for t in range(n_t):
        pos = np.stack([rng.uniform(0, g.lx, n_atoms), rng.uniform(0, g.ly, n_atoms),
                        rng.uniform(0, g.n_slices * g.dz, n_atoms)], axis=1)
        v[t] = O.projected_potential(g, pos, np.zeros(n_atoms, int), [[25.0, 0.3]])
    return v


@pytest.mark.parametrize("nx,ny,n_slices", [(64, 64, 5), (128, 64, 4), (256, 256, 3)])
def test_multislice_backward_matches_oracle_and_checkpointing(api, nx, ny, n_slices):
    g = _grid(nx, ny, nx * 0.25, ny * 0.25, n_slices)
    n_t = 2
    v = _potentials(g, n_t, nx + ny)
    rng = np.random.default_rng(7)
    gx = (rng.standard_normal((n_t, ny, nx)) + 1j * rng.standard_normal((n_t, ny, nx))).astype(np.complex64)
    outs = [api.multislice_backward(g, _dev(v), _dev(gx), ckpt_every=k).cpu() for k in (0, 1, 2, n_slices)]
    for o in outs[1:]:
        assert torch.equal(outs[0], o)          # recomputation from checkpoints is exact
    for t in range(n_t):
        ref, _ = A.multislice_backward(g, v[t].astype(np.float64), gx[t].astype(np.complex128))
        assert rel_l2(outs[0][t].numpy(), ref) < 2e-5


def test_potential_backward_matches_oracle(api):
    g = _grid(128, 96, 24.0, 18.0, 4, 1.5)
    rng = np.random.default_rng(11)
    n_t, n = 3, 50
    pos = np.stack([np.stack([rng.uniform(-0.5, g.lx + 0.5, n), rng.uniform(-0.5, g.ly + 0.5, n),
                              rng.uniform(-0.5, 6.5, n)], axis=1) for _ in range(n_t)]).astype(np.float32)
    species = rng.integers(0, 2, n).astype(np.int32)
    amp_sigma = np.array([[20.0, 0.3], [12.0, 0.42]], dtype=np.float32)
    dv = rng.standard_normal((n_t, g.n_slices, g.ny, g.nx)).astype(np.float32)
    grad = api.potential_backward(g, _dev(pos), _dev(species), amp_sigma, _dev(dv)).cpu().numpy()
    ref = sum(A.potential_backward(g, pos[t].astype(np.float64), species, amp_sigma.astype(np.float64),
                                   dv[t].astype(np.float64)) for t in range(n_t))
    assert np.allclose(grad, ref, rtol=1e-5, atol=1e-6 * np.abs(ref).max())


def _chain_case():
    g = O.Grid(64, 64, 16.2, 16.2, 4, 2.0, 0.0, 200.0, 2.0 / 3.0)
    w = W.WORKLOADS["differentiation"].with_(ncell=(4, 4, 2), n_t=16,
                                               grid=W.GridSpec(64, 64, 16.2, 16.2, 4, 2.0, 0.0, 200.0))
    inp = W.build_inputs(w)
    pos = inp.positions()
    species = (np.arange(pos.shape[1]) % 2).astype(np.int32)
    amp_sigma = np.array([[20.0, 0.3], [14.0, 0.36]], dtype=np.float32)
    return g, w, pos, species, amp_sigma


def test_autograd_chain_matches_oracle_chain(api):
    from paper_2401_15599_gb300.autograd import spectrum_from_atoms
    g, w, pos, species, amp_sigma = _chain_case()
    dt = w.dt_fs
    n_t = pos.shape[0]
    # target spectrum: amplitudes x 1.05 (FP64 oracle)
    psi_t = O.exit_waves(g, pos.astype(np.float64), species, amp_sigma.astype(np.float64) * [[1.05, 1.0]])
    target, _, e = O.spectrum(psi_t, dt)
    wts = A.loss_weights(g, n_t, e)
    # oracle chain gradient
    psi = O.exit_waves(g, pos.astype(np.float64), species, amp_sigma.astype(np.float64))
    inten, _, _ = O.spectrum(psi, dt)
    dl_di = A.loss_grad(inten, target, wts)
    g_psi = A.spectrum_backward(psi, dt, dl_di).reshape(n_t, g.ny, g.nx)
    ref = np.zeros((2, 2))
    for t in range(n_t):
        v = O.projected_potential(g, pos[t].astype(np.float64), species, amp_sigma.astype(np.float64))
        g_v, _ = A.multislice_backward(g, v, g_psi[t])
        ref += A.potential_backward(g, pos[t].astype(np.float64), species, amp_sigma.astype(np.float64), g_v)
    # GPU through autograd
    asg = torch.tensor(amp_sigma, dtype=torch.float64, requires_grad=True)
    i_gpu = spectrum_from_atoms(asg, _dev(pos), _dev(species), g, dt, batch=5, ckpt_every=2)
    tgt = _dev(target.astype(np.float32)).double()
    wt = _dev(wts)
    loss = torch.sum(wt * (i_gpu.double() - tgt) ** 2) / torch.sum(wt * tgt ** 2)
    loss.backward()
    assert np.allclose(asg.grad.numpy(), ref, rtol=1e-3, atol=1e-3 * np.abs(ref).max())


def test_autograd_potentials_matches_oracle(api):
    from paper_2401_15599_gb300.autograd import spectrum_from_potentials
    g = _grid(64, 64, 16.0, 16.0, 3)
    n_t = 12
    v = _potentials(g, n_t, 3)
    rng = np.random.default_rng(2)
    dl_di = rng.standard_normal((g.nx * g.ny, n_t)).astype(np.float32)
    vt = _dev(v).requires_grad_(True)
    inten = spectrum_from_potentials(vt, g, 5.0, batch=5, ckpt_every=2)
    inten.backward(_dev(dl_di))
    psi = np.stack([O.multislice(g, v[t].astype(np.float64)) for t in range(n_t)])
    g_psi = A.spectrum_backward(psi, 5.0, dl_di.astype(np.float64)).reshape(n_t, g.ny, g.nx)
    ref = np.stack([A.multislice_backward(g, v[t].astype(np.float64), g_psi[t])[0] for t in range(n_t)])
    assert rel_l2(vt.grad.cpu().numpy(), ref) < 1e-4


def test_differentiation_workload_gradient_vs_finite_differences(api):
    # Full size: fcc 10x10x25 (10 000 atoms), 256^2, 50 slices, 1024 snapshots,
    # loss against amplitudes x 1.05; GPU gradient vs GPU central differences.
    from paper_2401_15599_gb300.autograd import spectrum_from_atoms
    w = W.WORKLOADS["differentiation"]
    g = w.grid
    inp = W.build_inputs(w)
    pos = _dev(inp.positions())
    species = _dev(inp.species)
    base = torch.tensor([[20.0, 0.3]], dtype=torch.float64)
    with torch.no_grad():
        tgt = spectrum_from_atoms(base * torch.tensor([[1.05, 1.0]], dtype=torch.float64), pos, species, g,
                                  w.dt_fs, batch=128).double()
    e = O.natural_energies(w.n_t, w.dt_fs)
    wt = _dev(A.loss_weights(O.grid_from_spec(g), w.n_t, e))
    norm = torch.sum(wt * tgt ** 2)

    def loss_of(asg):
        i = spectrum_from_atoms(asg, pos, species, g, w.dt_fs, batch=128, ckpt_every=7)
        return torch.sum(wt * (i.double() - tgt) ** 2) / norm

    asg = base.clone().requires_grad_(True)
    loss_of(asg).backward()
    grad = asg.grad.numpy()
    for c, h in ((0, 0.02), (1, 3e-4)):
        d = torch.zeros_like(base)
        d[0, c] = h
        with torch.no_grad():
            fd = (loss_of(base + d) - loss_of(base - d)).item() / (2 * h)
        assert grad[0, c] == pytest.approx(fd, rel=1e-3), (c, grad[0, c], fd)
