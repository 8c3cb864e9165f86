"""GPU parity: the CUDA path (called through the C-ABI) against the FP64
oracle on the same seeded inputs.

Tolerances: slice potentials are FP32 sums of FP32 Gaussians (relative
error ~1e-6 of the peak); exit waves are FP32 multislice (rounding of a few
hundred FP32 butterflies, ~1e-6 of the wave's norm); spectra must meet the
relative-L2 bound 2e-5 on I(q, E) against the FP64 oracle.
"""

import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SPEC_TOL = 2e-5


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_15599_gb300 import build
    build.build()
    from paper_2401_15599_gb300 import api as A
    return A


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) else np.float64)
    b = np.asarray(b, dtype=a.dtype)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _grid(nx=64, ny=64, lx=32.0, ly=32.0, n_slices=4, dz=2.0, z0=0.0, kev=200.0, bl=2.0 / 3.0):
    return O.Grid(nx, ny, lx, ly, n_slices, dz, z0, kev, bl)


def _random_atoms(rng, n, g, n_species, margin=0.7):
    pos = np.stack([rng.uniform(-margin, g.lx + margin, n), rng.uniform(-margin, g.ly + margin, n),
                    rng.uniform(g.z0 - 1.0, g.z0 + g.n_slices * g.dz + 1.0, n)], axis=1)
    return pos.astype(np.float32), rng.integers(0, n_species, n).astype(np.int32)


def _dev(x, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(x))
    return t.to("cuda") if dtype is None else t.to(device="cuda", dtype=dtype)


# ---------------------------------------------------------------- potential
@pytest.mark.parametrize("shape", [(64, 64, 32.0, 32.0, 4, 2.0), (48, 40, 9.0, 7.5, 3, 1.5),
                                   (512, 512, 81.0, 81.0, 6, 2.0)])
def test_potential_matches_oracle(api, shape):
    nx, ny, lx, ly, ns, dz = shape
    g = _grid(nx, ny, lx, ly, ns, dz, z0=0.5)
    rng = np.random.default_rng(nx + ny)
    amp_sigma = np.array([[20.0, 0.3], [11.0, 0.41], [27.0, 0.25]], dtype=np.float32)
    n_t = 3
    pos = np.stack([_random_atoms(rng, 60, g, 3)[0] for _ in range(n_t)])
    species = rng.integers(0, 3, 60).astype(np.int32)
    v = api.potential(g, _dev(pos), _dev(species), amp_sigma).cpu().numpy()
    for t in range(n_t):
        ref = O.projected_potential(g, pos[t].astype(np.float64), species, amp_sigma.astype(np.float64))
        assert np.max(np.abs(v[t] - ref)) <= 2e-6 * np.max(np.abs(ref)) + 1e-6


def test_potential_deterministic_and_order_insensitive(api):
    g = _grid(128, 128, 40.5, 40.5, 5, 2.0)
    rng = np.random.default_rng(5)
    pos0, species = _random_atoms(rng, 400, g, 2)
    perm = rng.permutation(400)
    amp_sigma = np.array([[20.0, 0.3], [15.0, 0.35]], dtype=np.float32)
    # identical snapshots (and repeated calls) give bit-identical potentials
    pos = np.stack([pos0, pos0])
    v0 = api.potential(g, _dev(pos), _dev(species), amp_sigma).cpu()
    v0b = api.potential(g, _dev(pos), _dev(species), amp_sigma).cpu()
    assert torch.equal(v0[0], v0[1])
    assert torch.equal(v0, v0b)
    # listing the atoms in another order only changes the FP32 summation order
    v1 = api.potential(g, _dev(pos0[perm][None]), _dev(species[perm]), amp_sigma).cpu()
    assert torch.max(torch.abs(v1[0] - v0[0])).item() <= 1e-6 * torch.max(torch.abs(v0[0])).item()


def test_potential_edge_cases(api):
    g = _grid(64, 64, 32.0, 32.0, 4, 2.0)
    # no atoms: V = 0
    v = api.potential(g, torch.zeros((2, 0, 3), device="cuda"), torch.zeros(0, dtype=torch.int32, device="cuda"),
                      [[20.0, 0.3]])
    assert torch.count_nonzero(v).item() == 0
    # an atom with an out-of-range species is skipped
    pos = np.array([[[5.0, 6.0, 3.0], [20.0, 20.0, 3.0]]], dtype=np.float32)
    sp = np.array([0, 7], dtype=np.int32)
    v = api.potential(g, _dev(pos), _dev(sp), [[20.0, 0.3]]).cpu().numpy()[0]
    ref = O.projected_potential(g, pos[0, :1].astype(np.float64), sp[:1], [[20.0, 0.3]])
    assert np.max(np.abs(v - ref)) <= 2e-6 * ref.max()


@pytest.mark.parametrize("dz", [2.5, 2.0])     # 6 s = 2.46 A: neighbouring slices only / two either side
def test_potential_reach_across_a_short_last_tile(api, dz):
    # 200 x 136 pixels: the last column tile is 8 wide and the last band 8 high, so
    # atoms in column / row 0 reach pixels two tiles over through the periodic wrap
    g = _grid(200, 136, 40.0, 27.0, 3, dz, z0=0.5)
    rng = np.random.default_rng(31)
    n = 120
    x, y, z = rng.uniform(0.0, 40.0, n), rng.uniform(0.0, 27.0, n), rng.uniform(0.5, 0.5 + 3 * dz, n)
    x[:n // 2] = rng.uniform(0.0, 40.0 / 200, n // 2)              # column 0
    y[n // 2:] = rng.uniform(0.0, 27.0 / 136, n - n // 2)          # row 0
    pos = np.stack([x, y, z], axis=1).astype(np.float32)
    species = np.zeros(n, np.int32)
    amp_sigma = [[27.0, 0.41]]
    v = api.potential(g, _dev(pos[None]), _dev(species), amp_sigma).cpu().numpy()[0]
    ref = O.projected_potential(g, pos.astype(np.float64), species, np.asarray(amp_sigma, np.float64))
    assert np.max(np.abs(v - ref)) <= 2e-6 * np.max(np.abs(ref)) + 1e-6


# ---------------------------------------------------------------- multislice
def _smooth_potential(g, n_t, seed):
    rng = np.random.default_rng(seed)
    v = np.empty((n_t, g.n_slices, g.ny, g.nx), dtype=np.float32)
    for t in range(n_t):
        pos, sp = _random_atoms(rng, max(8, g.nx * g.ny // 300), g, 1)
        v[t] = O.projected_potential(g, pos.astype(np.float64), sp, [[25.0, 0.3]]).astype(np.float32)
    return v


@pytest.mark.parametrize("nx,ny", [(64, 64), (128, 128), (256, 256), (512, 512), (1024, 1024),
                                   (128, 64), (64, 256), (384, 384), (768, 768), (384, 128), (256, 768)])
def test_multislice_matches_oracle(api, nx, ny):
    d = 0.25
    g = _grid(nx, ny, nx * d, ny * d, 3, 2.0, kev=100.0)
    n_t = 2
    v = _smooth_potential(g, n_t, nx * 7 + ny)
    out = api.multislice(g, _dev(v)).cpu().numpy()
    for t in range(n_t):
        ref = O.multislice(g, v[t].astype(np.float64))
        assert rel_l2(out[t], ref) < 3e-6, (nx, ny, t)


def test_multislice_incident_wave_free_space_closed_form(api):
    # V = 0 and a Gaussian incident wave: the exit wave is the paraxial Fresnel
    # solution (w'^2 = w^2 + i lambda z / 2 pi), independent of the oracle.
    g = _grid(128, 128, 64.0, 64.0, 20, 50.0, kev=100.0)
    w = 3.0
    x = np.arange(g.nx) * g.lx / g.nx
    r2 = (x[None, :] - 32.0) ** 2 + (x[:, None] - 32.0) ** 2
    psi_in = np.exp(-r2 / (2 * w * w)).astype(np.complex64)
    v = np.zeros((1, g.n_slices, g.ny, g.nx), dtype=np.float32)
    out = api.multislice(g, _dev(v), psi_in=_dev(psi_in)).cpu().numpy()[0]
    psi_r = O.ifft2_unitary(out.astype(np.complex128))
    w2 = w * w + 1j * O.wavelength(g.kev) * g.n_slices * g.dz / (2 * np.pi)
    ref = (w * w / w2) * np.exp(-r2 / (2 * w2))
    assert np.max(np.abs(psi_r - ref)) < 2e-5


def test_multislice_plane_wave_through_vacuum(api):
    g = _grid(256, 256, 64.0, 64.0, 5, 2.0)
    v = np.zeros((2, g.n_slices, g.ny, g.nx), dtype=np.float32)
    out = api.multislice(g, _dev(v)).cpu().numpy()
    ref = np.zeros((g.ny, g.nx), complex)
    ref[0, 0] = 1.0
    for t in range(2):
        assert np.max(np.abs(out[t] - ref)) < 1e-6


def test_multislice_snapshot_sum(api):
    g = _grid(64, 64, 16.0, 16.0, 2, 2.0)
    v = _smooth_potential(g, 5, 3)
    s = torch.zeros((g.ny, g.nx), dtype=torch.complex128, device="cuda")
    s += 1.0
    out = api.multislice(g, _dev(v), psi_sum=s)
    ref = out.cpu().numpy().astype(np.complex128).sum(axis=0) + 1.0
    assert np.allclose(s.cpu().numpy(), ref, rtol=1e-14, atol=1e-15)


# ---------------------------------------------------------------- spectrum
def _waves(rng, n_t, nq, inel=0.02):
    base = 1.0 + 0.3 * (rng.standard_normal(nq) + 1j * rng.standard_normal(nq))
    return (base[None, :] + inel * (rng.standard_normal((n_t, nq)) + 1j * rng.standard_normal((n_t, nq)))
            ).astype(np.complex64)


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
@pytest.mark.parametrize("n_t,nq", [(256, 4096), (100, 1000), (37, 65), (1, 70), (512, 300)])
def test_spectrum_natural_grid_matches_oracle(api, n_t, nq, precision):
    rng = np.random.default_rng(n_t + nq)
    psi = _waves(rng, n_t, nq)
    inten, iel = api.spectrum(_dev(psi), 5.0, precision=precision)
    ref, ref_el, _ = O.spectrum(psi.astype(np.complex128), 5.0)
    assert inten.shape == (nq, n_t)
    if n_t == 1:
        assert torch.count_nonzero(inten).item() == 0
    else:
        assert rel_l2(inten.cpu().numpy(), ref) < SPEC_TOL
    assert rel_l2(iel.cpu().numpy(), ref_el) < 1e-13


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_spectrum_explicit_grid_kubo_normalise(api, precision):
    rng = np.random.default_rng(9)
    n_t, nq = 200, 777
    psi = _waves(rng, n_t, nq)
    omega = np.linspace(-200.0, 200.0, 1024, endpoint=False)
    inten, iel = api.spectrum(_dev(psi), 5.0, omega_meV=omega, kubo=True, temperature_K=300.0,
                              normalize=True, precision=precision)
    ref, ref_el, _ = O.spectrum(psi.astype(np.complex128), 5.0, omega, kubo=True, temperature_K=300.0,
                                normalize=True)
    assert rel_l2(inten.cpu().numpy(), ref) < SPEC_TOL
    assert rel_l2(iel.cpu().numpy(), ref_el) < 1e-6
    assert float(inten.double().sum() + iel.sum()) == pytest.approx(1.0, abs=1e-6)


def test_spectrum_given_sum_equals_computed_sum(api):
    rng = np.random.default_rng(4)
    psi = _dev(_waves(rng, 64, 300))
    s = psi.to(torch.complex128).sum(dim=0)
    a, ael = api.spectrum(psi, 5.0)
    b, bel = api.spectrum(psi, 5.0, psi_sum=s)
    assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) < 1e-6


# ---------------------------------------------------------------- end to end
def _e2e(api, w, snapshots=None, batch=64, precision="fp32"):
    from paper_2401_15599_gb300.pipeline import TimeToSpectrum
    inp = W.build_inputs(w)
    pos = inp.positions(snapshots)
    n_t = pos.shape[0]
    tts = TimeToSpectrum(w.grid, n_t, pos.shape[1], inp.amp_sigma, w.dt_fs, batch=batch,
                         precision=precision)
    tts.prepare(None, None)
    inten, iel = tts.run(_dev(pos), _dev(inp.species))
    torch.cuda.synchronize()
    return inp, pos, tts, inten.cpu().numpy(), iel.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_end_to_end_plain_small(api, precision):
    w = W.WORKLOADS["plain_small"]
    inp, pos, tts, inten, iel = _e2e(api, w, precision=precision)
    g = O.grid_from_spec(w.grid)
    psi = O.exit_waves(g, pos.astype(np.float64), inp.species, inp.amp_sigma.astype(np.float64))
    ref, ref_el, _ = O.spectrum(psi, w.dt_fs)
    assert rel_l2(tts.psi.cpu().numpy(), psi) < 3e-6
    assert rel_l2(inten, ref) < SPEC_TOL
    assert rel_l2(iel, ref_el) < 1e-6


def test_host_input_path_matches_device_path(api):
    # run_host: positions from pinned host memory in batches on a copy stream,
    # I(q, E) back to host memory; same kernels and inputs as run(), so the
    # outputs are bit-identical (uneven last batch: 48 snapshots in batches of 20)
    from paper_2401_15599_gb300.pipeline import TimeToSpectrum
    w = W.WORKLOADS["plain_small"].with_(n_t=48)
    inp = W.build_inputs(w)
    pos = inp.positions()
    tts = TimeToSpectrum(w.grid, 48, pos.shape[1], inp.amp_sigma, w.dt_fs, batch=20)
    tts.prepare(None, None)
    sp = _dev(inp.species)
    inten, iel = tts.run(_dev(pos), sp)
    inten, iel = inten.cpu(), iel.cpu()
    pos_host = torch.from_numpy(pos).pin_memory()
    for _ in range(2):                                   # the staging buffers are reused
        out, out_el = tts.run_host(pos_host, sp)
        tts.wait_host()
        torch.cuda.current_stream().synchronize()
        assert torch.equal(out, inten) and torch.equal(out_el, iel)
    # back-to-back calls into the same host buffers: each call's transform waits for
    # the previous call's copies; a captured run() replays bit-identically
    o1, e1 = tts.run_host(pos_host, sp)
    o1, e1 = tts.run_host(pos_host, sp, out=o1, out_el=e1)
    tts.wait_host()
    torch.cuda.current_stream().synchronize()
    assert torch.equal(o1, inten) and torch.equal(e1, iel)
    pos_dev = _dev(pos)
    tts.capture(pos_dev, sp)
    tts.I.zero_()
    i2, el2 = tts.replay()
    torch.cuda.synchronize()
    assert torch.equal(i2.cpu(), inten) and torch.equal(el2.cpu(), iel)
    with pytest.raises(ValueError):
        tts.run_host(pos_host[:10], sp)


def test_static_lattice_gives_exactly_zero(api):
    w = W.WORKLOADS["plain_small"].with_(n_t=16)
    from paper_2401_15599_gb300.pipeline import TimeToSpectrum
    inp = W.build_inputs(w)
    pos = W.static_positions(inp.crystal, 16)
    tts = TimeToSpectrum(w.grid, 16, pos.shape[1], inp.amp_sigma, w.dt_fs, batch=5)
    inten, iel = tts.run(_dev(pos), _dev(inp.species))
    assert torch.count_nonzero(inten).item() == 0
    psi0 = tts.psi[0].reshape(-1).to(torch.complex128)
    assert torch.equal(iel, (psi0.real ** 2 + psi0.imag ** 2))
    assert all(torch.equal(tts.psi[0], tts.psi[t]) for t in range(16))


def test_paper_scale_sampled_exit_waves(api):
    # 512^2 grid, 101 slices, fcc 20x20x50 (80 000 atoms): snapshots drawn
    # across the 4096-snapshot trajectory, batched as in the benchmark.
    w = W.WORKLOADS["paper_scale"]
    snaps = [0, 1365, 4095]
    inp = W.build_inputs(w)
    pos = inp.positions(snaps)
    from paper_2401_15599_gb300.pipeline import TimeToSpectrum
    tts = TimeToSpectrum(w.grid, len(snaps), pos.shape[1], inp.amp_sigma, w.dt_fs, batch=32)
    tts.prepare(None, None)
    tts.exit_waves(_dev(pos), _dev(inp.species))
    out = tts.psi.cpu().numpy()
    g = O.grid_from_spec(w.grid)
    for i in range(len(snaps)):
        v = O.projected_potential(g, pos[i].astype(np.float64), inp.species, inp.amp_sigma.astype(np.float64))
        ref = O.multislice(g, v)
        assert rel_l2(out[i], ref) < 1e-5, snaps[i]
