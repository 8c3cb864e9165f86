"""GPU parity of the slice-potential builder when every atom's z cut-off 6 s
stays within one slice thickness, so an atom of slab k reaches only slices
k-1, k and k+1 (the band-walking kernel: one block per band of 8 rows walks the
slices with per-slab candidate lists sorted by column), against the FP64
oracle: ragged grids (odd widths, a short last band, widths that take two
column passes), one and two slices, atoms beyond both ends of the stack and
across the periodic edges, several species, and crowded slabs whose candidate
lists exceed a list slot (processed per slice in chunks).  Bound as for the
other potential tests: 2e-6 of the peak; identical configurations give
bit-identical potentials."""

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_15599_gb300 import build
    build.build()
    from paper_2401_15599_gb300 import api as A
    return A


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).to("cuda")


def _check(api, g, pos, species, amp_sigma):
    v = api.potential(g, _dev(pos), _dev(species), amp_sigma).cpu().numpy()
    for t in range(pos.shape[0]):
        ref = O.projected_potential(g, pos[t].astype(np.float64), species, np.asarray(amp_sigma, np.float64))
        assert np.max(np.abs(v[t] - ref)) <= 2e-6 * max(np.max(np.abs(ref)), 1e-30) + 1e-6, t
    return v


# (nx, ny, lx, ly, n_slices, dz): every case has 6 s_max <= dz
@pytest.mark.parametrize("shape", [(64, 64, 32.0, 32.0, 5, 2.0), (96, 40, 24.0, 10.0, 3, 2.5),
                                   (512, 512, 81.0, 81.0, 7, 2.0), (200, 136, 40.0, 27.0, 1, 2.0),
                                   (128, 128, 40.5, 40.5, 2, 2.0), (97, 61, 24.25, 15.25, 3, 2.0),
                                   (768, 100, 121.5, 15.8, 3, 2.0), (1024, 64, 162.0, 10.125, 2, 2.0)])
def test_slab_walk_matches_oracle(api, shape):
    nx, ny, lx, ly, ns, dz = shape
    g = O.Grid(nx, ny, lx, ly, ns, dz, 0.5, 200.0, 2.0 / 3.0)
    rng = np.random.default_rng(nx * 3 + ny + ns)
    amp_sigma = np.array([[20.0, 0.3], [11.0, 0.25], [27.0, 0.33]], dtype=np.float32)
    n = 300
    pos = np.stack([np.stack([rng.uniform(-1.0, lx + 1.0, n), rng.uniform(-1.0, ly + 1.0, n),
                              rng.uniform(g.z0 - 2.5, g.z0 + ns * dz + 2.5, n)], axis=1) for _ in range(2)])
    species = rng.integers(0, 3, n).astype(np.int32)
    _check(api, g, pos.astype(np.float32), species, amp_sigma)


def test_crowded_slabs(api):
    # 2000 atoms in a 6 A x 6 A x 4 A corner: hundreds of sources and candidates per slab and tile
    g = O.Grid(128, 128, 40.0, 40.0, 4, 2.0, 0.0, 200.0, 2.0 / 3.0)
    rng = np.random.default_rng(77)
    n = 2000
    pos = np.stack([rng.uniform(-3.0, 3.0, n), rng.uniform(-3.0, 3.0, n), rng.uniform(1.0, 5.0, n)], axis=1)
    species = rng.integers(0, 2, n).astype(np.int32)
    _check(api, g, pos[None].astype(np.float32), species, [[20.0, 0.3], [15.0, 0.28]])


def test_many_slices_reload_the_bin_table(api):
    # 400 slices of 0.5 A: the bin ranges of 6 bins per slab fill the table after 315
    # slabs, so the walk reloads it part-way (no staged records for that slab)
    g = O.Grid(128, 128, 20.0, 20.0, 400, 0.5, 0.0, 200.0, 2.0 / 3.0)
    rng = np.random.default_rng(9)
    n = 1500
    pos = np.stack([rng.uniform(-0.5, 20.5, n), rng.uniform(-0.5, 20.5, n), rng.uniform(-1.0, 201.0, n)], axis=1)
    species = rng.integers(0, 2, n).astype(np.int32)
    _check(api, g, pos[None].astype(np.float32), species, [[20.0, 0.08], [12.0, 0.07]])


def test_slab_walk_is_deterministic(api):
    g = O.Grid(256, 256, 40.5, 40.5, 10, 2.0, 0.0, 200.0, 2.0 / 3.0)
    rng = np.random.default_rng(5)
    n = 4000
    pos0 = np.stack([rng.uniform(0, 40.5, n), rng.uniform(0, 40.5, n), rng.uniform(0, 20.0, n)], axis=1)
    pos = np.stack([pos0, pos0]).astype(np.float32)
    species = np.zeros(n, np.int32)
    a = api.potential(g, _dev(pos), _dev(species), [[20.0, 0.3]]).cpu()
    b = api.potential(g, _dev(pos), _dev(species), [[20.0, 0.3]]).cpu()
    assert torch.equal(a[0], a[1]) and torch.equal(a, b)
