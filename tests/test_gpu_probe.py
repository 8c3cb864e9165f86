"""GPU parity of the convergent-probe incident wave (tacaw_probe, through the
C-ABI) against the FP64 oracle, alone and as psi_in of the multislice.

The GPU probe is an FP64 pruned DFT rounded once to float: relative L2 below
1e-7 of the oracle (whose lambda is computed independently, so aperture
radii are chosen away from grid-point radii).  Through the FP32 multislice the
exit waves keep the multislice bound of 3e-6.
"""

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


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _grid(nx, ny, lx, ly, n_slices=3, dz=2.0, kev=200.0):
    return O.Grid(nx, ny, lx, ly, n_slices, dz, 0.0, kev, 2.0 / 3.0)


@pytest.mark.parametrize("nx,ny,lx,ly,alpha,defocus,x0,y0", [
    (512, 512, 81.0, 81.0, 1.0, 0.0, 0.0, 0.0),          # the paper's 200 kV, 1 mrad probe
    (256, 256, 40.5, 40.5, 21.7, 35.0, 20.25, 10.0),
    (384, 128, 60.0, 20.0, 12.3, -50.0, 3.3, 17.9),
    (64, 64, 16.0, 16.0, 500.0, 0.0, 8.0, 8.0),          # aperture beyond Nyquist: every q
    (128, 96, 32.0, 24.0, 1e-3, 0.0, 0.0, 0.0),          # only q = 0: the plane wave
])
def test_probe_matches_oracle(api, nx, ny, lx, ly, alpha, defocus, x0, y0):
    g = _grid(nx, ny, lx, ly)
    got = api.probe(g, alpha, defocus, x0, y0).cpu().numpy()
    ref = O.probe(g, alpha, defocus, x0, y0)
    assert rel_l2(got, ref) < 1e-7
    assert np.mean(np.abs(got.astype(np.complex128)) ** 2) == pytest.approx(1.0, abs=1e-6)


def test_probe_through_multislice(api):
    g = _grid(256, 256, 40.5, 40.5, n_slices=4)
    rng = np.random.default_rng(41)
    pos = np.stack([rng.uniform(0, g.lx, 300), rng.uniform(0, g.ly, 300), rng.uniform(0, 8.0, 300)], axis=1)
    v = O.projected_potential(g, pos, np.zeros(300, np.int32), [[20.0, 0.3]]).astype(np.float32)
    psi_in = api.probe(g, 18.0, defocus_A=25.0, x0=20.0, y0=20.0)
    got = api.multislice(g, torch.as_tensor(v[None]).cuda(), psi_in=psi_in).cpu().numpy()[0]
    ref = O.multislice(g, v.astype(np.float64), psi_in=O.probe(g, 18.0, defocus_A=25.0, x0=20.0, y0=20.0))
    assert rel_l2(got, ref) < 3e-6


def test_probe_errors(api):
    g = _grid(64, 64, 16.0, 16.0)
    with pytest.raises(RuntimeError):
        api.probe(g, -1.0)
    with pytest.raises(RuntimeError):
        api.probe(_grid(64, 64, 16.0, 16.0, kev=-5.0), 1.0)
