"""The sharded time-to-spectrum driver with the library's kernels (one rank:
the collectives are identities, every other step is the multi-GPU code path):
slice potentials and multislice of the rank's snapshots, the FP64 mean,
Phi accumulated with global times and finished, against the FP64 oracle
spectrum of the whole trajectory on an explicit energy grid and on the
natural energies."""

import numpy as np
import pytest

import oracle as O
import workloads as W

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


@pytest.mark.parametrize("natural", [False, True])
def test_one_rank_sharded_spectrum_matches_oracle(api, natural):
    from paper_2401_15599_gb300.sharded import ShardedTimeToSpectrum
    w = W.WORKLOADS["plain_small"].with_(n_t=64)
    inp = W.build_inputs(w)
    pos = inp.positions()
    omega = O.natural_energies(w.n_t, w.dt_fs) if natural else np.arange(384) * (300.0 / 384) - 150.0
    sh = ShardedTimeToSpectrum(w.grid, w.n_t, pos.shape[1], inp.amp_sigma, w.dt_fs, omega, batch=16,
                               precision="bf16x6", kubo=True)
    inten, iel = sh.run(torch.from_numpy(pos).cuda(), torch.from_numpy(inp.species).cuda())
    api.status()
    g = O.grid_from_spec(w.grid)
    psi = O.exit_waves(g, pos.astype(np.float64), inp.species, inp.amp_sigma.astype(np.float64))
    ref, ref_el, _ = O.spectrum(psi, w.dt_fs, None if natural else omega, kubo=True)
    got = inten.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 2e-5
    assert np.linalg.norm(iel.cpu().numpy() - ref_el) / np.linalg.norm(ref_el) < 1e-6
