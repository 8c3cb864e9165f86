"""The paper-scale workload's spectrum against the FP64 oracle.

Snapshots 0, 64, ..., 4032 of the paper-scale trajectory (fcc 20x20x50 cells,
80 000 atoms, 512^2 grid over 81 A, 101 slices of 2 A, 200 keV, 5 fs steps)
form a 64-snapshot trajectory at 320 fs.  Both sides run the whole procedure
after Eq. (9) on it: slice potentials and multislice per snapshot, time mean
(elastic part), transform over time and |Phi|^2 / T^2 (Eq. (9)) on the natural
energy grid.  The GPU path is the one the benchmark times (slab potential,
staged multislice, FP32 FFT over time); the oracle runs its snapshots in a
spawn-started process pool on the host cores.  Bound: relative L2 of I(q, E)
below 2e-5, of I_el below 1e-6.  The exit waves of these snapshots carry the
physical structure (strong Bragg beams, weak inelastic part) that the
synthetic waves of the other spectrum tests lack.
"""

import os

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


def test_subsampled_paper_scale_spectrum(api):
    from paper_2401_15599_gb300.pipeline import TimeToSpectrum
    w = W.WORKLOADS["paper_scale"]
    snaps = list(range(0, w.n_t, 64))
    inp = W.build_inputs(w)
    pos = inp.positions(snaps)
    dt = 64 * w.dt_fs
    # oracle first: its pool is spawn-started, and it never touches the GPU
    g = O.grid_from_spec(w.grid)
    psi_ref = O.exit_waves(g, pos.astype(np.float64), inp.species, inp.amp_sigma.astype(np.float64),
                           processes=min(len(snaps), os.cpu_count() or 1))
    ref, ref_el, _ = O.spectrum(psi_ref.reshape(len(snaps), -1), dt)

    tts = TimeToSpectrum(w.grid, len(snaps), pos.shape[1], inp.amp_sigma, dt, batch=32, precision="fft32")
    tts.prepare(None, None)
    inten, iel = tts.run(torch.from_numpy(pos).cuda(), torch.from_numpy(inp.species).cuda())
    api.status()
    got_psi = tts.psi.cpu().numpy()
    wave_err = max(np.linalg.norm(got_psi[i] - psi_ref[i]) / np.linalg.norm(psi_ref[i]) for i in range(len(snaps)))
    got, got_el = inten.cpu().numpy().astype(np.float64), iel.cpu().numpy()
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    err_el = np.linalg.norm(got_el - ref_el) / np.linalg.norm(ref_el)
    e = O.natural_energies(len(snaps), dt)            # +-6.5 meV in steps of 0.2 meV at 320 fs
    bands = []
    for k in range(4):                                 # quarters of the energy axis
        sel = np.zeros(len(e), dtype=bool)
        sel[k * len(e) // 4:(k + 1) * len(e) // 4] = True
        sel &= e != 0.0
        bands.append((e[sel].min(), e[sel].max(),
                      np.linalg.norm(got[:, sel] - ref[:, sel]) / np.linalg.norm(ref[:, sel])))
    print(f"\nC1 64-snapshot subsample: waves {wave_err:.2e}, I {err:.2e}, I_el {err_el:.2e}; bands (meV) " +
          ", ".join(f"[{a:.2f},{b:.2f}] {x:.2e}" for a, b, x in bands))
    assert wave_err < 1e-5
    assert err < SPEC_TOL
    assert err_el < 1e-6
