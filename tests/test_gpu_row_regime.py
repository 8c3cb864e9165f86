"""The multislice row pass in the regime the benchmark runs it in.

After the first slice the row pass is a persistent grid: each block walks
many row groups through a two-stage shared-memory ring filled by bulk
asynchronous copies, so stage reuse, the mbarrier phase flips and the
prefetch of the next group all take part.  These calls hold several to many
row groups per resident block (2048 and 4096 groups, and a long call of
16384), and every snapshot's exit wave is compared element by element with
the FP64 oracle (second step of the procedure after Eq. (9): the multislice
of each snapshot), as well as the FP64 running sum over snapshots.  Both
thread layouts of the 512-point row pass are covered (two warps per row, and
one warp per row with 16 values per thread), and both forms of the
512-point column pass (the persistent pass with TMA-staged tiles, and one
block per column block).
"""

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WAVE_TOL = 3e-6


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_15599_gb300 import build
    build.build()
    from paper_2401_15599_gb300 import api as A
    return A


def _grid(n, n_slices, pixel=0.158203125):
    return O.Grid(n, n, n * pixel, n * pixel, n_slices, 2.0, 0.0, 200.0, 2.0 / 3.0)


@pytest.mark.parametrize("n,n_slices,n_t,with_psi_in,ms_flags", [
    (256, 4, 64, False, 0),          # 32 groups of 8 rows per snapshot: 2048 groups
    (512, 3, 32, True, 0),           # 128 groups of 4 rows per snapshot: 4096 groups; staged columns
    (512, 2, 128, False, 0),         # 16384 groups, about 27 per resident block
    (512, 3, 32, True, 1),           # one warp per row: 64 groups of 8 rows per snapshot
    (512, 2, 128, False, 1),
    (512, 3, 32, True, 2),           # one block per column block
    (512, 2, 64, False, 3),
])
def test_row_pass_many_groups_per_block(api, n, n_slices, n_t, with_psi_in, ms_flags):
    g = _grid(n, n_slices)
    rng = np.random.default_rng(1000 + n + n_t)
    v = rng.uniform(0.0, 30.0, (n_t, n_slices, n, n)).astype(np.float32)
    psi_in = None
    if with_psi_in:
        psi_in = (1.0 + 0.1 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))).astype(np.complex64)
    V = torch.from_numpy(v).cuda()
    pin = None if psi_in is None else torch.from_numpy(psi_in).cuda()
    psum = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
    out = api.multislice(g, V, psi_in=pin, psi_sum=psum, ms_flags=ms_flags)
    api.status()
    got = out.cpu().numpy()
    ref_sum = np.zeros((n, n), dtype=np.complex128)
    worst, worst_abs = 0.0, 0.0
    for t in range(n_t):
        ref = O.multislice(g, v[t].astype(np.float64), None if psi_in is None else psi_in.astype(np.complex128))
        ref_sum += ref
        err = np.linalg.norm(got[t] - ref) / np.linalg.norm(ref)
        worst = max(worst, err)
        worst_abs = max(worst_abs, float(np.max(np.abs(got[t] - ref))))
        assert err < WAVE_TOL, (t, err)
    print(f"\n{n}^2 x {n_slices} slices x {n_t} snapshots (flags {ms_flags}): worst rel-L2 {worst:.2e}, max |diff| {worst_abs:.2e}")
    # the FP64 running sum adds the FP32 exit waves: compare it with their own sum, and with the oracle's
    own = got.astype(np.complex128).sum(axis=0)
    assert np.allclose(psum.cpu().numpy(), own, rtol=1e-12, atol=1e-12)
    assert np.linalg.norm(psum.cpu().numpy() - ref_sum) / np.linalg.norm(ref_sum) < WAVE_TOL
