"""Bounded device waits report through tacaw_status.

The multislice row pass after the first slice waits on mbarriers for the bulk
copies of its next row group.  With the wait limit set to 0 polls every such
wait gives up at once: the kernel stops, drains the copies it has issued and
returns normally (no trap, no hang), and tacaw_status reports TACAW_ETIMEOUT
once, clearing the flag.  With the default limit restored the same call gives
the oracle's exit waves and a clean status.  The split-BF16 transform reports
a clean status after a normal call.
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


def _grid(n, n_slices):
    return O.Grid(n, n, n * 0.15, n * 0.15, n_slices, 2.0, 0.0, 200.0, 2.0 / 3.0)


def test_wait_timeout_is_reported_and_cleared(api):
    from paper_2401_15599_gb300 import _lib as L
    g = _grid(256, 3)
    n_t = 64                                   # 2048 row groups: every block waits several times
    rng = np.random.default_rng(11)
    v = rng.uniform(0.0, 30.0, (n_t, g.n_slices, g.ny, g.nx)).astype(np.float32)
    V = torch.from_numpy(v).cuda()
    api.status()                               # start from a clear flag
    api.set_wait_limit(0)
    try:
        api.multislice(g, V)
        with pytest.raises(L.TacawError) as exc:
            api.status()
        assert exc.value.code == L.TACAW_ETIMEOUT
    finally:
        api.set_wait_limit(None)
    api.status()                               # read once, then clear
    out = api.multislice(g, V)
    api.status()
    got = out.cpu().numpy()
    for t in (0, 31, 63):
        ref = O.multislice(g, v[t].astype(np.float64))
        assert np.linalg.norm(got[t] - ref) / np.linalg.norm(ref) < 3e-6, t


def test_tensor_core_transform_reports_clean_status(api):
    rng = np.random.default_rng(5)
    z = (1.0 + 0.05 * (rng.standard_normal((256, 512)) + 1j * rng.standard_normal((256, 512)))).astype(np.complex64)
    omega = np.linspace(-100.0, 100.0, 384, endpoint=False)
    inten, _ = api.spectrum(torch.from_numpy(z).cuda(), 5.0, omega_meV=omega, precision="bf16x6")
    api.status()
    ref, _, _ = O.spectrum(z.astype(np.complex128), 5.0, omega)
    assert np.linalg.norm(inten.cpu().numpy() - ref) / np.linalg.norm(ref) < 2e-5
