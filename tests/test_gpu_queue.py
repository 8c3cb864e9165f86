"""The persistent work-queue multislice (tacaw_multislice_queue, and
tacaw_multislice with TACAW_MS_QUEUE).

Every snapshot is an independent multislice run (second step of the
procedure after Eq. (9)); the queue only changes which block runs which pass
of which slice, and when.  So its exit waves must equal those of the
per-slice launches bit for bit, and the oracle's to the FP32 tolerance.  The
cases drive the queue through several waves (a partial last one included),
jobs of different sizes, slice counts and lengths in one call, dependency
waits in every pass, and a wait limit of 0 polls (every dependent item gives
up at once: the launch stops and tacaw_status reports the timeout).
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


def _grid(n, n_slices, pixel=0.158203125, kev=200.0):
    return O.Grid(n, n, n * pixel, n * pixel, n_slices, 2.0, 0.0, kev, 2.0 / 3.0)


def _potentials(rng, n_t, g):
    return rng.uniform(0.0, 30.0, (n_t, g.n_slices, g.ny, g.nx)).astype(np.float32)


def _incident(rng, n):
    return (1.0 + 0.1 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))).astype(np.complex64)


@pytest.mark.parametrize("n,n_slices,n_t,wave,span,with_psi_in", [
    (256, 4, 13, 4, 8, False),     # waves of 4, 4, 4 and 1 snapshots; items of one 8-row tile
    (512, 3, 20, 8, 0, True),      # 32 row and 32 column items per snapshot and slice
    (512, 2, 80, 0, 64, False),    # default wave (64 at 512^2): a full and a partial wave; 8 items per pass
    (64, 5, 33, 7, 0, True),
    (1024, 2, 3, 2, 32, False),
])
def test_queue_equals_per_slice_launches(api, n, n_slices, n_t, wave, span, with_psi_in):
    g = _grid(n, n_slices)
    rng = np.random.default_rng(500 + n + n_t)
    v = _potentials(rng, n_t, g)
    psi_in = _incident(rng, n) if with_psi_in else None
    V = torch.from_numpy(v).cuda()
    pin = None if psi_in is None else torch.from_numpy(psi_in).cuda()
    s_ref = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
    ref = api.multislice(g, V, psi_in=pin, psi_sum=s_ref)
    out = torch.full((n_t, n, n), float("nan"), dtype=torch.complex64, device="cuda")
    s_q = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
    api.multislice_batch([dict(grid=g, V=V, out=out, psi_in=pin, psi_sum=s_q)], queue=True, wave=wave, span=span)
    api.status()
    assert torch.equal(out, ref), float((out - ref).abs().max())
    assert torch.equal(s_q, s_ref)
    got = out.cpu().numpy()
    for t in sorted({0, n_t // 2, n_t - 1}):
        want = O.multislice(g, v[t].astype(np.float64), None if psi_in is None else psi_in.astype(np.complex128))
        assert np.linalg.norm(got[t] - want) / np.linalg.norm(want) < WAVE_TOL, t


def test_queue_flag_of_tacaw_multislice(api):
    from paper_2401_15599_gb300 import _lib as L
    g = _grid(512, 4)
    rng = np.random.default_rng(77)
    v = _potentials(rng, 24, g)
    V = torch.from_numpy(v).cuda()
    s0 = torch.zeros((512, 512), dtype=torch.complex128, device="cuda")
    s1 = torch.zeros_like(s0)
    a = api.multislice(g, V, psi_sum=s0)
    b = api.multislice(g, V, psi_sum=s1, ms_flags=L.TACAW_MS_QUEUE)
    api.status()
    assert torch.equal(a, b) and torch.equal(s0, s1)


def test_queue_uneven_jobs_in_one_call(api):
    """Jobs of four grid sizes (one launch each), different slice counts,
    lengths, energies and incident waves, interleaved in the job list."""
    specs = [(256, 5, 9, 200.0, False), (128, 3, 17, 100.0, True), (384, 2, 5, 200.0, False),
             (256, 2, 21, 300.0, True), (768, 3, 3, 200.0, False), (128, 6, 4, 200.0, False)]
    rng = np.random.default_rng(4242)
    jobs_b, jobs_q, host = [], [], []
    for n, ns, n_t, kev, with_in in specs:
        g = _grid(n, ns, kev=kev)
        v = _potentials(rng, n_t, g)
        pin = _incident(rng, n) if with_in else None
        V = torch.from_numpy(v).cuda()
        P = None if pin is None else torch.from_numpy(pin).cuda()
        host.append((g, v, pin))
        for lst in (jobs_b, jobs_q):
            lst.append(dict(grid=g, V=V, psi_in=P,
                            out=torch.full((n_t, n, n), float("nan"), dtype=torch.complex64, device="cuda"),
                            psi_sum=torch.zeros((n, n), dtype=torch.complex128, device="cuda")))
    api.multislice_batch(jobs_b)
    api.multislice_batch(jobs_q, queue=True, wave=3)
    api.status()
    for jb, jq, (g, v, pin) in zip(jobs_b, jobs_q, host):
        assert torch.equal(jb["out"], jq["out"]), g.nx
        assert torch.equal(jb["psi_sum"], jq["psi_sum"]), g.nx
        got = jq["out"].cpu().numpy()
        t = v.shape[0] - 1
        want = O.multislice(g, v[t].astype(np.float64), None if pin is None else pin.astype(np.complex128))
        assert np.linalg.norm(got[t] - want) / np.linalg.norm(want) < WAVE_TOL, g.nx


def test_queue_wait_timeout_is_reported(api):
    from paper_2401_15599_gb300 import _lib as L
    g = _grid(256, 3)
    rng = np.random.default_rng(3)
    V = torch.from_numpy(_potentials(rng, 8, g)).cuda()
    out = torch.empty((8, 256, 256), dtype=torch.complex64, device="cuda")
    api.status()
    api.set_wait_limit(0)
    try:
        api.multislice_batch([dict(grid=g, V=V, out=out)], queue=True)
        with pytest.raises(L.TacawError) as exc:
            api.status()
        assert exc.value.code == L.TACAW_ETIMEOUT
    finally:
        api.set_wait_limit(None)
    api.status()
    api.multislice_batch([dict(grid=g, V=V, out=out)], queue=True)
    api.status()
    assert torch.equal(out, api.multislice(g, V))
