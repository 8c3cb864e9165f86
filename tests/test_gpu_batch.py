"""Batched uneven jobs: tacaw_multislice_batch against one tacaw_multislice
call per job, the batched time-to-spectrum against the FP64 oracle, and CUDA
graph capture / replay against the eager run."""

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
    from paper_2401_15599_gb300 import api as a
    return a


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_batch_equals_individual_calls(api):
    rng = np.random.default_rng(0)
    specs = [(64, 3, 3), (384, 5, 2), (128, 2, 5), (768, 4, 1), (256, 1, 4), (64, 6, 7), (384, 2, 3)]
    jobs, refs = [], []
    for i, (n, ns, nt) in enumerate(specs):
        g = W.GridSpec(n, n, n * 0.158203125, n * 0.158203125, ns, 2.0, 0.0, 200.0 if i % 2 else 100.0)
        v = torch.from_numpy(rng.uniform(0, 30, (nt, ns, n, n)).astype(np.float32)).cuda()
        psi_in = None
        if i == 5:
            psi_in = torch.from_numpy((1 + 0.1 * rng.standard_normal((n, n))).astype(np.complex64)).cuda()
        out = torch.empty((nt, n, n), dtype=torch.complex64, device="cuda")
        s = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
        jobs.append({"grid": g, "V": v, "out": out, "psi_in": psi_in, "psi_sum": s})
        s_ref = torch.zeros_like(s)
        refs.append((api.multislice(g, v, psi_in=psi_in, psi_sum=s_ref), s_ref))
    api.multislice_batch(jobs)
    for j, (ref, s_ref) in zip(jobs, refs):
        assert torch.equal(j["out"], ref)
        assert torch.allclose(j["psi_sum"], s_ref, rtol=1e-12, atol=1e-12)


def _small_jobs():
    jobs = W.batching_jobs(n_jobs=4, seed0=2000, sizes=(64, 128), slices=(2, 4), snapshots=(8, 24), n_modes=6)
    out = []
    for w in jobs:
        inp = W.build_inputs(w)
        out.append((w, inp, inp.positions()))
    return out


@pytest.mark.parametrize("precision,queue", [("fp32", "auto"), ("bf16x3", "auto"), ("fp32", True)])
def test_batch_time_to_spectrum_matches_oracle(api, precision, queue):
    """Both multislice engines of the batched driver (per-slice launches, the
    default at windows this small, and the work queue) against the oracle."""
    from paper_2401_15599_gb300.batch import BatchTimeToSpectrum, Job
    cases = _small_jobs()
    jobs = [Job(w.grid, torch.from_numpy(p).cuda(), torch.from_numpy(inp.species).cuda(), inp.amp_sigma, w.dt_fs)
            for w, inp, p in cases]
    if queue is True and not all(w.grid.nx == w.grid.ny for w, _, _ in cases):
        pytest.skip("the work queue runs square grids")
    run = BatchTimeToSpectrum(jobs, window=5, precision=precision, queue=queue)
    run.prepare()
    res = run.run()
    torch.cuda.synchronize()
    for (w, inp, p), (inten, iel) in zip(cases, res):
        g = O.grid_from_spec(w.grid)
        psi = O.exit_waves(g, p.astype(np.float64), inp.species, inp.amp_sigma.astype(np.float64))
        ref, ref_el, _ = O.spectrum(psi, w.dt_fs)
        assert rel_l2(inten.cpu().numpy(), ref) < 2e-5
        assert rel_l2(iel.cpu().numpy(), ref_el) < 1e-6


def test_batch_graph_capture_replay(api):
    from paper_2401_15599_gb300.batch import BatchTimeToSpectrum, Job
    cases = _small_jobs()
    jobs = [Job(w.grid, torch.from_numpy(p).cuda(), torch.from_numpy(inp.species).cuda(), inp.amp_sigma, w.dt_fs)
            for w, inp, p in cases]
    run = BatchTimeToSpectrum(jobs, window=7)
    run.capture()
    eager = [(i.clone(), e.clone()) for i, e in run.run()]
    for st in run.state:
        st["I"].zero_()
    replayed = run.replay()
    torch.cuda.synchronize()
    for (a, ae), (b, be) in zip(eager, replayed):
        assert torch.equal(a, b)
        assert torch.equal(ae, be)


@pytest.mark.parametrize("precision", ["bf16x6", "fp32"])
def test_chunked_batch_matches_oracle(api, precision):
    """Time-chunked batched spectra (one window of exit waves per job, Phi
    accumulated per window, positions synthesised on the device per window)
    against the oracle's spectrum of each whole trajectory on an explicit
    energy grid."""
    from paper_2401_15599_gb300.batch import BatchTimeToSpectrum, Job
    cases = _small_jobs()
    omega = np.arange(256) * (400.0 / 256) - 200.0
    jobs = []
    for w, inp, p in cases:
        jobs.append(Job(w.grid, None, torch.from_numpy(inp.species).cuda(), inp.amp_sigma, w.dt_fs,
                        omega_meV=omega, n_t=w.n_t, positions=inp.synth("cuda")))
    run = BatchTimeToSpectrum(jobs, window=5, precision=precision, chunked=True,
                              queue=all(w.grid.nx == w.grid.ny for w, _, _ in cases))
    run.prepare()
    res = run.run()
    torch.cuda.synchronize()
    for (w, inp, p), (inten, iel) in zip(cases, res):
        g = O.grid_from_spec(w.grid)
        psi = O.exit_waves(g, p.astype(np.float64), inp.species, inp.amp_sigma.astype(np.float64))
        ref, ref_el, _ = O.spectrum(psi, w.dt_fs, omega)
        assert rel_l2(inten.cpu().numpy(), ref) < 2e-5
        assert rel_l2(iel.cpu().numpy(), ref_el) < 1e-6
    # the same run as one CUDA graph gives the same bits
    eager = [(i.clone(), e.clone()) for i, e in res]
    run.capture()
    for st in run.state:
        st["I"].zero_()
    for (a, ae), (b, be) in zip(eager, run.replay()):
        assert torch.equal(a, b) and torch.equal(ae, be)
