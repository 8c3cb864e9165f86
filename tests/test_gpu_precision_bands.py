"""Precision of the temporal transform per energy band.

On the paper-scale exit waves (512^2 grid, 101 slices, 4096 snapshots at 5 fs)
the explicit grid of 1024 bins over [-200, 200) meV is taken on 1024 q-points
with the three-term split-BF16 tensor-core GEMM (BF16X6, the form for explicit
grids), the FP32 SIMT GEMM and the two-term split (BF16X3, kept for timing
comparisons), against the FP64 oracle DFT.  The q-points are q = 0, every
reciprocal-lattice point of the crystal inside the band limit (the Bragg
beams, where the elastic wave is strongest and the inelastic signal is the
smallest fraction of |psi|), and a seeded random remainder.  BF16X6 and FP32
stay below 2e-5 relative L2 over all bins and in every 50 meV band; BF16X3
does not in the weak outer bands (its ~2^-16 error is relative to
sum |A||e|, not to |Phi|) and is only bounded loosely.  (Before the tensor-core
accumulators were drained into round-to-nearest FP32 sums every two K blocks,
their truncation bias alone gave 5e-5 at this T.)  The tables are printed
(pytest -s)."""

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


def band_q_points(w, n=1024, seed=7):
    """Flat FFT-order indices: q = 0, the reciprocal-lattice points of the
    supercell's ncell[0] x ncell[1] cells inside the band limit, then seeded
    random q-points up to n."""
    g = w.grid
    kmax = g.bandlimit * min(g.nx / 2.0, g.ny / 2.0 * g.lx / g.ly)     # band-limit radius in x-index units
    cx, cy = w.ncell[0], w.ncell[1]                                        # one cell = cx (cy) FFT indices apart
    beams = []
    for h in range(-g.nx // (2 * cx), g.nx // (2 * cx) + 1):
        for k in range(-g.ny // (2 * cy), g.ny // (2 * cy) + 1):
            kx, ky = h * cx, k * cy
            if kx * kx + (ky * g.lx / g.ly) ** 2 <= kmax * kmax:
                beams.append((ky % g.ny) * g.nx + (kx % g.nx))
    beams = sorted(set(beams))
    assert 0 in beams and len(beams) > 200
    rng = np.random.default_rng(seed)
    rest = np.setdiff1d(np.arange(g.nx * g.ny), beams)
    extra = rng.choice(rest, n - len(beams), replace=False)
    return np.sort(np.concatenate([np.array(beams), extra]))


@pytest.fixture(scope="module")
def waves(api):
    from paper_2401_15599_gb300.pipeline import TimeToSpectrum
    w = W.WORKLOADS["paper_scale"]
    inp = W.build_inputs(w)
    pos = torch.from_numpy(inp.positions()).cuda()
    tts = TimeToSpectrum(w.grid, pos.shape[0], pos.shape[1], inp.amp_sigma, w.dt_fs, batch=32)
    tts.prepare(None, None)
    tts.exit_waves(pos, torch.from_numpy(inp.species).cuda())
    torch.cuda.synchronize()
    del pos
    q = band_q_points(w)
    sub = tts.psi.reshape(tts.n_t, -1)[:, torch.from_numpy(q).cuda()].contiguous()
    omega = np.arange(1024) * (400.0 / 1024) - 200.0
    ref, ref_el, _ = O.spectrum(sub.cpu().numpy().astype(np.complex128), w.dt_fs, omega)
    return w, sub, omega, ref, ref_el


BAND_BOUND = {"bf16x6": SPEC_TOL, "fp32": SPEC_TOL, "bf16x3": 1e-3}   # BF16X3: timing comparisons only


@pytest.mark.parametrize("precision", ["bf16x6", "fp32", "bf16x3"])
def test_explicit_grid_per_band(api, waves, precision):
    w, sub, omega, ref, ref_el = waves
    inten, iel = api.spectrum(sub, w.dt_fs, omega_meV=omega, precision=precision)
    got = inten.cpu().numpy().astype(np.float64)
    rows = []
    for lo in range(-200, 200, 50):
        sel = (omega >= lo) & (omega < lo + 50)
        rows.append((lo, lo + 50, np.linalg.norm(got[:, sel] - ref[:, sel]) / np.linalg.norm(ref[:, sel])))
    total = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"\n{precision}: all bins {total:.2e}; per band (meV): " +
          ", ".join(f"[{a},{b}) {e:.2e}" for a, b, e in rows))
    assert total < BAND_BOUND[precision]
    for a, b, e in rows:
        assert e < BAND_BOUND[precision], (a, b, e)
    assert np.linalg.norm(iel.cpu().numpy() - ref_el) / np.linalg.norm(ref_el) < 1e-12


@pytest.mark.parametrize("n_t,nq,n_w", [(200, 777, 1024), (37, 65, 300), (1024, 2048, 512)])
def test_bf16x6_matches_oracle(api, n_t, nq, n_w):
    rng = np.random.default_rng(n_t + nq)
    z = (1.0 + 0.05 * (rng.standard_normal((n_t, nq)) + 1j * rng.standard_normal((n_t, nq)))).astype(np.complex64)
    omega = np.linspace(-150.0, 150.0, n_w, endpoint=False)
    inten, iel = api.spectrum(torch.from_numpy(z).cuda(), 5.0, omega_meV=omega, kubo=True, normalize=True,
                              precision="bf16x6")
    ref, ref_el, _ = O.spectrum(z.astype(np.complex128), 5.0, omega, kubo=True, normalize=True)
    assert np.linalg.norm(inten.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-5
    natural, _ = api.spectrum(torch.from_numpy(z).cuda(), 5.0, precision="bf16x6")
    ref_n, _, _ = O.spectrum(z.astype(np.complex128), 5.0)
    assert np.linalg.norm(natural.cpu().numpy() - ref_n) / np.linalg.norm(ref_n) < 1e-5


@pytest.mark.parametrize("precision", ["bf16x6", "fp32", "bf16x3"])
def test_explicit_grid_per_band_synthetic_waves(api, precision):
    """The same per-band bound on seeded exit-wave-like series (strong beams
    with weak phase modulation and a broadband floor; workloads.modulated_waves):
    inputs that come from neither implementation, with outer bands four orders
    of magnitude weaker than the inner ones, as in the paper-scale waves."""
    z = W.modulated_waves(4096, 2048, 5.0, n_strong=64, seed=2401)
    omega = np.arange(1024) * (400.0 / 1024) - 200.0
    inten, iel = api.spectrum(torch.from_numpy(z).cuda(), 5.0, omega_meV=omega, precision=precision)
    ref, ref_el, _ = O.spectrum(z.astype(np.complex128), 5.0, omega)
    got = inten.cpu().numpy().astype(np.float64)
    rows = []
    for lo in range(-200, 200, 50):
        sel = (omega >= lo) & (omega < lo + 50)
        rows.append((lo, lo + 50, np.linalg.norm(got[:, sel] - ref[:, sel]) / np.linalg.norm(ref[:, sel])))
    total = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"\n{precision} (synthetic): all bins {total:.2e}; per band (meV): " +
          ", ".join(f"[{a},{b}) {e:.2e}" for a, b, e in rows))
    assert total < BAND_BOUND[precision]
    for a, b, e in rows:
        assert e < BAND_BOUND[precision], (a, b, e)
    assert np.linalg.norm(iel.cpu().numpy() - ref_el) / np.linalg.norm(ref_el) < 1e-12
