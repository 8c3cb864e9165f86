"""The allocation-free multislice entry point (tacaw_multislice_static).

Some callers cannot allocate device memory at all (a plug-in whose host
application owns every device allocation, a real-time service that forbids
allocation after start-up).  tacaw_multislice_static serves them with a
fixed scratch array inside the library.  This test calls it through the
C-ABI twice in a row and checks each result against tacaw_multislice (the
workspace entry point) on the same inputs.  It lives in a file that pytest
collects last and must pass alone in a fresh process as well as after the
other GPU tests.
"""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


class _G:
    pass


def _grid(nx, ny, n_slices):
    g = _G()
    g.nx, g.ny, g.lx, g.ly, g.n_slices, g.dz, g.z0, g.kev, g.bandlimit = \
        nx, ny, nx * 0.25, ny * 0.25, n_slices, 2.0, 0.0, 200.0, 2.0 / 3.0
    return g


def _call_static(lib, L, g, n_t, v, psi_in, out, psum, stream):
    gc = L.make_grid(g)
    return lib.tacaw_multislice_static(ctypes.byref(gc), n_t, ctypes.c_void_p(v.data_ptr()),
                                       ctypes.c_void_p(0 if psi_in is None else psi_in.data_ptr()),
                                       ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(psum.data_ptr()), 0, stream)


def test_static_scratch_multislice_matches_workspace_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_15599_gb300 import build
    build.build()
    from paper_2401_15599_gb300 import _lib as L
    from paper_2401_15599_gb300 import api
    lib = L.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(2024)
    # two calls in a row with different tables, then the plane wave (psi_in NULL)
    for nx, ny, with_psi_in in ((256, 256, True), (128, 64, True), (512, 512, False)):
        g = _grid(nx, ny, 4)
        n_t = 3
        v = torch.from_numpy(rng.uniform(0.0, 30.0, (n_t, g.n_slices, ny, nx)).astype(np.float32)).cuda()
        psi_in = None
        if with_psi_in:
            psi_in = torch.from_numpy((1.0 + 0.1 * rng.standard_normal((ny, nx))).astype(np.complex64)).cuda()
        ref = api.multislice(g, v, psi_in=psi_in)
        sum_ref = torch.zeros((ny, nx), dtype=torch.complex128, device="cuda")
        api.multislice(g, v, psi_in=psi_in, psi_sum=sum_ref)
        out = torch.full((n_t, ny, nx), float("nan"), dtype=torch.complex64, device="cuda")
        psum = torch.zeros((ny, nx), dtype=torch.complex128, device="cuda")
        L.check("tacaw_multislice_static", _call_static(lib, L, g, n_t, v, psi_in, out, psum, stream))
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 3e-6
        assert np.allclose(psum.cpu().numpy(), sum_ref.cpu().numpy(), rtol=1e-12, atol=1e-12)
    api.status()


def test_static_entry_point_allocates_no_device_memory():
    """A second call of the same size leaves the device's free memory exactly
    as it was (the first call may load the library's kernels)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_15599_gb300 import build
    build.build()
    from paper_2401_15599_gb300 import _lib as L
    lib = L.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    g = _grid(256, 256, 3)
    rng = np.random.default_rng(7)
    v = torch.from_numpy(rng.uniform(0.0, 30.0, (2, 3, 256, 256)).astype(np.float32)).cuda()
    out = torch.empty((2, 256, 256), dtype=torch.complex64, device="cuda")
    psum = torch.zeros((256, 256), dtype=torch.complex128, device="cuda")
    L.check("tacaw_multislice_static", _call_static(lib, L, g, 2, v, None, out, psum, stream))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        L.check("tacaw_multislice_static", _call_static(lib, L, g, 2, v, None, out, psum, stream))
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
