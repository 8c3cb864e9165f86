"""C-ABI checks that need no GPU: the library loads, exports every function
declared in include/tacaw.h, reports workspace sizes and rejects bad
arguments on the host before anything is enqueued."""

import ctypes
import os
import re

import pytest

import oracle as O
from paper_2401_15599_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tacaw.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2401_15599_gb300 import build
    build.build()
    return L.load()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tacaw_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("tacaw_potential", "tacaw_multislice", "tacaw_spectrum", "tacaw_spectrum_backward"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name
    assert set(_declared_functions()) <= set(L.SIGNATURES)


def test_version_and_beam_constants(lib):
    assert lib.tacaw_version() >= 100
    for kev in (60.0, 100.0, 200.0, 300.0):
        lam, sig = ctypes.c_double(), ctypes.c_double()
        assert lib.tacaw_beam_constants(kev, ctypes.byref(lam), ctypes.byref(sig)) == 0
        assert lam.value == pytest.approx(O.wavelength(kev), rel=1e-14)
        assert sig.value == pytest.approx(O.interaction_constant(kev), rel=1e-14)
    assert lib.tacaw_beam_constants(-1.0, ctypes.byref(lam), ctypes.byref(sig)) == L.TACAW_EINVAL
    assert b"bad argument" in lib.tacaw_last_error()


def _grid(nx=64, ny=64, n_slices=8):
    class G:
        pass
    g = G()
    g.nx, g.ny, g.lx, g.ly, g.n_slices, g.dz, g.z0, g.kev, g.bandlimit = \
        nx, ny, 32.0, 32.0, n_slices, 4.0, 0.0, 100.0, 2.0 / 3.0
    return L.make_grid(g)


def test_workspace_queries(lib):
    g = _grid()
    n = ctypes.c_size_t(0)
    null = ctypes.c_void_p(0)
    assert lib.tacaw_multislice(ctypes.byref(g), 4, null, null, null, null, 0, null, ctypes.byref(n), null) == 0
    assert 0 < n.value < 1 << 20
    amp = (ctypes.c_float * 2)(20.0, 0.3)
    n2 = ctypes.c_size_t(0)
    assert lib.tacaw_potential(ctypes.byref(g), 4, 512, null, null, 1, amp, null, null, ctypes.byref(n2), null) == 0
    assert n2.value >= 4 * 512 * 16
    n3 = ctypes.c_size_t(0)
    assert lib.tacaw_spectrum(4096, 256, 5.0, 256, null, null, null, null, null, L.TACAW_FP32, 0, 300.0,
                              null, ctypes.byref(n3), null) == 0
    assert n3.value >= 4096 * 256 * 8 + 256 * 256 * 8


def test_host_side_argument_errors(lib):
    null = ctypes.c_void_p(0)
    n = ctypes.c_size_t(0)
    bad = _grid(nx=100)
    assert lib.tacaw_multislice(ctypes.byref(bad), 4, null, null, null, null, 0, null, ctypes.byref(n),
                                null) == L.TACAW_EUNSUPPORTED
    assert b"nx = 100" in lib.tacaw_last_error()
    g = _grid()
    assert lib.tacaw_multislice(ctypes.byref(g), -1, null, null, null, null, 0, null, ctypes.byref(n),
                                null) == L.TACAW_EINVAL
    assert lib.tacaw_multislice(None, 1, null, null, null, null, 0, null, ctypes.byref(n), null) == L.TACAW_EINVAL
    # short workspace -> ENOMEM, checked before any launch
    fake = ctypes.c_void_p(1 << 20)
    small = ctypes.c_size_t(16)
    assert lib.tacaw_multislice(ctypes.byref(g), 1, fake, null, fake, null, 0, fake, ctypes.byref(small),
                                null) == L.TACAW_ENOMEM
    amp = (ctypes.c_float * 2)(20.0, 20.0)      # 6 sigma = 120 A > half the box
    assert lib.tacaw_potential(ctypes.byref(g), 1, 1, fake, fake, 1, amp, fake, fake,
                               ctypes.byref(ctypes.c_size_t(1 << 30)), null) == L.TACAW_EINVAL
    assert lib.tacaw_potential(ctypes.byref(g), 1, 1, fake, fake, 9, amp, fake, fake,
                               ctypes.byref(ctypes.c_size_t(1 << 30)), null) == L.TACAW_EINVAL
    # pixel pairs are packed in 16 + 16 bits while binning
    amp = (ctypes.c_float * 2)(20.0, 0.3)
    wide = _grid(nx=70000)
    assert lib.tacaw_potential(ctypes.byref(wide), 1, 1, fake, fake, 1, amp, fake, fake,
                               ctypes.byref(ctypes.c_size_t(1 << 40)), null) == L.TACAW_EUNSUPPORTED
    assert b"65535" in lib.tacaw_last_error()
    # a width reaching 192 pixels and 3 slabs either side: too many neighbouring bins per tile
    fine = _grid(nx=512, ny=512)
    amp = (ctypes.c_float * 2)(20.0, 2.0)
    assert lib.tacaw_potential(ctypes.byref(fine), 1, 1, fake, fake, 1, amp, fake, fake,
                               ctypes.byref(ctypes.c_size_t(1 << 40)), null) == L.TACAW_EUNSUPPORTED
    assert b"neighbouring bins" in lib.tacaw_last_error()
    # spectrum: natural grid needs n_omega == T; Kubo needs a temperature
    assert lib.tacaw_spectrum(16, 8, 5.0, 9, null, fake, null, fake, null, 0, 0, 300.0, null,
                              ctypes.byref(n), null) == L.TACAW_EINVAL
    assert lib.tacaw_spectrum(16, 8, 5.0, 8, null, fake, null, fake, null, 0, L.TACAW_KUBO, 0.0, null,
                              ctypes.byref(n), null) == L.TACAW_EINVAL
    assert lib.tacaw_spectrum(16, 8, 5.0, 8, null, fake, null, fake, null, 7, 0, 300.0, null,
                              ctypes.byref(n), null) == L.TACAW_EINVAL


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(L, "_lib", None)
    monkeypatch.setattr(L, "LIB_PATH", str(tmp_path / "libtacaw.so"))
    with pytest.raises(RuntimeError, match="not built"):
        L.load()


def test_queue_arguments_and_workspace(lib):
    """tacaw_multislice_queue and the TACAW_MS_QUEUE flag: square grids only,
    the flag alone, and a workspace that grows by 8 bytes per snapshot."""
    fake = ctypes.c_void_p(1 << 20)
    null = ctypes.c_void_p(0)

    def grid(nx, ny):
        return L.make_grid(O.Grid(nx, ny, nx * 0.15, ny * 0.15, 3, 2.0, 0.0, 200.0, 2.0 / 3.0))

    def queue_bytes(jobs):
        arr = (L.TacawJob * len(jobs))(*jobs)
        n = ctypes.c_size_t(0)
        assert lib.tacaw_multislice_queue(arr, len(jobs), 0, 0, null, ctypes.byref(n), null) == L.TACAW_OK
        return n.value

    g = grid(256, 256)
    one = queue_bytes([L.TacawJob(g, 10, fake, None, fake, None)])
    two = queue_bytes([L.TacawJob(g, 10, fake, None, fake, None), L.TacawJob(g, 30, fake, None, fake, None)])
    tables = ctypes.c_size_t(0)
    assert lib.tacaw_multislice(ctypes.byref(g), 10, null, null, null, null, 0, null, ctypes.byref(tables),
                                null) == L.TACAW_OK
    assert one >= tables.value + 8 * 10 + 16
    assert two >= 2 * tables.value + 8 * 40 + 16
    flag = ctypes.c_size_t(0)
    assert lib.tacaw_multislice(ctypes.byref(g), 10, null, null, null, null, L.TACAW_MS_QUEUE, null,
                                ctypes.byref(flag), null) == L.TACAW_OK
    assert flag.value == one
    big = ctypes.byref(ctypes.c_size_t(1 << 40))
    rect = grid(256, 128)
    arr = (L.TacawJob * 1)(L.TacawJob(rect, 4, fake, None, fake, None))
    assert lib.tacaw_multislice_queue(arr, 1, 0, 0, fake, big, null) == L.TACAW_EUNSUPPORTED
    assert lib.tacaw_multislice(ctypes.byref(rect), 4, fake, null, fake, null, L.TACAW_MS_QUEUE, fake, big,
                                null) == L.TACAW_EUNSUPPORTED
    assert lib.tacaw_multislice(ctypes.byref(g), 4, fake, null, fake, null, L.TACAW_MS_QUEUE | L.TACAW_MS_WARP_ROWS,
                                fake, big, null) == L.TACAW_EINVAL
    arr = (L.TacawJob * 1)(L.TacawJob(g, 4, fake, None, fake, None))
    assert lib.tacaw_multislice_queue(arr, 1, -1, 0, fake, big, null) == L.TACAW_EINVAL
    arr = (L.TacawJob * 1)(L.TacawJob(g, 4, None, None, fake, None))
    assert lib.tacaw_multislice_queue(arr, 1, 0, 0, fake, big, null) == L.TACAW_EINVAL


def test_queue_workspace_query_takes_any_pointer(lib):
    """The workspace query answers before the arrays are checked (callers
    query with placeholder pointers); a real call checks their alignment."""
    g = L.make_grid(O.Grid(256, 256, 38.4, 38.4, 3, 2.0, 0.0, 200.0, 2.0 / 3.0))
    arr = (L.TacawJob * 1)(L.TacawJob(g, 8, 1, None, 1, None))
    n = ctypes.c_size_t(0)
    assert lib.tacaw_multislice_queue(arr, 1, 0, 0, None, ctypes.byref(n), None) == L.TACAW_OK and n.value > 0
    big = ctypes.byref(ctypes.c_size_t(1 << 40))
    assert lib.tacaw_multislice_queue(arr, 1, 0, 0, ctypes.c_void_p(1 << 20), big, None) == L.TACAW_EINVAL
    assert b"16-byte aligned" in lib.tacaw_last_error()
