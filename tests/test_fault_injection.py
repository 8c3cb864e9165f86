"""Host-side fault injection (no GPU needed): with TACAW_FAULT=launch every
computing entry point returns TACAW_ECUDA just before it would enqueue work,
with TACAW_FAULT=symbol the lookups of the library's device variables fail,
and with TACAW_FAULT=timeout tacaw_status reports a bounded-wait timeout.
Arguments are valid, and the device pointers are never touched: the fault is
raised on the host before any CUDA call."""

import ctypes

import pytest

from paper_2401_15599_gb300 import _lib as L

FAKE = ctypes.c_void_p(1 << 20)            # 256-byte aligned, never dereferenced
NULL = ctypes.c_void_p(0)


@pytest.fixture(scope="module")
def lib():
    from paper_2401_15599_gb300 import build
    build.build()
    return L.load()


def _grid(nx=64, ny=64, n_slices=4):
    class G:
        pass
    g = G()
    g.nx, g.ny, g.lx, g.ly, g.n_slices, g.dz, g.z0, g.kev, g.bandlimit = \
        nx, ny, 32.0, 32.0, n_slices, 2.0, 0.0, 200.0, 2.0 / 3.0
    return L.make_grid(g)


def _big():
    return ctypes.byref(ctypes.c_size_t(1 << 40))


def _entry_points(lib):
    """(name, call) for every entry point that enqueues device work."""
    g = _grid()
    amp = (ctypes.c_float * 2)(20.0, 0.3)
    jobs = (L.TacawJob * 1)(L.TacawJob(g, 2, FAKE, None, FAKE, None))
    cands = (ctypes.c_int32 * 2)(1, 2)
    ms = (ctypes.c_float * 2)()
    best = ctypes.c_int32(0)
    return [
        ("tacaw_potential", lambda: lib.tacaw_potential(ctypes.byref(g), 2, 4, FAKE, FAKE, 1, amp, FAKE, FAKE,
                                                        _big(), NULL)),
        ("tacaw_multislice", lambda: lib.tacaw_multislice(ctypes.byref(g), 2, FAKE, NULL, FAKE, NULL, 0, FAKE,
                                                          _big(), NULL)),
        ("tacaw_multislice_static", lambda: lib.tacaw_multislice_static(ctypes.byref(g), 2, FAKE, NULL, FAKE,
                                                                        NULL, 0, NULL)),
        ("tacaw_multislice_batch", lambda: lib.tacaw_multislice_batch(jobs, 1, FAKE, _big(), NULL)),
        ("tacaw_multislice_queue", lambda: lib.tacaw_multislice_queue(jobs, 1, 0, 0, FAKE, _big(), NULL)),
        ("tacaw_spectrum", lambda: lib.tacaw_spectrum(64, 8, 5.0, 8, NULL, FAKE, NULL, FAKE, FAKE, L.TACAW_FP32, 0,
                                                      300.0, FAKE, _big(), NULL)),
        ("tacaw_spectrum_segments", lambda: lib.tacaw_spectrum_segments(64, 16, 5.0, 8, 4, 0, 8, NULL, FAKE, FAKE,
                                                                        FAKE, L.TACAW_FP32, 0, 300.0, FAKE, _big(),
                                                                        NULL)),
        ("tacaw_spectrum_backward", lambda: lib.tacaw_spectrum_backward(64, 8, 5.0, 8, NULL, FAKE, NULL, FAKE, FAKE,
                                                                        FAKE, _big(), NULL)),
        ("tacaw_multislice_backward", lambda: lib.tacaw_multislice_backward(ctypes.byref(g), 2, FAKE, NULL, FAKE,
                                                                            FAKE, 0, FAKE, _big(), NULL)),
        ("tacaw_potential_backward", lambda: lib.tacaw_potential_backward(ctypes.byref(g), 2, 4, FAKE, FAKE, 1, amp,
                                                                          FAKE, FAKE, FAKE, _big(), NULL)),
        ("tacaw_qep_intensity", lambda: lib.tacaw_qep_intensity(64, 8, 0, 1, 0, FAKE, FAKE, NULL)),
        ("tacaw_energy_integral", lambda: lib.tacaw_energy_integral(64, 8, FAKE, FAKE, FAKE, NULL)),
        ("tacaw_line_profile", lambda: lib.tacaw_line_profile(8, 8, 32.0, 0.025, FAKE, FAKE, FAKE, NULL)),
        ("tacaw_azimuthal_profile", lambda: lib.tacaw_azimuthal_profile(8, 8, 32.0, 32.0, 0.025, 1.0, 4, FAKE, FAKE,
                                                                        FAKE, FAKE, _big(), NULL)),
        ("tacaw_relative_difference", lambda: lib.tacaw_relative_difference(16, FAKE, FAKE, FAKE, NULL)),
        ("tacaw_probe", lambda: lib.tacaw_probe(64, 64, 32.0, 32.0, 200.0, 1.0, 0.0, 0.0, 0.0, FAKE, FAKE, _big(),
                                                NULL)),
        ("tacaw_time_mean", lambda: lib.tacaw_time_mean(64, 8, FAKE, FAKE, NULL)),
        ("tacaw_time_to_spectrum_host", lambda: lib.tacaw_time_to_spectrum_host(
            ctypes.byref(g), 64, 4, FAKE, FAKE, 1, amp, 5.0, 16, 0, L.TACAW_FFT32, 0, 300.0, FAKE, FAKE, FAKE, _big(),
            NULL)),
        ("tacaw_spectrum_accumulate", lambda: lib.tacaw_spectrum_accumulate(64, 0, 8, 5.0, 16, FAKE, FAKE, FAKE, FAKE,
                                                                            L.TACAW_FP32, FAKE, _big(), NULL)),
        ("tacaw_spectrum_finish", lambda: lib.tacaw_spectrum_finish(64, 8, 5.0, 16, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE,
                                                                    0, 300.0, FAKE, _big(), NULL)),
        ("tacaw_tune_multislice", lambda: lib.tacaw_tune_multislice(ctypes.byref(g), 2, FAKE, FAKE, cands, 2, 1, 0,
                                                                    ms, ctypes.byref(best), FAKE, _big(), NULL)),
    ]


def test_every_computing_entry_point_is_covered(lib):
    import re
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(root, "include", "tacaw.h")).read(), flags=re.S)
    declared = set(re.findall(r"\b(tacaw_\w+)\s*\(", text))
    host_only = {"tacaw_last_error", "tacaw_version", "tacaw_beam_constants", "tacaw_status",
                 "tacaw_set_wait_limit"}
    assert declared - host_only == {name for name, _ in _entry_points(lib)}


def test_injected_launch_failure_gives_ecuda(lib, monkeypatch):
    monkeypatch.setenv("TACAW_FAULT", "launch")
    for name, call in _entry_points(lib):
        rc = call()
        assert rc == L.TACAW_ECUDA, (name, rc, lib.tacaw_last_error())
        msg = lib.tacaw_last_error().decode()
        assert name in msg and "injected launch failure" in msg, (name, msg)
        with pytest.raises(L.TacawError) as exc:
            L.check(name, rc)
        assert exc.value.code == L.TACAW_ECUDA


def test_workspace_queries_and_argument_errors_come_first(lib, monkeypatch):
    """The injected fault sits after validation: size queries still answer and
    bad arguments are still reported as such."""
    monkeypatch.setenv("TACAW_FAULT", "launch,symbol")
    g = _grid()
    n = ctypes.c_size_t(0)
    assert lib.tacaw_multislice(ctypes.byref(g), 2, NULL, NULL, NULL, NULL, 0, NULL, ctypes.byref(n), NULL) == 0
    assert n.value > 0
    assert lib.tacaw_multislice(ctypes.byref(g), -1, FAKE, NULL, FAKE, NULL, 0, FAKE, _big(),
                                NULL) == L.TACAW_EINVAL
    assert lib.tacaw_multislice_static(ctypes.byref(g), 2, FAKE, NULL, FAKE, NULL, 4, NULL) == L.TACAW_EINVAL
    assert lib.tacaw_multislice_static(ctypes.byref(g), 0, FAKE, NULL, FAKE, NULL, 0, NULL) == L.TACAW_OK


def test_injected_symbol_lookup_failure(lib, monkeypatch):
    monkeypatch.setenv("TACAW_FAULT", "symbol")
    g = _grid()
    rc = lib.tacaw_multislice_static(ctypes.byref(g), 2, FAKE, NULL, FAKE, NULL, 0, NULL)
    assert rc == L.TACAW_ECUDA
    assert b"injected symbol lookup failure" in lib.tacaw_last_error()
    rc = lib.tacaw_multislice(ctypes.byref(g), 2, FAKE, NULL, FAKE, NULL, 0, FAKE, _big(), NULL)
    assert rc == L.TACAW_ECUDA and b"injected symbol" in lib.tacaw_last_error()
    rc = lib.tacaw_status(NULL)
    assert rc == L.TACAW_ECUDA and b"tacaw_status" in lib.tacaw_last_error()


def test_injected_timeout_is_reported_by_status(lib, monkeypatch):
    monkeypatch.setenv("TACAW_FAULT", "timeout")
    rc = lib.tacaw_status(NULL)
    assert rc == L.TACAW_ETIMEOUT
    assert b"timeout" in lib.tacaw_last_error()
    with pytest.raises(L.TacawError) as exc:
        L.check("tacaw_status", rc)
    assert exc.value.code == L.TACAW_ETIMEOUT and "ETIMEOUT" in str(exc.value)


def test_wait_limit_setter_accepts_any_value(lib):
    for polls in (0, 1, 1 << 40, -5, -1):
        assert lib.tacaw_set_wait_limit(polls) == L.TACAW_OK
    assert lib.tacaw_last_error() == b""


def test_static_scratch_holds_the_largest_grid(lib):
    """tacaw_multislice_static checks its fixed 64 KiB scratch against the
    tables of the grid before the n_t == 0 early return; the largest grid's
    tables are 37120 bytes, as the library states."""
    g = _grid(1024, 1024)
    n = ctypes.c_size_t(0)
    assert lib.tacaw_multislice(ctypes.byref(g), 1, NULL, NULL, NULL, NULL, 0, NULL, ctypes.byref(n), NULL) == 0
    assert n.value == 37120 <= 64 * 1024
    assert lib.tacaw_multislice_static(ctypes.byref(g), 0, NULL, NULL, NULL, NULL, 0, NULL) == L.TACAW_OK
    for nx, ny in ((64, 1024), (768, 384), (1024, 64)):
        g = _grid(nx, ny)
        assert lib.tacaw_multislice(ctypes.byref(g), 1, NULL, NULL, NULL, NULL, 0, NULL, ctypes.byref(n), NULL) == 0
        assert n.value <= 37120
