"""ctypes binding of libtacaw.so: argument types of every C-ABI entry point.

The library is loaded from this package directory.  There is no fallback:
if it is missing or fails to load, importing the binding raises, so the
product path can never silently run anything but the CUDA kernels.
"""

from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtacaw.so")

TACAW_OK = 0
TACAW_EINVAL = -1
TACAW_ECUDA = -2
TACAW_ENOMEM = -3
TACAW_ETIMEOUT = -4
TACAW_EUNSUPPORTED = -5
TACAW_FP32 = 0
TACAW_BF16X3 = 1
TACAW_FFT32 = 2
TACAW_BF16X6 = 3
TIME_FFT_SIZES = (64, 128, 256, 384, 512, 768, 1024, 2048, 4096)   # T with a TACAW_FFT32 plan
TACAW_KUBO = 1
TACAW_NORMALIZE = 2
TACAW_MAX_SPECIES = 8
TACAW_MAX_BATCH = 64
TACAW_MS_WARP_ROWS = 1
TACAW_MS_BLOCK_COLS = 2
TACAW_MS_QUEUE = 4

ERRORS = {
    TACAW_EINVAL: "EINVAL", TACAW_ECUDA: "ECUDA", TACAW_ENOMEM: "ENOMEM",
    TACAW_ETIMEOUT: "ETIMEOUT", TACAW_EUNSUPPORTED: "EUNSUPPORTED",
}


class TacawGrid(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double),
        ("n_slices", ctypes.c_int32),
        ("dz", ctypes.c_double), ("z0", ctypes.c_double),
        ("kev", ctypes.c_double), ("bandlimit", ctypes.c_double),
    ]


class TacawJob(ctypes.Structure):
    _fields_ = [
        ("grid", TacawGrid), ("n_t", ctypes.c_int32),
        ("V", ctypes.c_void_p), ("psi_in", ctypes.c_void_p),
        ("psi_q", ctypes.c_void_p), ("psi_sum", ctypes.c_void_p),
    ]


class TacawError(RuntimeError):
    def __init__(self, fn, code, msg):
        super().__init__(f"{fn} failed with {ERRORS.get(code, code)}: {msg}")
        self.code = code


_P = ctypes.c_void_p
_SZ = ctypes.POINTER(ctypes.c_size_t)
SIGNATURES = {
    "tacaw_last_error": (ctypes.c_char_p, []),
    "tacaw_version": (ctypes.c_int32, []),
    "tacaw_status": (ctypes.c_int, [_P]),
    "tacaw_set_wait_limit": (ctypes.c_int, [ctypes.c_int64]),
    "tacaw_beam_constants": (ctypes.c_int, [ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                            ctypes.POINTER(ctypes.c_double)]),
    "tacaw_potential": (ctypes.c_int, [ctypes.POINTER(TacawGrid), ctypes.c_int32, ctypes.c_int32, _P, _P,
                                       ctypes.c_int32, ctypes.POINTER(ctypes.c_float), _P, _P, _SZ, _P]),
    "tacaw_multislice": (ctypes.c_int, [ctypes.POINTER(TacawGrid), ctypes.c_int32, _P, _P, _P, _P,
                                        ctypes.c_int32, _P, _SZ, _P]),
    "tacaw_multislice_static": (ctypes.c_int, [ctypes.POINTER(TacawGrid), ctypes.c_int32, _P, _P, _P, _P,
                                               ctypes.c_int32, _P]),
    "tacaw_multislice_batch": (ctypes.c_int, [ctypes.POINTER(TacawJob), ctypes.c_int32, _P, _SZ, _P]),
    "tacaw_multislice_queue": (ctypes.c_int, [ctypes.POINTER(TacawJob), ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int32, _P, _SZ, _P]),
    "tacaw_spectrum": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_int32, _P,
                                      _P, _P, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                      _P, _SZ, _P]),
    "tacaw_spectrum_segments": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                               ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P,
                                               ctypes.c_int32, ctypes.c_int32, ctypes.c_double, _P, _SZ, _P]),
    "tacaw_qep_intensity": (ctypes.c_int, [ctypes.c_int32] * 5 + [_P, _P, _P]),
    "tacaw_time_mean": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _P, _P, _P]),
    "tacaw_time_to_spectrum_host": (ctypes.c_int, [ctypes.POINTER(TacawGrid), ctypes.c_int32, ctypes.c_int32, _P, _P,
                                                   ctypes.c_int32, ctypes.POINTER(ctypes.c_float), ctypes.c_double,
                                                   ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                   ctypes.c_double, _P, _P, _P, _SZ, _P]),
    "tacaw_spectrum_accumulate": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                                 ctypes.c_int32, _P, _P, _P, _P, ctypes.c_int32, _P, _SZ, _P]),
    "tacaw_spectrum_finish": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_int32, _P,
                                             _P, _P, _P, _P, _P, ctypes.c_int32, ctypes.c_double, _P, _SZ, _P]),
    "tacaw_energy_integral": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P]),
    "tacaw_line_profile": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                          _P, _P, _P, _P]),
    "tacaw_azimuthal_profile": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_int32, _P, _P, _P, _P,
                                               _SZ, _P]),
    "tacaw_relative_difference": (ctypes.c_int, [ctypes.c_int64, _P, _P, _P, _P]),
    "tacaw_probe": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32] + [ctypes.c_double] * 7 + [_P, _P, _SZ, _P]),
    "tacaw_tune_multislice": (ctypes.c_int, [ctypes.POINTER(TacawGrid), ctypes.c_int32, _P, _P, _P, ctypes.c_int32,
                                             ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _SZ, _P]),
    "tacaw_spectrum_backward": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                               ctypes.c_int32, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "tacaw_multislice_backward": (ctypes.c_int, [ctypes.POINTER(TacawGrid), ctypes.c_int32, _P, _P, _P, _P,
                                                 ctypes.c_int32, _P, _SZ, _P]),
    "tacaw_potential_backward": (ctypes.c_int, [ctypes.POINTER(TacawGrid), ctypes.c_int32, ctypes.c_int32, _P, _P,
                                                ctypes.c_int32, ctypes.POINTER(ctypes.c_float), _P, _P, _P, _SZ,
                                                _P]),
}

_lib = None


def load() -> ctypes.CDLL:
    """Load libtacaw.so once (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libtacaw.so is not built ({LIB_PATH}); run "
                               "`python -m paper_2401_15599_gb300.build` first")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(fn_name: str, code: int) -> None:
    if code != TACAW_OK:
        msg = load().tacaw_last_error().decode(errors="replace")
        raise TacawError(fn_name, code, msg)


def make_grid(g) -> TacawGrid:
    return TacawGrid(int(g.nx), int(g.ny), float(g.lx), float(g.ly), int(g.n_slices),
                     float(g.dz), float(g.z0), float(g.kev), float(g.bandlimit))
