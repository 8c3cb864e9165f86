"""Error bound of the small-phase sin/cos series used for the transmission
function exp(i sigma_e v): the truncated Taylor series (sin to x^9, cos to
x^10, Horner's rule in FP32, as in csrc/common.cuh) against numpy's FP64
sin/cos on |x| <= 0.5.  A few FP32 ulps is the bound."""

import numpy as np


def _series(x):
    x = x.astype(np.float32)
    x2 = (x * x).astype(np.float32)
    f = np.float32
    ps = f(1.0 / 362880.0)
    ps = (x2 * ps + f(-1.0 / 5040.0)).astype(np.float32)
    ps = (x2 * ps + f(1.0 / 120.0)).astype(np.float32)
    ps = (x2 * ps + f(-1.0 / 6.0)).astype(np.float32)
    ps = (x2 * ps + f(1.0)).astype(np.float32)
    pc = f(-1.0 / 3628800.0)
    for coef in (1.0 / 40320.0, -1.0 / 720.0, 1.0 / 24.0, -0.5, 1.0):
        pc = (x2 * pc + f(coef)).astype(np.float32)
    return (x * ps).astype(np.float32), pc


def test_small_phase_series_error_bound():
    x = np.linspace(-0.5, 0.5, 200001)
    s, c = _series(x)
    xs = x.astype(np.float32).astype(np.float64)
    ulp = np.spacing(np.float32(1.0))
    assert np.max(np.abs(s - np.sin(xs))) <= 3 * ulp
    assert np.max(np.abs(c - np.cos(xs))) <= 3 * ulp
    # relative accuracy of sin for tiny phases (where the exp is ~ 1 + i x)
    tiny = xs[np.abs(xs) > 1e-6][:1000]
    st, _ = _series(tiny)
    assert np.max(np.abs(st - np.sin(tiny)) / np.abs(np.sin(tiny))) <= 4 * ulp
