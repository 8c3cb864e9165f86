"""Error bound of the small-phase sin/cos series used for the transmission
function exp(i sigma_e v): the truncated Taylor series (|x| <= 0.25: sin to
x^7, cos to x^8; |x| <= 0.5: sin to x^9, cos to x^10; Horner's rule in FP32,
as in csrc/common.cuh) against numpy's FP64 sin/cos.  A few FP32 ulps is the
bound."""

import numpy as np

F = np.float32


def _horner(x2, coefs):
    acc = F(coefs[0])
    for coef in coefs[1:]:
        acc = (x2 * acc + F(coef)).astype(np.float32)
    return acc


def _series(x):
    """|x| <= 0.5: sin to x^9, cos to x^10."""
    x = x.astype(np.float32)
    x2 = (x * x).astype(np.float32)
    ps = _horner(x2, (1.0 / 362880.0, -1.0 / 5040.0, 1.0 / 120.0, -1.0 / 6.0, 1.0))
    pc = _horner(x2, (-1.0 / 3628800.0, 1.0 / 40320.0, -1.0 / 720.0, 1.0 / 24.0, -0.5, 1.0))
    return (x * ps).astype(np.float32), pc


def _series_small(x):
    """|x| <= 0.25: sin to x^7, cos to x^8."""
    x = x.astype(np.float32)
    x2 = (x * x).astype(np.float32)
    ps = _horner(x2, (-1.0 / 5040.0, 1.0 / 120.0, -1.0 / 6.0, 1.0))
    pc = _horner(x2, (1.0 / 40320.0, -1.0 / 720.0, 1.0 / 24.0, -0.5, 1.0))
    return (x * ps).astype(np.float32), pc


def _check(series, lim):
    x = np.linspace(-lim, lim, 200001)
    s, c = series(x)
    xs = x.astype(np.float32).astype(np.float64)
    ulp = np.spacing(np.float32(1.0))
    assert np.max(np.abs(s - np.sin(xs))) <= 3 * ulp
    assert np.max(np.abs(c - np.cos(xs))) <= 3 * ulp
    # relative accuracy of sin for tiny phases (where the exp is ~ 1 + i x)
    tiny = xs[np.abs(xs) > 1e-6][:1000]
    st, _ = series(tiny)
    assert np.max(np.abs(st - np.sin(tiny)) / np.abs(np.sin(tiny))) <= 4 * ulp


def test_small_phase_series_error_bound():
    _check(_series, 0.5)


def test_smaller_phase_series_error_bound():
    _check(_series_small, 0.25)


def test_truncation_below_fp32_rounding():
    # the first dropped term of each series at the edge of its range
    assert 0.25 ** 9 / 362880.0 < 2e-11 and 0.25 ** 10 / 3628800.0 < 2e-11
    assert 0.5 ** 11 / 39916800.0 < 2e-11 and 0.5 ** 12 / 479001600.0 < 2e-11
