"""The device computes a sample's opacity 1 - exp(-x) (x = sigma_max a dt)
with the Taylor series to x^5 for |x| < 1/16 and the library's expm1f above.
This pins the series' coefficients and its error bound: evaluated the way
the device does (Horner with fused multiply-adds, each rounded to float32),
it stays within 4 float32 roundings of the exact value over the whole range,
and its truncation error there is below x^6 / 720."""
import math

import numpy as np


def _fma32(a, b, c):
    """float32 fused multiply-add: the float32 product is exact in float64,
    one rounding of the sum to float32."""
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def _series32(x):
    x = np.float32(x)
    q = _fma32(-x, np.float32(1.0 / 120.0), np.float32(1.0 / 24.0))
    q = _fma32(-x, q, np.float32(1.0 / 6.0))
    q = _fma32(-x, q, np.float32(0.5))
    q = _fma32(-x, q, np.float32(1.0))
    return np.float32(x * q)


def test_series_within_four_roundings():
    xs = np.concatenate([np.linspace(-0.0625, 0.0625, 20001), np.geomspace(1e-12, 0.0625, 2001),
                         -np.geomspace(1e-12, 0.0625, 2001)]).astype(np.float32)
    xs = xs[np.abs(xs) < np.float32(0.0625)]
    exact = -np.expm1(-xs.astype(np.float64))
    got = np.array([_series32(x) for x in xs], dtype=np.float64)
    ulp = np.spacing(np.abs(exact).astype(np.float32)).astype(np.float64)
    err = np.abs(got - exact)[exact != 0] / ulp[exact != 0]
    assert err.max() <= 4.0, err.max()


def test_truncation_bound():
    # the first dropped term is x^6 / 720 (alternating series: it bounds the rest)
    x = 0.0625
    series = sum((-1) ** (k + 1) * x ** k / math.factorial(k) for k in range(1, 6))
    exact = -math.expm1(-x)
    assert abs(series - exact) <= x ** 6 / 720
    assert abs(series - exact) / exact <= 1.4e-9
