"""The polynomial constants the bins use (paper_2108_11560_gb300/csrc/kv_bins.cuh), read from the
source and checked against the functions they stand for in 30-digit arithmetic, with the
coefficients rounded as the kernels hold them (float for the FP32 bins, double for the FP64 bins):

  phi(s) = e^s - 1 - s = z (E(z) + s O(z)), z = s^2, |s| <= 1   (the x-part of the bins' exponent)
  tanh(y) = y + y^3 P(y^2), |y| < 0.35                           (the d/dv integrand near vt = 0)
  expm1(y) = y + y^2 (1/2 + y/6 + ... + y^6/8!), |y| < 1/2        (e^{-2vt} - e^{-2u} near the peak)

Each must be below half an ulp of the result's precision, so that the polynomial's error does not
show next to the rounding of the arithmetic itself."""
import os
import re

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")
mp.mp.dps = 30

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2108_11560_gb300", "csrc", "kv_bins.cuh")
NUM = r"-?\d+\.\d+(?:e-?\d+)?"


def _text():
    with open(SRC) as f:
        return f.read()


def _macro(name):
    t = _text()
    i = t.index("#define " + name)
    return t[i:t.index("\n\n", i)]


def _function(signature):
    t = _text()
    i = t.index(signature)
    return t[i:t.index("\n}", i)]


def _horner(coeffs_high_first, z):
    p = mp.mpf(0)
    for c in coeffs_high_first:
        p = p * z + c
    return p


def _fp32_phi_coeffs():
    nums = [float(x) for x in re.findall(r"(" + NUM + r")f", _macro("KV_PHI_SERIES"))]
    assert len(nums) == 8
    e = [mp.mpf(float(np.float32(c))) for c in nums[:4]]   # E: c3, c2, c1, c0
    o = [mp.mpf(float(np.float32(c))) for c in nums[4:]]   # O: c3, c2, c1, c0
    return e, o


def _fp64_phi_coeffs():
    body = _function("void phi_parts_f64(")
    nums = [float(x) for x in re.findall(r"(?<![\w.])(" + NUM + r")(?![\w.])", body)]
    assert len(nums) == 14
    return [mp.mpf(c) for c in nums[:7]], [mp.mpf(c) for c in nums[7:]]


def _phi(s):
    return mp.expm1(s) - s


def _grid(lo, hi, n=801):
    return [mp.mpf(lo) + (mp.mpf(hi) - mp.mpf(lo)) * k / (n - 1) for k in range(n)]


@pytest.mark.parametrize("kind", ["fp32", "fp64"])
def test_phi_polynomials(kind):
    e, o = _fp32_phi_coeffs() if kind == "fp32" else _fp64_phi_coeffs()
    half_ulp = mp.mpf(2) ** (-24 if kind == "fp32" else -53)
    worst = mp.mpf(0)
    for s in _grid(-1, 1):
        if s == 0:
            continue
        z = s * s
        approx = z * (_horner(e, z) + s * _horner(o, z))
        worst = max(worst, abs(approx - _phi(s)) / _phi(s))
    assert worst < half_ulp, (kind, worst)


def test_phi_polynomials_are_not_taylor_truncations():
    """The FP32 polynomials are the minimax fits: the degree-3 Taylor polynomials of E and O
    would leave errors above FP32 rounding at |s| = 1 (a plausible regression to the textbook
    coefficients fails the bound above)."""
    e_taylor = [mp.mpf(1) / mp.factorial(8), mp.mpf(1) / mp.factorial(6), mp.mpf(1) / 24, mp.mpf(1) / 2]
    z = mp.mpf(1)
    assert abs(_horner(e_taylor, z) - (mp.cosh(1) - 1)) > mp.mpf(2) ** -24


def test_tanh_polynomial():
    nums = [float(x) for x in re.findall(r"(" + NUM + r")f", _macro("KV_TANH_POLY"))]
    assert len(nums) == 4
    p = [mp.mpf(float(np.float32(c))) for c in nums]
    worst = mp.mpf(0)
    for y in _grid(0, "0.35"):
        if y == 0:
            continue
        approx = y + y ** 3 * _horner(p, y * y)
        worst = max(worst, abs(approx - mp.tanh(y)) / mp.tanh(y))
    assert worst < mp.mpf(2) ** -24, worst
    # the threshold the bins use for switching to the quotient form
    assert re.search(r"TANH_SERIES_MAX = 0\.35f", _text())


def test_expm1_polynomial():
    body = _function("float2 expm1_small2(")
    den = [int(d) for d in re.findall(r"1\.0f / (\d+)\.0f", body)]
    assert den == [40320, 5040, 720, 120, 24, 6] and "f2(0.5f)" in body
    coeffs = [mp.mpf(float(np.float32(1.0 / d))) for d in den] + [mp.mpf(0.5)]
    worst = mp.mpf(0)
    for y in _grid("-0.5", "0.5"):
        if y == 0:
            continue
        approx = y + y * y * _horner(coeffs, y)
        worst = max(worst, abs(approx - mp.expm1(y)) / abs(mp.expm1(y)))
    assert worst < mp.mpf(2) ** -24, worst
