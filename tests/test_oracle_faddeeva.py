"""Pins of the oracle's Faddeeva function w(z) = H + i F (Section 5 profiles).

The oracle evaluates w by the Matta-Reichel trapezoid; these tests pin it to
things it does not compute that way: brute-force quadrature of the Voigt and
Faraday-Voigt integrals, the damping-free closed forms, the asymptotic series,
the derivative identity, and scipy's independent implementation.
"""
import math

import numpy as np
import pytest
from scipy import integrate, special


def _quad_HF(a, v):
    """H = (a/pi) Int e^-t^2 / ((v-t)^2 + a^2) dt, F = (1/pi) Int (v-t) e^-t^2 / (...) dt."""
    def fh(t):
        return math.exp(-t * t) / ((v - t) ** 2 + a * a)

    def ff(t):
        return (v - t) * math.exp(-t * t) / ((v - t) ** 2 + a * a)

    pts = sorted(set([max(-12.0, min(12.0, v)), -12.0, 12.0]))
    H = F = 0.0
    for lo, hi in zip(pts[:-1], pts[1:]):
        if hi > lo:
            H += integrate.quad(fh, lo, hi, epsabs=1e-16, epsrel=1e-13, limit=400)[0]
            F += integrate.quad(ff, lo, hi, epsabs=1e-16, epsrel=1e-13, limit=400)[0]
    return a / math.pi * H, F / math.pi


@pytest.mark.parametrize("a", [0.02, 0.1, 0.5, 1.5])
def test_quadrature(orc, a):
    for v in [-9.0, -3.2, -1.0, -0.3, 0.0, 0.7, 2.5, 5.0, 15.0]:
        H, F = _quad_HF(a, v)
        w = orc.faddeeva(v, a)
        assert abs(w.real - H) < 1e-12 * max(1.0, abs(H)), (a, v, w, H)
        assert abs(w.imag - F) < 1e-12 * max(1.0, abs(F)), (a, v, w, F)


def test_damping_free_limit(orc):
    v = np.linspace(-30, 30, 6001)
    w = orc.faddeeva(v, np.zeros_like(v))
    assert np.max(np.abs(w.real - np.exp(-v * v))) < 1e-14
    daw = 2.0 / math.sqrt(math.pi) * special.dawsn(v)
    assert np.max(np.abs(w.imag - daw)) < 2e-14


def test_origin_and_asymptote(orc):
    assert abs(orc.faddeeva(0.0, 0.0) - 1.0) < 1e-15
    for z in [1e3 + 0.1j, -800 + 2j, 300 + 0.0j, 50 + 40j]:
        w = orc.faddeeva(z.real, z.imag)
        # w ~ (i / (sqrt(pi) z)) (1 + 1/(2 z^2) + 3/(4 z^4) + 15/(8 z^6))
        s = 1 + 1 / (2 * z * z) + 3 / (4 * z ** 4) + 15 / (8 * z ** 6)
        asym = 1j / (math.sqrt(math.pi) * z) * s
        assert abs(w - asym) < 1e-11 * abs(asym), z


def test_derivative_identity(orc):
    # w'(z) = -2 z w(z) + 2 i / sqrt(pi)
    h = 1e-5
    for x in [-4.0, -1.3, 0.2, 0.9, 3.3, 8.0]:
        for y in [0.0, 0.05, 0.4]:
            d = (orc.faddeeva(x + h, y) - orc.faddeeva(x - h, y)) / (2 * h)
            z = x + 1j * y
            rhs = -2 * z * orc.faddeeva(x, y) + 2j / math.sqrt(math.pi)
            assert abs(d - rhs) < 1e-8, (x, y)


def test_against_scipy(orc):
    x = np.linspace(-150, 150, 30001)
    for y in [0.0, 1e-8, 1e-3, 0.05, 0.25, 0.5, 1.0, 3.0, 7.0, 20.0]:
        w = orc.faddeeva(x, np.full_like(x, y))
        ref = special.wofz(x + 1j * y)
        assert np.max(np.abs(w - ref)) < 5e-15, y


def test_lower_half_plane_reflection(orc):
    x = np.linspace(-6, 6, 121)
    for y in [-0.01, -0.2, -1.0]:
        w = orc.faddeeva(x, np.full_like(x, y))
        ref = special.wofz(x + 1j * y)
        assert np.max(np.abs(w - ref) / np.abs(ref)) < 1e-13
