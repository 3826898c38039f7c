"""The small-splitting series of the FP32 Jacobian, checked as mathematics.

Near a line core the Jacobian forms the sigma-minus-pi combinations of a
weakly split effective triplet from Taylor series in the splitting d about the
pi point z = v + i a:

    h  = (w(z+d) + w(z-d)) / 2 - w(z)      = sum_k d^2k / (2k)! w^(2k)(z)
    hp = (w'(z+d) + w'(z-d)) / 2 - w'(z)   = sum_k d^2k / (2k)! w^(2k+1)(z)
    g1 = (w'(z+d) - w'(z-d)) / 2           = sum_k d^(2k-1) / (2k-1)! w^(2k)(z)

for k = 1..5, with the derivatives of w from w' = -2 z w + 2i/sqrt(pi) and
w^(n+1) = -2 z w^(n) - 2 n w^(n-1).  The same recurrence and coefficient
updates, restated here in double precision, must reproduce the differences
taken at 30 digits (mpmath) in the region where the kernel uses them
(|d| <= 0.25 with |z|^2 <= 16, |d| <= 0.1 with |z|^2 <= 36), to 1e-8 of each
sum: a wrong sign, index or coefficient in the recurrence fails by orders of
magnitude."""
import numpy as np
import pytest

mp = pytest.importorskip("mpmath")
mp.mp.dps = 30


def _w(z):
    return mp.exp(-z * z) * mp.erfc(-1j * z)


def _wp(z):
    return -2 * z * _w(z) + 2j / mp.sqrt(mp.pi)


def series(v, a, d):
    z = complex(v, a)
    wm = complex(_w(mp.mpc(v, a)))
    wc = -2 * z * wm + 2j / np.sqrt(np.pi)
    c, h, hp, g1 = d, 0j, 0j, 0j
    for n in range(1, 11):
        wn = -2 * z * wc - 2 * n * wm          # w^(n+1)
        cn = c * d / (n + 1)                   # d^(n+1) / (n+1)!
        if (n + 1) % 2 == 0:
            h += cn * wn
            g1 += c * wn
        else:
            hp += c * wn
        wm, wc, c = wc, wn, cn
    return h, hp, g1


def _cases():
    rng = np.random.default_rng(7)
    out = []
    while len(out) < 120:
        v, a = rng.uniform(-6, 6), rng.uniform(0, 0.5)
        r2 = v * v + a * a
        dmax = 0.25 if r2 <= 16 else (0.1 if r2 <= 36 else 0.0)
        if dmax == 0.0:
            continue
        d = rng.choice([-1.0, 1.0]) * rng.uniform(1e-3, dmax)
        out.append((v, a, d))
    return out


def test_series_equals_the_differences():
    worst = 0.0
    for v, a, d in _cases():
        h, hp, g1 = series(v, a, d)
        W = lambda x: _w(mp.mpc(x, a))  # noqa: E731
        Wp = lambda x: _wp(mp.mpc(x, a))  # noqa: E731
        ref = [complex((W(v + d) + W(v - d)) / 2 - W(v)),
               complex((Wp(v + d) + Wp(v - d)) / 2 - Wp(v)),
               complex((Wp(v + d) - Wp(v - d)) / 2)]
        for got, want in zip((h, hp, g1), ref):
            worst = max(worst, abs(got - want) / abs(want))
    assert worst < 1e-8, worst


def test_series_has_teeth():
    """A recurrence with the wrong index (2 (n + 1) w^(n-1)) is far off."""
    v, a, d = 1.3, 0.2, 0.2
    z = complex(v, a)
    wm = complex(_w(mp.mpc(v, a)))
    wc = -2 * z * wm + 2j / np.sqrt(np.pi)
    c, h = d, 0j
    for n in range(1, 11):
        wn = -2 * z * wc - 2 * (n + 1) * wm
        cn = c * d / (n + 1)
        if (n + 1) % 2 == 0:
            h += cn * wn
        wm, wc, c = wc, wn, cn
    want = complex((_w(mp.mpc(v + d, a)) + _w(mp.mpc(v - d, a))) / 2 - _w(mp.mpc(v, a)))
    assert abs(h - want) / abs(want) > 1e-2
