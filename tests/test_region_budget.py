"""The FP32 pair path's w(z) regions keep their error budget.

The region thresholds are read from the CUDA headers, each branch formula is
evaluated in float32 (numpy; the far field, the even (three-node) convergent
of the outer shell and the 3rd convergent in the pair path's s-forms with its
fused multiply-adds kept, the others without them, which is a little
pessimistic) beyond its threshold, and compared with scipy's wofz: those three
and the 5th convergent of the Laplace continued fraction
w = (i/sqrt(pi)) / (z - (1/2) / (z - 1 / (z - (3/2) / ...))) must stay within
1.5e-7 absolute (1.3e-7 with the kernel's FMAs).  Moving a threshold
inward past the budget fails here.  Weideman's series, the branch a mixed
warp may take anywhere, is checked the same way in the pair path's
algebraic form (coefficients from their defining integral, N and L read
from the host code)."""
import os
import re

import numpy as np
import pytest

special = pytest.importorskip("scipy.special")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1208_0302_gb300", "csrc")
BUDGET = 1.5e-7
f32 = np.float32


def _constant(path, pattern):
    with open(os.path.join(CSRC, path)) as fh:
        m = re.search(pattern, fh.read())
    assert m, pattern
    return float(m.group(1))


def thresholds():
    return {"far": _constant("me_pair.cuh", r"constexpr float kFarR2 = ([0-9.]+)f;"),
            "even2": _constant("me_pair.cuh", r"constexpr float kEven2R2 = ([0-9.]+)f;"),
            "mid": _constant("me_pair.cuh", r"constexpr float kMidR2 = ([0-9.]+)f;"),
            "ext": _constant("me_device.cuh", r"static constexpr float R2 = ([0-9.]+)f;"),
            "K": _constant("me_device.cuh", r"static constexpr int K = ([0-9]+);")}


def convergent_polys(k):
    """The k-th convergent (odd k) as w = (i/sqrt(pi)) z b(u) / a(u), u = z^2:
    coefficients of a and b (monic) in ascending powers of u."""
    num, den = np.zeros(k + 3), np.zeros(k + 3)   # t = num / den, t_k = z
    num[1], den[0] = 1.0, 1.0
    for m in range(k, 0, -1):                      # t <- z - (m/2) / t
        nn = np.zeros(k + 3)
        nn[1:] += num[:-1]
        nn -= 0.5 * m * den
        num, den = nn, num
    return num[0::2][: (k + 1) // 2 + 1], den[1::2][: (k - 1) // 2 + 1]


def cf32(x, y, k):
    a, b = convergent_polys(k)
    x, y = x.astype(f32), f32(y)
    ux, uy = x * x - f32(y * y), x * (f32(2) * y)
    ax, ay = ux + f32(a[-2]), uy
    for c in a[-3::-1]:
        ax, ay = ax * ux - ay * uy + f32(c), ax * uy + ay * ux
    bx, by = ux + f32(b[-2]), uy
    for c in b[-3::-1]:
        bx, by = bx * ux - by * uy + f32(c), bx * uy + by * ux
    nx, ny = x * bx - y * by, x * by + y * bx
    inv = (f32(1) / (ax * ax + ay * ay)) * f32(0.56418958354775628695)
    return ((nx * ay - ny * ax) * inv).astype(float) + 1j * ((nx * ax + ny * ay) * inv).astype(float)


def fma32(a, b, c):
    """A float32 fused multiply-add: the float64 product of two float32 values
    is exact, so one rounding of the float64 sum stands for the kernel's."""
    return (np.float64(a) * np.float64(b) + np.float64(c)).astype(f32)


def far32(x, y):
    """The far-field approximant (i/sqrt(pi)) z / (z^2 - 1/2) in float32, in the
    pair path's algebraic form (FMAs kept): y (s + 1/2) + i x (s - 1/2) over
    (s - 1/2)^2 + 2 y^2, s = x^2 + y^2, all in u = s - 1/2."""
    x, y = x.astype(f32), f32(y)
    a2 = f32(y * y)
    u = fma32(x, x, a2 - f32(0.5))
    qi = f32(0.56418958354775628695) * (f32(1) / fma32(u, u, f32(2) * a2))
    return (qi * fma32(y, u, y)).astype(float) + 1j * (qi * (x * u)).astype(float)


def even2_32(x, y):
    """The outer shell's even convergent (i/sqrt(pi)) (z^2 - 1) / (z (z^2 - 3/2))
    in float32, in the pair path's algebraic form (FMAs kept): y P + i x (P - s)
    over s (m^2 + 6 y^2), P = m s + 4 y^2 + 1.5, m = s - 3/2."""
    x, y = x.astype(f32), f32(y)
    a2 = f32(y * y)
    s = fma32(x, x, a2)
    m = fma32(x, x, a2 - f32(1.5))
    pr = fma32(m, s, f32(4) * a2 + f32(1.5))
    u = fma32(m, m, f32(6) * a2)
    qi = f32(0.56418958354775628695) * (f32(1) / (s * u))
    return (qi * (y * pr)).astype(float) + 1j * (qi * (x * (pr - s))).astype(float)


def cf3_s32(x, y):
    """The 3rd convergent (i/sqrt(pi)) z (z^2 - 5/2) / (z^4 - 3 z^2 + 3/4) in
    float32 in the pair path's s-form (s = x^2 + y^2, the kernel's FMAs kept):
    y (s^3 - 4.5 s^2 + c1 s + c0) + i x (s^3 - 5.5 s^2 + (c1 + 3) s - c0) over
    s^4 - 6 s^3 + d2 s^2 + (6 - d2) s + d0."""
    x, y = x.astype(f32), f32(y)
    a2 = f32(y * y)
    c1, c0 = fma32(10.0, a2, 5.25), fma32(3.0, a2, 1.875)
    d2, d0 = fma32(12.0, a2, 10.5), fma32(fma32(12.0, a2, 9.0), a2, 0.5625)
    s = fma32(x, x, a2)
    pr = fma32(fma32(s, s + f32(-4.5), c1), s, c0)
    pi = fma32(fma32(s, s + f32(-5.5), c1 + f32(3)), s, -c0)
    den = fma32(fma32(fma32(s + f32(-6), s, d2), s, f32(6) - d2), s, d0)
    qi = f32(0.56418958354775628695) * (f32(1) / den)
    return (qi * (y * pr)).astype(float) + 1j * (qi * (x * pi)).astype(float)


def worst_beyond(fn, r2):
    worst = 0.0
    for y in np.concatenate([[0.0], np.geomspace(1e-4, 1.0, 30)]):
        x0 = np.sqrt(max(r2 - y * y, 0.0))
        x = x0 + np.linspace(0.0, 7.0, 6001) ** 2 + 1e-6
        worst = max(worst, float(np.max(np.abs(fn(x, y) - special.wofz(x + 1j * y)))))
    return worst


def test_threshold_order():
    t = thresholds()
    assert 0 < t["mid"] < t["ext"] < t["even2"] < t["far"]
    assert t["K"] == 3


def test_even_convergent_within_budget():
    assert worst_beyond(even2_32, thresholds()["even2"]) < BUDGET


def test_even_convergent_budget_has_teeth():
    """Moved a little inward, the outer shell's formula exceeds the budget."""
    assert worst_beyond(even2_32, 0.8 * thresholds()["even2"]) > BUDGET


def test_far_field_within_budget():
    assert worst_beyond(far32, thresholds()["far"]) < BUDGET


def test_third_convergent_within_budget():
    assert worst_beyond(cf3_s32, thresholds()["ext"]) < BUDGET


def test_third_convergent_s_form_is_the_convergent():
    """The s-form is the same rational function as the complex polynomials of
    the continued fraction (checked in float64, away from rounding)."""
    x = np.linspace(0.0, 40.0, 401)
    for y in (0.0, 0.05, 0.7):
        z = x + 1j * y
        ref = 1j / np.sqrt(np.pi) * z * (z * z - 2.5) / (z ** 4 - 3 * z * z + 0.75)
        a, b = convergent_polys(3)
        u = z * z
        poly = 1j / np.sqrt(np.pi) * z * np.polyval(b[::-1], u) / np.polyval(a[::-1], u)
        assert np.allclose(ref, poly, rtol=1e-13, atol=0)
        s = x * x + y * y
        c1, c0, d2, d0 = 5.25 + 10 * y * y, 1.875 + 3 * y * y, 10.5 + 12 * y * y, 12 * y ** 4 + 9 * y * y + 0.5625
        w = (y * (s ** 3 - 4.5 * s * s + c1 * s + c0) + 1j * x * (s ** 3 - 5.5 * s * s + (c1 + 3) * s - c0)) \
            / (s ** 4 - 6 * s ** 3 + d2 * s * s + (6 - d2) * s + d0) / np.sqrt(np.pi)
        assert np.allclose(w, ref, rtol=1e-12, atol=1e-300)


def test_third_convergent_budget_has_teeth():
    """Moved a little inward, the 3rd convergent exceeds the budget."""
    assert worst_beyond(cf3_s32, 0.9 * thresholds()["ext"]) > BUDGET


def test_fifth_convergent_within_budget():
    assert worst_beyond(lambda x, y: cf32(x, y, 5), thresholds()["mid"]) < BUDGET


def test_budget_is_tight_enough_to_fail():
    """The check has teeth: the far field a little further in exceeds it."""
    assert worst_beyond(far32, 0.8 * thresholds()["far"]) > BUDGET


def _weideman_setup():
    with open(os.path.join(CSRC, "api.cu")) as fh:
        src = fh.read()
    m = re.search(r"const double L = ([0-9.]+);\s*const std::vector<double> a = weideman_coefficients\((\d+), L\);", src)
    assert m, "FP32 Weideman parameters"
    L, n = float(m.group(1)), int(m.group(2))
    # a_k = (1/K) sum over the midpoint rule of exp(-t^2) (L^2 + t^2) cos(k theta), t = L tan(theta/2)
    kk = 8192
    th = -np.pi + 2 * np.pi * (np.arange(kk) + 0.5) / kk
    t = L * np.tan(0.5 * th)
    g = np.exp(-t * t) * (L * L + t * t)
    a = np.array([np.mean(g * np.cos(k * th)) for k in range(n + 1)])
    return L, n, a


def weideman32(x, y, L, n, a):
    """The pair path's interior branch in float32: Z = ((L^2 - y^2 - x^2) + 2iLx)
    / ((L+y)^2 + x^2), p(Z) by real-quadratic synthetic division with the
    doubled coefficients, w = (p r + 1/sqrt(pi)) r, r = 1/(L - iz) (the
    kernel's FMAs kept)."""
    x, y = x.astype(f32), f32(y)
    Lf = f32(L)
    dx = Lf + y
    inv = f32(1) / fma32(x, x, dx * dx)
    rx, ry = dx * inv, x * inv
    zx = fma32(-x, x, (Lf - y) * dx) * inv
    zy = ry * (f32(2) * Lf)
    w = [f32(2 * c) for c in a]
    r, sq = zx + zx, -fma32(zx, zx, zy * zy)
    b2 = np.full_like(x, w[n])
    b1 = fma32(r, b2, w[n - 1])
    for j in range(n - 3, 0, -1):
        b2, b1 = b1, fma32(r, b1, fma32(sq, b2, w[j + 1]))
    px, py = fma32(sq, b2, fma32(b1, zx, w[1])), b1 * zy
    ux = fma32(px, rx, fma32(-py, ry, f32(0.56418958354775628695)))
    uy = fma32(px, ry, py * rx)
    wx = fma32(ux, rx, -(uy * ry))
    wy = fma32(ux, ry, uy * rx)
    return wx.astype(float) + 1j * wy.astype(float)


def test_weideman_series_fp32():
    """Everywhere (the branch a mixed warp may take): within the FP32 floor at
    the line centre, where |w| is about 1, and at truncation level beyond."""
    L, n, a = _weideman_setup()
    xs = np.concatenate([np.linspace(0.0, 6.0, 3001), np.geomspace(6.0, 1e4, 2000)])
    near, far = 0.0, 0.0
    for y in np.concatenate([[0.0], np.geomspace(1e-4, 1.0, 25)]):
        e = np.abs(weideman32(xs, y, L, n, a) - special.wofz(xs + 1j * y))
        near = max(near, float(np.max(e[xs < 6.0])))
        far = max(far, float(np.max(e[xs >= 6.0])))
    assert near < 1.0e-6 and far < 5.0e-8, (near, far)
