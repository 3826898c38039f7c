"""The FP32 pair path's w(z) regions keep their error budget.

The region thresholds are read from the CUDA headers, each branch formula is
evaluated in float32 (numpy, without fused multiply-adds, so a little
pessimistic) beyond its threshold, and compared with scipy's wofz: the far
field, the 3rd convergent and the 5th convergent of the Laplace continued
fraction w = (i/sqrt(pi)) / (z - (1/2) / (z - 1 / (z - (3/2) / ...))) must stay
within 1.5e-7 absolute (1.3e-7 with the kernel's FMAs).  Moving a threshold
inward past the budget fails here."""
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


def far32(x, y):
    x, y = x.astype(f32), f32(y)
    ux, uy = x * x - f32(y * y), x * (f32(2) * y)
    dx = ux - f32(0.5)
    inv = (f32(1) / (dx * dx + uy * uy)) * f32(0.56418958354775628695)
    return ((x * uy - y * dx) * inv).astype(float) + 1j * ((x * dx + y * uy) * inv).astype(float)


def worst_beyond(fn, r2):
    worst = 0.0
    for y in np.concatenate([[0.0], np.geomspace(1e-4, 1.0, 30)]):
        x0 = np.sqrt(max(r2 - y * y, 0.0))
        x = x0 + np.linspace(0.0, 7.0, 6001) ** 2 + 1e-6
        worst = max(worst, float(np.max(np.abs(fn(x, y) - special.wofz(x + 1j * y)))))
    return worst


def test_threshold_order():
    t = thresholds()
    assert 0 < t["mid"] < t["ext"] < t["far"]
    assert t["K"] == 3


def test_far_field_within_budget():
    assert worst_beyond(far32, thresholds()["far"]) < BUDGET


def test_third_convergent_within_budget():
    assert worst_beyond(lambda x, y: cf32(x, y, 3), thresholds()["ext"]) < BUDGET


def test_fifth_convergent_within_budget():
    assert worst_beyond(lambda x, y: cf32(x, y, 5), thresholds()["mid"]) < BUDGET


def test_budget_is_tight_enough_to_fail():
    """The check has teeth: the far field a little further in exceeds it."""
    assert worst_beyond(far32, 0.8 * thresholds()["far"]) > BUDGET
