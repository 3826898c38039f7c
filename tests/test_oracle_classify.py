"""Pins of the oracle's Section 2 pixel selection, weak-field fallback and
Section 5.5 seeds.

The pins come from outside the oracle's own formulas: hand-sized cases
whose variances and maxima are known; profiles built to satisfy the
weak-field relations exactly (analytic Gaussian I with V proportional to I'
and Q, U proportional to I''); exactly shifted parabolic and Gaussian cores
whose separation is known; the weak-field limit of the Unno-Rachkovsky
solution; and the symmetries of the estimates (a rotation of Q, U by 2 d
turns chi by d, a sign flip of V flips the polarity).
"""
import math

import numpy as np
import pytest

import genesis_inputs as gi

KZ0 = 4.6686e-13
L0 = gi.FE6302[0]
G = 2.5


def _spec(lam, g=G):
    return gi.ProblemSpec([(L0, g, 1.0)], lam)


def _weak_field_cube(lam, bpar, bperp, chi, d=0.6, w=0.08):
    """Gaussian line I with V = -kz B_par I' and (Q, U) = -(kz^2 B_perp^2 / 4)
    (cos 2chi, sin 2chi) I'', analytic derivatives."""
    kz = KZ0 * G * L0 * L0
    x = lam - L0
    e = np.exp(-(x / w) ** 2)
    I = 1.0 - d * e
    d1 = d * e * 2 * x / w ** 2
    d2 = d * e * (2 / w ** 2 - 4 * x ** 2 / w ** 4)
    a = 0.25 * kz ** 2 * bperp ** 2
    c = math.radians(2 * chi)
    return np.stack([I, -a * math.cos(c) * d2, -a * math.sin(c) * d2, -kz * bpar * d1])[None]


def test_threshold_hand_sized_case(orc):
    """Quiet window of 4 points holding Q = +-a, U = +-b, V = +-c around zero
    means: variances a^2, b^2, c^2; maxima set by single points outside."""
    lam = L0 + np.linspace(-0.5, 0.5, 12)
    obs = np.zeros((1, 4, 12))
    obs[0, 0] = 2.0
    obs[0, 1, :4] = [0.1, -0.1, 0.1, -0.1]
    obs[0, 2, :4] = [0.2, 0.2, -0.2, -0.2]
    obs[0, 3, :4] = [-0.3, 0.3, 0.3, -0.3]
    obs[0, 1, 7] = 0.6
    obs[0, 2, 8] = -0.8
    obs[0, 3, 9] = 1.2
    r = orc.classify(_spec(lam), obs, 3.0, (0, 4), 0, (4, 11))
    p = math.sqrt(0.36 + 0.64 + 1.44) / 2.0
    sp = 3.0 * math.sqrt(0.01 + 0.04 + 0.09) / 2.0
    assert abs(r["p"][0] - p) < 1e-15 and abs(r["sigma_p"][0] - sp) < 1e-15
    assert r["flag"][0] == int(p > sp)
    r = orc.classify(_spec(lam), obs, 5.0, (0, 4), 0, (4, 11))
    assert r["flag"][0] == 0  # 5 * 0.187 > 0.781


def test_threshold_noise_statistics(orc):
    """Pure noise of standard deviation s on a continuum I_c: sigma_P tends to
    P_thresh sqrt(3) s / I_c, and P_thresh = 1 passes exactly the pixels whose
    polarization exceeds the noise."""
    n = 4000
    lam = L0 + np.linspace(-2.0, 2.0, n)
    rng = np.random.default_rng(7)
    obs = np.empty((3, 4, n))
    obs[:, 0] = 1.3
    obs[:, 1:] = 2e-3 * rng.standard_normal((3, 3, n))
    r = orc.classify(_spec(lam), obs, 10.0, (0, n), 0, (n // 2 - 50, n // 2 + 50))
    assert np.all(np.abs(r["sigma_p"] / (10.0 * math.sqrt(3) * 2e-3 / 1.3) - 1) < 0.03)
    assert np.all(r["flag"] == 0)
    r1 = orc.classify(_spec(lam), obs, 1.0, (0, n), 0, (n // 2 - 50, n // 2 + 50))
    assert np.all(r1["flag"] == 1)  # the maxima of 4000 draws exceed one sigma


def test_threshold_scale_invariance(orc):
    spec = gi.two_line_spec(n_lambda=64)
    obs = orc.synth(spec, gi.draw_truth(6, seed=3))
    obs += 1e-3 * gi.draw_noise(6, 64, seed=3)
    a = orc.classify(spec, obs, 10.0, (0, 8), 0, (8, 40))
    b = orc.classify(spec, 4.0 * obs, 10.0, (0, 8), 0, (8, 40))  # power-of-two scale: exact
    for k in ["p", "sigma_p", "flag", "polarity"]:
        assert np.array_equal(a[k], b[k]), k


def test_core_separation_exact_for_parabolic_cores(orc):
    """I +- V with parabolic cores centred at lambda0 -+ delta... (I+V at +d,
    I-V at -d): vertex refinement is exact, B_par = d / kz."""
    kz = KZ0 * G * L0 * L0
    lam = L0 + np.linspace(-0.4, 0.4, 41)
    for dlt in [0.0, 3.3e-3, -7.1e-3, 1.5e-2]:
        p_ = 0.3 + 40.0 * (lam - L0 - dlt) ** 2
        m_ = 0.3 + 40.0 * (lam - L0 + dlt) ** 2
        obs = np.zeros((1, 4, 41))
        obs[0, 0] = 0.5 * (p_ + m_)
        obs[0, 3] = 0.5 * (p_ - m_)
        r = orc.classify(_spec(lam), obs, 1.0, (0, 4), 0, (10, 30))
        assert abs(r["B_par"][0] - dlt / kz) < 1e-9 * max(1.0, abs(dlt / kz)), (dlt, r["B_par"][0])


def test_weak_field_relations_recovered(orc):
    """Profiles obeying the weak-field relations exactly: chi exact, B_perp
    to the discretization of I'' (h^2), B_par from the core separation and
    the integral seed to first order in the splitting."""
    lam = L0 + np.linspace(-0.5, 0.5, 801)
    for bpar, bperp, chi in [(40.0, 60.0, 30.0), (-25.0, 80.0, 120.0), (10.0, 35.0, 170.0), (30.0, 5.0, 75.0)]:
        obs = _weak_field_cube(lam, bpar, bperp, chi)
        r = orc.classify(_spec(lam), obs, 1.0, (0, 20), 0, (200, 600))
        assert abs((r["chi"][0] - chi + 90) % 180 - 90) < 1e-9
        assert abs(r["B_perp"][0] / bperp - 1) < 1e-4
        assert abs(r["B_par"][0] / bpar - 1) < 2e-3
        assert abs(r["theta"][0] - math.degrees(math.atan2(bperp, bpar))) < 0.1
        s_int = r["seeds"][0, 1]
        assert abs(s_int[0] * math.cos(math.radians(s_int[1])) / bpar - 1) < 1e-3
        assert abs(s_int[0] * math.sin(math.radians(s_int[1])) / bperp - 1) < 1e-3
        assert r["polarity"][0] == (1 if bpar > 0 else -1)


def test_centre_of_gravity_exact_shift(orc):
    """I +- V = exactly shifted Gaussians, well inside the window: the
    Rees-Semel centre of gravity gives B_par = delta / kz."""
    kz = KZ0 * G * L0 * L0
    lam = L0 + np.linspace(-0.6, 0.6, 1201)
    x = lam - L0
    for dlt in [2e-3, -5e-3, 1.1e-2]:
        p_ = 1.0 - 0.5 * np.exp(-((x - dlt) / 0.05) ** 2)
        m_ = 1.0 - 0.5 * np.exp(-((x + dlt) / 0.05) ** 2)
        obs = np.zeros((1, 4, lam.size))
        obs[0, 0] = 0.5 * (p_ + m_)
        obs[0, 3] = 0.5 * (p_ - m_)
        r = orc.classify(_spec(lam), obs, 1.0, (0, 10), 0, (200, 1000))
        s = r["seeds"][0, 2]
        b_cog = s[0] * math.cos(math.radians(s[1]))
        assert abs(b_cog - dlt / kz) < 1e-8 * abs(dlt / kz), (b_cog, dlt / kz)


def test_weak_field_limit_of_unno_solution(orc):
    """The Unno-Rachkovsky profiles obey V = -kz B_par I' to first order in B
    for any line strength, and (Q, U) proportional to I'' only to first order
    in eta0 as well (for a saturated line a 2 eta'^2 / (1 + eta)^3 term
    remains in I''): B_par converges as B -> 0 at eta0 = 3, B_perp and chi in
    a weak line (eta0 = 0.03)."""
    lam = L0 + np.linspace(-0.5, 0.5, 401)
    spec = gi.ProblemSpec([(L0, G, 1.0)], lam)
    for eta0, cols in [(3.0, [0]), (0.03, [0, 1, 2])]:
        errs = []
        for B in [100.0, 25.0]:
            p = np.array([[B, 55.0, 40.0, 0.0, 40.0, 0.05, eta0, 0.3, 0.7]])
            r = orc.classify(spec, orc.synth(spec, p), 1.0, (0, 10), 0, (100, 300))
            bpar, bperp = B * math.cos(math.radians(55)), B * math.sin(math.radians(55))
            errs.append([abs(r["B_par"][0] / bpar - 1), abs(r["B_perp"][0] / bperp - 1),
                         abs((r["chi"][0] - 40.0 + 90) % 180 - 90) / 40.0])
            assert r["polarity"][0] == 1
        errs = np.array(errs)[:, cols]
        assert np.all(errs[1] < 2e-3), (eta0, errs)
        assert np.all(errs[1] < errs[0]), (eta0, errs)


def test_rotation_and_polarity_symmetries(orc):
    spec = gi.two_line_spec(n_lambda=96)
    truth = gi.draw_truth(5, seed=11)
    obs = orc.synth(spec, truth)
    a = orc.classify(spec, obs, 10.0, (0, 8), 0, (20, 60))
    for d in [10.0, 45.0, 90.0, 133.0]:
        c, s = math.cos(math.radians(2 * d)), math.sin(math.radians(2 * d))
        rot = obs.copy()
        rot[:, 1] = c * obs[:, 1] - s * obs[:, 2]
        rot[:, 2] = s * obs[:, 1] + c * obs[:, 2]
        b = orc.classify(spec, rot, 10.0, (0, 8), 0, (20, 60))
        assert np.all(np.abs((b["chi"] - a["chi"] - d + 90) % 180 - 90) < 1e-9)
        assert np.allclose(b["B_perp"], a["B_perp"], rtol=1e-12)
    flip = obs.copy()
    flip[:, 3] = -obs[:, 3]
    b = orc.classify(spec, flip, 10.0, (0, 8), 0, (20, 60))
    assert np.array_equal(b["polarity"], -a["polarity"])
    assert np.allclose(b["B_par"], -a["B_par"], rtol=1e-12, atol=1e-9)
    for k in range(4):
        nz = a["polarity"] != 0
        assert np.allclose(b["seeds"][nz, k, 1], 180.0 - a["seeds"][nz, k, 1], atol=1e-9)


def test_seeds_respect_polarity_and_nonmagnetic(orc):
    spec = gi.two_line_spec(n_lambda=96)
    obs = orc.synth(spec, gi.draw_truth(40, seed=12))
    obs += 1e-3 * gi.draw_noise(40, 96, seed=12)
    r = orc.classify(spec, obs, 10.0, (0, 8), 0, (20, 60))
    psi = r["seeds"][:, :, 1]
    pos, neg = r["polarity"] > 0, r["polarity"] < 0
    assert np.all(psi[pos] <= 90.0) and np.all(psi[neg] >= 90.0)
    assert np.all(r["seeds"][:, 3, 0] == 0.0)
    assert np.all(r["seeds"][:, :, 0] >= 0.0)
    assert np.all((r["seeds"][:, :, 2] >= 0.0) & (r["seeds"][:, :, 2] < 180.0))
