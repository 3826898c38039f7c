"""Pins of the oracle's full Zeeman pattern (Section 5: the pattern of the
configured line is computed at start-up; Fe I 6301.5, 5P2-5D2, has four
components in each of sigma_b, pi, sigma_r).

Checked against what angular-momentum algebra and the effective-triplet limit
fix: 3j special values, orthogonality and symmetry; each group's strengths sum
to 1; the strength-weighted sigma shifts equal the textbook g_eff; a J=1 -> 0
transition reproduces the effective triplet exactly; in the weak-field limit V
equals the effective triplet's V with g_eff (first moment), to O(B^2).
"""
import math

import numpy as np
import pytest

import genesis_inputs as gi


def test_wigner3j_special_values_and_orthogonality(orc):
    for m in (-1, 0, 1):
        assert orc.wigner3j(1, 1, 0, m, -m, 0) == pytest.approx((-1) ** (1 - m) / math.sqrt(3), abs=1e-15)
    assert orc.wigner3j(2, 2, 1, 0, 0, 0) == 0.0     # j1 + j2 + j3 odd with all m = 0
    assert abs(orc.wigner3j(1, 1, 1, 1, 0, -1)) == pytest.approx(1 / math.sqrt(6), abs=1e-15)
    for j1, j2 in [(1, 1), (2, 1), (2, 2), (3, 2)]:
        for j3 in range(abs(j1 - j2), j1 + j2 + 1):
            for j3b in range(abs(j1 - j2), j1 + j2 + 1):
                for m3 in range(-min(j3, j3b), min(j3, j3b) + 1):
                    s = sum(orc.wigner3j(j1, j2, j3, m1, m2, m3) * orc.wigner3j(j1, j2, j3b, m1, m2, m3)
                            for m1 in range(-j1, j1 + 1) for m2 in range(-j2, j2 + 1))
                    assert s == pytest.approx((j3 == j3b) / (2 * j3 + 1), abs=1e-13)
    # odd column permutation multiplies by (-1)^(j1+j2+j3)
    for args in [(2, 1, 2, 1, -1, 0), (3, 2, 1, -2, 1, 1), (2, 2, 1, 1, -2, 1)]:
        j1, j2, j3, m1, m2, m3 = args
        ph = (-1) ** (j1 + j2 + j3)
        assert orc.wigner3j(j2, j1, j3, m2, m1, m3) == pytest.approx(ph * orc.wigner3j(*args), abs=1e-14)


def _geff(jl, gl, ju, gu):
    return 0.5 * (gu + gl) + 0.25 * (gu - gl) * (ju * (ju + 1) - jl * (jl + 1))


@pytest.mark.parametrize("jl,gl,ju,gu", [(2, 11 / 6, 2, 1.5), (1, 2.5, 0, 0.0), (1, 1.5, 2, 1.5),
                                         (3, 1.25, 2, 1.0), (2, 1.0, 3, 1.25), (4, 1.3, 4, 1.1)])
def test_strength_sum_rules_and_first_moment(orc, jl, gl, ju, gu):
    groups = orc.zeeman_components(jl, gl, ju, gu)
    for sh, st in groups:
        assert np.all(st > 0) and st.sum() == pytest.approx(1.0, abs=1e-13)
    (sb, wb), (sp, wp), (sr, wr) = groups
    g = _geff(jl, gl, ju, gu)
    assert (sb * wb).sum() == pytest.approx(-g, abs=1e-12)
    assert (sr * wr).sum() == pytest.approx(g, abs=1e-12)
    assert (sp * wp).sum() == pytest.approx(0.0, abs=1e-12)
    # mirror symmetry of the pattern
    assert np.allclose(np.sort(-sb), np.sort(sr)) and np.allclose(np.sort(-sp), np.sort(sp))


def test_fe6301_pattern_has_four_components_per_group(orc):
    for sh, st in orc.zeeman_components(2, 11 / 6, 2, 1.5):
        assert len(sh) == 4
    assert _geff(2, 11 / 6, 2, 1.5) == pytest.approx(1.6667, abs=1e-4)   # Table 1


def _spec(lines, grid):
    return gi.ProblemSpec(lines=lines, lambda_grid=grid)


def test_normal_triplet_pattern_equals_effective_triplet(orc):
    l0 = gi.FE6302[0]
    grid = l0 + np.linspace(-0.6, 0.6, 97)
    trip = _spec([(l0, 2.5, 1.0)], grid)
    full = _spec([(l0, 2.5, 1.0, 1, 2.5, 0, 0.0)], grid)
    P = gi.draw_params_uniform(50, seed=60)
    assert np.max(np.abs(orc.synth(full, P) - orc.synth(trip, P))) < 1e-14


def test_full_pattern_weak_field_matches_effective_triplet(orc):
    l0 = gi.FE6301[0]
    grid = l0 + np.linspace(-0.5, 0.5, 161)
    full = _spec([(l0, 1.667, 1.0, 2, 11 / 6, 2, 1.5)], grid)
    trip = _spec([(l0, _geff(2, 11 / 6, 2, 1.5), 1.0)], grid)
    base = np.array([0.0, 35.0, 20.0, 0.3, 30.0, 0.2, 8.0, 0.3, 0.7])
    errs = []
    for B in [4.0, 8.0, 16.0]:
        p = base.copy(); p[0] = B
        vf, vt = orc.synth(full, p)[0, 3], orc.synth(trip, p)[0, 3]
        errs.append(np.max(np.abs(vf - vt)) / np.max(np.abs(vt)))
    assert errs[0] < 1e-3
    assert 2.5 < errs[1] / errs[0] < 5.5 and 2.5 < errs[2] / errs[1] < 5.5, errs   # O(B^2)
    # strong field: the patterns differ visibly
    p = base.copy(); p[0] = 2500.0
    assert np.max(np.abs(orc.synth(full, p) - orc.synth(trip, p))) > 1e-3


def test_full_pattern_symmetries(orc):
    l0 = gi.FE6301[0]
    full = _spec([(l0, 1.667, 1.0, 2, 11 / 6, 2, 1.5)], l0 + np.linspace(-0.6, 0.6, 65))
    P = gi.draw_params_uniform(30, seed=61)
    s = orc.synth(full, P)
    P0 = P.copy(); P0[:, 0] = 0.0
    assert np.max(np.abs(orc.synth(full, P0)[:, 1:])) < 1e-15
    P90 = P.copy(); P90[:, 2] += 90.0
    s90 = orc.synth(full, P90)
    assert np.max(np.abs(s90[:, 1:3] + s[:, 1:3])) < 1e-12
    Pv = P.copy(); Pv[:, 3] = 0.0
    sv = orc.synth(full, Pv)
    assert np.max(np.abs(sv[:, 3] + sv[:, 3, ::-1])) < 1e-13     # V odd about the centre
