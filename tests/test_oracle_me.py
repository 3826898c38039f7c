"""Pins of the oracle's Unno-Rachkovsky synthesis, weights and chi2 (Section 5).

Each check is something the physics or mathematics fixes independently of how
the oracle computes the Stokes vector: the direct 4x4 solve, the symmetries of
the Zeeman pattern, the field-free and weak-field limits, continuum values and
the chi-square distribution at truth.
"""
import math

import numpy as np
import pytest

import genesis_inputs as gi


def _ic(p, mu=1.0):
    return p[7] + mu * p[8]


@pytest.mark.parametrize("two", [False, True])
def test_closed_form_matches_direct_solve(orc, two):
    spec = gi.two_line_spec() if two else gi.one_line_spec()
    P = gi.draw_params_uniform(200, seed=11 + two)
    s = orc.synth(spec, P)
    for i in range(len(P)):
        slu = orc.synth_lu(spec, P[i])
        assert np.max(np.abs(s[i] - slu)) < 1e-13 * _ic(P[i])


def _sym_spec(n=65, half=0.6):
    l0 = gi.FE6302[0]
    return gi.ProblemSpec(lines=[(l0, 2.5, 1.0)], lambda_grid=l0 + np.linspace(-half, half, n))


def test_field_free(orc):
    spec = _sym_spec()
    P = gi.draw_params_uniform(50, seed=12)
    P[:, 0] = 0.0
    P[:, 3] = 0.0
    s = orc.synth(spec, P)
    assert np.max(np.abs(s[:, 1:])) == 0.0           # Q = U = V = 0
    assert np.max(np.abs(s[:, 0] - s[:, 0, ::-1])) < 1e-14   # I symmetric about line centre


def test_inclination_limits(orc):
    spec = gi.two_line_spec()
    P = gi.draw_params_uniform(40, seed=13)
    P[:, 1] = 0.0
    s = orc.synth(spec, P)
    assert np.max(np.abs(s[:, 1:3])) == 0.0            # theta = 0: Q = U = 0
    P[:, 1] = 90.0
    s = orc.synth(spec, P)
    assert np.max(np.abs(s[:, 3])) < 1e-14             # theta = 90: V = 0


def test_azimuth_symmetries(orc):
    spec = gi.two_line_spec()
    P = gi.draw_params_uniform(40, seed=14)
    s = orc.synth(spec, P)
    P180 = P.copy(); P180[:, 2] += 180.0
    P90 = P.copy(); P90[:, 2] += 90.0
    s180 = orc.synth(spec, P180)
    s90 = orc.synth(spec, P90)
    tol = 1e-12
    assert np.max(np.abs(s180 - s)) < tol
    assert np.max(np.abs(s90[:, 1:3] + s[:, 1:3])) < tol   # Q, U flip sign
    assert np.max(np.abs(s90[:, 0] - s[:, 0])) < tol
    assert np.max(np.abs(s90[:, 3] - s[:, 3])) < tol


def test_parity_about_line_centre(orc):
    spec = _sym_spec()
    P = gi.draw_params_uniform(40, seed=15)
    P[:, 3] = 0.0
    s = orc.synth(spec, P)
    for k in range(3):
        assert np.max(np.abs(s[:, k] - s[:, k, ::-1])) < 1e-13, k   # I, Q, U even
    assert np.max(np.abs(s[:, 3] + s[:, 3, ::-1])) < 1e-13         # V odd


def test_continuum_and_no_line(orc):
    l0 = gi.FE6302[0]
    far = gi.ProblemSpec(lines=[(l0, 2.5, 1.0)], lambda_grid=l0 + np.array([-40.0, -25.0, 30.0]))
    P = gi.draw_params_uniform(30, seed=16)
    P[:, 5] = 0.0      # no Lorentzian wings: the far wing is exactly continuum
    for mu in [1.0, 0.37]:
        s = orc.synth(far, P, mu=mu)
        ic = P[:, 7] + mu * P[:, 8]
        assert np.max(np.abs(s[:, 0] - ic[:, None])) < 1e-6 * ic.max()
        assert np.max(np.abs(s[:, 1:])) < 1e-6
    P = gi.draw_params_uniform(30, seed=17)
    P[:, 6] = 0.0      # eta0 = 0: K = 1
    s = orc.synth(gi.two_line_spec(), P, mu=0.8)
    ic = P[:, 7] + 0.8 * P[:, 8]
    assert np.max(np.abs(s[:, 0] - ic[:, None])) < 1e-15
    assert np.max(np.abs(s[:, 1:])) == 0.0


def test_weak_field_limit(orc):
    """V -> -dlambda_B cos(theta) dI/dlambda with an O(B^2) error."""
    l0, g = gi.FE6302[0], 2.5
    lam = l0 + np.linspace(-0.5, 0.5, 201)
    h = 1e-5
    spec = gi.ProblemSpec(lines=[(l0, g, 1.0)], lambda_grid=lam)
    specp = gi.ProblemSpec(lines=[(l0, g, 1.0)], lambda_grid=lam + h)
    specm = gi.ProblemSpec(lines=[(l0, g, 1.0)], lambda_grid=lam - h)
    base = np.array([0.0, 30.0, 20.0, 0.4, 30.0, 0.2, 8.0, 0.3, 0.7])
    errs = []
    for B in [2.0, 4.0, 8.0]:
        p = base.copy(); p[0] = B
        s = orc.synth(spec, p)[0]
        dI = (orc.synth(specp, p)[0, 0] - orc.synth(specm, p)[0, 0]) / (2 * h)
        dlB = 4.6686e-13 * g * l0 * l0 * B
        vwf = -dlB * math.cos(math.radians(p[1])) * dI
        errs.append(np.max(np.abs(s[3] - vwf)) / np.max(np.abs(s[3])))
    assert errs[0] < 1e-4
    r1, r2 = errs[1] / errs[0], errs[2] / errs[1]
    assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0, errs   # error ~ B^2


def test_degree_of_polarisation_bounded(orc):
    P = gi.draw_params_uniform(300, seed=18)
    s = orc.synth(gi.two_line_spec(), P)
    pol = np.sqrt(s[:, 1] ** 2 + s[:, 2] ** 2 + s[:, 3] ** 2)
    # the K^-1 e part is a partially polarised beam: |QUV| <= I - S0
    assert np.all(pol <= (s[:, 0] - P[:, 7:8]) * (1 + 1e-12))


def test_weights_invmax_handbuilt(orc):
    n = 8
    obs = np.zeros((4, n))
    obs[0] = [1.0, 0.9, 0.5, 0.2, 0.4, 0.95, 1.0, 1.0]
    obs[1] = [0, 0.01, -0.04, 0.02, 0, 0, 0, 0]
    obs[2] = [0, 0, 0, 0, 0, 0, 0, 0]
    obs[3] = [0.1, -0.25, 0, 0, 0.2, 0, 0, 0]
    w = orc.weights_invmax(obs)
    assert w[0] == pytest.approx(1 / 0.8)
    assert w[1] == pytest.approx(1 / 0.04)
    assert w[2] == pytest.approx(1 / 1e-6)      # identically zero profile: floored
    assert w[3] == pytest.approx(1 / 0.25)


def test_chi2_zero_at_truth_and_unit_with_sigma_weights(orc):
    spec = gi.two_line_spec()
    npix = 512
    P = gi.draw_truth(npix, seed=21)
    clean = orc.synth(spec, P)
    w = np.ones(4)
    assert orc.chi2(clean[0], clean[0], w) == 0.0
    noise = gi.draw_noise(npix, spec.n_lambda, seed=21)
    sig = 1e-3 * (P[:, 7] + P[:, 8])
    obs = clean + sig[:, None, None] * noise
    c2 = np.array([orc.chi2(obs[i], clean[i], np.full(4, 1 / sig[i])) for i in range(npix)])
    nl = spec.n_lambda
    expect = 4 * nl / (4 * nl - 9)
    sd = math.sqrt(2 * 4 * nl) / (4 * nl - 9) / math.sqrt(npix)
    assert abs(c2.mean() - expect) < 4 * sd
