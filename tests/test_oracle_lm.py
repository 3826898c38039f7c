"""Pins of the oracle's finite-difference Jacobian and L-M polish.

The Jacobian is pinned by derivatives the model fixes exactly: the source
function enters linearly (d/dS0, d/dS1), the azimuth rotates Q and U by 2 chi,
and for one line the velocity shifts the profile (d/dv = -(lambda0/c) d/dlambda).
The L-M polish is pinned by recovering a noiseless truth from an offset start.
"""
import math

import numpy as np

import genesis_inputs as gi

C_KMS = 299792.458


def test_linear_source_function_columns(orc):
    spec = gi.two_line_spec(n_lambda=48)
    for p in gi.draw_params_uniform(5, seed=40):
        J = orc.jacobian(spec, p)
        s = orc.synth(spec, p)[0]
        assert np.max(np.abs(J[0, :, 7] - 1.0)) < 1e-9 and np.max(np.abs(J[1:, :, 7])) < 1e-9
        ref = s.copy(); ref[0] -= p[7]
        assert np.max(np.abs(J[:, :, 8] - ref / p[8])) < 1e-9


def test_azimuth_column(orc):
    spec = gi.two_line_spec(n_lambda=48)
    k = math.pi / 180.0
    for p in gi.draw_params_uniform(5, seed=41):
        J = orc.jacobian(spec, p)
        s = orc.synth(spec, p)[0]
        assert np.max(np.abs(J[1, :, 2] + 2 * k * s[2])) < 1e-9
        assert np.max(np.abs(J[2, :, 2] - 2 * k * s[1])) < 1e-9
        assert np.max(np.abs(J[0, :, 2])) < 1e-9 and np.max(np.abs(J[3, :, 2])) < 1e-9


def test_velocity_column_is_a_wavelength_shift(orc):
    l0 = gi.FE6302[0]
    lam = l0 + np.linspace(-0.6, 0.6, 61)
    h = 1e-6
    spec = gi.ProblemSpec([(l0, 2.5, 1.0)], lam)
    sp = gi.ProblemSpec([(l0, 2.5, 1.0)], lam + h)
    sm = gi.ProblemSpec([(l0, 2.5, 1.0)], lam - h)
    for p in gi.draw_params_uniform(4, seed=42):
        J = orc.jacobian(spec, p)
        dl = (orc.synth(sp, p)[0] - orc.synth(sm, p)[0]) / (2 * h)
        scale = np.max(np.abs(J[:, :, 3])) + 1e-30
        assert np.max(np.abs(J[:, :, 3] + l0 / C_KMS * dl)) < 1e-6 * scale


def test_lm_recovers_noiseless_truth(orc):
    spec = gi.two_line_spec(n_lambda=96)
    truth = np.array([[1500.0, 60.0, 40.0, 0.7, 32.0, 0.15, 9.0, 0.3, 0.7],
                      [800.0, 130.0, 120.0, -1.2, 28.0, 0.3, 5.0, 0.4, 0.6]])
    obs = orc.synth(spec, truth)
    start = truth * (1 + 0.01 * np.array([1, -1, 1, -1, 1, -1, 1, -1, 1]))
    w = np.ones((2, 4)) * 1e3
    p, c2 = orc.lm_polish(spec, obs, start, gi.PRIOR_LO, gi.PRIOR_HI, iters=40, w=w)
    assert np.max(np.abs(p - truth) / np.abs(truth)) < 1e-8
    assert np.all(c2 < 1e-20)


def test_lm_never_increases_chi2(orc):
    spec = gi.two_line_spec(n_lambda=64)
    truth = gi.draw_truth(6, seed=43)
    noise = gi.draw_noise(6, 64, seed=43)
    obs = orc.synth(spec, truth) + 1e-3 * (truth[:, 7] + truth[:, 8])[:, None, None] * noise
    start = gi.draw_params_uniform(6, seed=44)
    c0 = np.array([orc.chi2(obs[i], orc.synth(spec, start[i])[0], orc.weights_invmax(obs[i]))
                   for i in range(6)])
    for iters in [1, 3, 10]:
        p, c2 = orc.lm_polish(spec, obs, start, gi.PRIOR_LO, gi.PRIOR_HI, iters=iters)
        assert np.all(c2 <= c0 * (1 + 1e-15))
        assert np.all(p >= gi.PRIOR_LO) and np.all(p <= gi.PRIOR_HI)


def test_uncertainty_matches_finite_difference_hessian(orc):
    """Section 6: sigma_i^2 = [H^-1]_ii chi2 / M.  The oracle forms H = (2/nu)
    J^T W^2 J; at a least-squares optimum with small residuals this equals the
    Hessian of chi2 itself, recomputed here by central second differences."""
    spec = gi.two_line_spec(n_lambda=64)
    truth = np.array([[1200.0, 55.0, 35.0, 0.5, 30.0, 0.2, 7.0, 0.35, 0.65]])
    clean = orc.synth(spec, truth)
    obs = clean + 1e-4 * 1.0 * gi.draw_noise(1, 64, seed=50)
    w = np.full((1, 4), 1e4)
    p, c2 = orc.lm_polish(spec, obs, truth, gi.PRIOR_LO, gi.PRIOR_HI, iters=40, w=w)
    sig = orc.lm_uncertainty(spec, obs, p, w=w)[0]

    def chi2(q):
        return orc.chi2(obs[0], orc.synth(spec, q)[0], w[0])

    x = p[0]
    h = 2e-4 * np.maximum(np.abs(x), [100.0, 1.0, 1.0, 0.1, 1.0, 0.01, 0.1, 0.01, 0.01])
    H = np.empty((9, 9))
    for a in range(9):
        for b in range(9):
            def f(sa, sb):
                q = x.copy()
                q[a] += sa * h[a]
                q[b] += sb * h[b]
                return chi2(q)
            H[a, b] = (f(1, 1) - f(1, -1) - f(-1, 1) + f(-1, -1)) / (4 * h[a] * h[b])
    sig_fd = np.sqrt(np.diag(np.linalg.inv(H)) * c2[0] / 9)
    assert np.max(np.abs(sig / sig_fd - 1)) < 2e-2, (sig, sig_fd)
