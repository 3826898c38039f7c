"""Pins of the oracle's Section 5.2 fill fraction alpha (10th parameter).

* alpha = 1 is the 9-parameter synthesis, bit for bit.
* alpha = 0 leaves Q = U = V = 0 and an I equal to the 9-parameter
  synthesis with B = 0, which reaches the field-free profile through the
  full propagation matrix (an independent path), for triplet and full-pattern
  lines.
* The model is affine in alpha, and the Jacobian's alpha column is the
  difference of the two end members.
* L-M recovers noiseless truth including alpha; the zero-generation GA
  places a seed in a 10-gene individual; the Section 6 uncertainty matches a
  finite-difference Hessian in 10 dimensions.
"""
import numpy as np
import pytest

import genesis_inputs as gi

FE6301_PATTERN = (gi.FE6301[0], 1.667, gi.eta_ratio_6301(), 2, 11.0 / 6.0, 2, 1.5)


def _specs(n_lambda=96):
    two = gi.two_line_spec(n_lambda=n_lambda)
    pat = gi.ProblemSpec([FE6301_PATTERN, (gi.FE6302[0], 2.5, 1.0)], two.lambda_grid)
    return [two, pat]


def _fill(spec):
    return gi.ProblemSpec(spec.lines, spec.lambda_grid, spec.lambda_dop, spec.mu, fill=True)


@pytest.mark.parametrize("k", [0, 1])
def test_alpha_one_is_the_magnetic_model(orc, k):
    spec = _specs()[k]
    p9 = gi.draw_truth(6, seed=30 + k)
    p10 = np.hstack([p9, np.ones((6, 1))])
    assert np.array_equal(orc.synth(_fill(spec), p10), orc.synth(spec, p9))


@pytest.mark.parametrize("k", [0, 1])
def test_alpha_zero_is_the_field_free_model(orc, k):
    spec = _specs()[k]
    p9 = gi.draw_truth(6, seed=40 + k)
    s0 = orc.synth(_fill(spec), np.hstack([p9, np.zeros((6, 1))]))
    assert np.all(s0[:, 1:] == 0.0)
    b0 = p9.copy()
    b0[:, 0] = 0.0
    ref = orc.synth(spec, b0)
    assert np.max(np.abs(s0[:, 0] - ref[:, 0])) < 1e-14


def test_affine_in_alpha_and_jacobian_column(orc):
    spec = _specs()[0]
    fs = _fill(spec)
    p9 = gi.draw_truth(4, seed=50)
    one = orc.synth(fs, np.hstack([p9, np.ones((4, 1))]))
    zero = orc.synth(fs, np.hstack([p9, np.zeros((4, 1))]))
    for a in [0.37, 0.81]:
        mid = orc.synth(fs, np.hstack([p9, np.full((4, 1), a)]))
        assert np.max(np.abs(mid - (a * one + (1 - a) * zero))) < 1e-14
    for i in range(4):
        p = np.append(p9[i], 0.6)
        J = orc.jacobian(fs, p)
        assert J.shape == (4, spec.n_lambda, 10)
        assert np.max(np.abs(J[:, :, 9] - (one[i] - zero[i]))) < 1e-9
        # the other columns are alpha times the magnetic ones plus (1 - alpha) times the field-free I's
        J9 = orc.jacobian(spec, p9[i])
        assert np.max(np.abs(J[1:, :, :9] - 0.6 * J9[1:])) < 1e-7 * (1 + np.max(np.abs(J9[1:])))


def test_lm_recovers_alpha(orc):
    fs = _fill(_specs()[0])
    truth = np.array([[1500.0, 60.0, 40.0, 0.7, 32.0, 0.15, 9.0, 0.3, 0.7, 0.45],
                      [800.0, 130.0, 120.0, -1.2, 28.0, 0.3, 5.0, 0.4, 0.6, 0.8]])
    obs = orc.synth(fs, truth)
    start = truth * (1 + 0.01 * np.array([1, -1, 1, -1, 1, -1, 1, -1, 1, -1]))
    p, c2 = orc.lm_polish(fs, obs, start, gi.PRIOR_LO_FILL, gi.PRIOR_HI_FILL, iters=60, w=np.full((2, 4), 1e3))
    assert np.max(np.abs(p - truth) / np.abs(truth)) < 1e-7, p - truth
    assert np.all(c2 < 1e-18)


def test_zero_generation_seed_in_ten_genes(orc):
    fs = _fill(_specs(64)[0])
    npop = 16
    cfg = orc.ga_config(npop, 0, seed=2)
    seeds = np.array([[[1100.0, 50.0, 70.0]]])
    g = np.array([orc.sobol_u32(npop, d) >> 16 for d in range(10)], dtype=np.uint16)
    for d in range(3):
        g[d] = orc.ga_encode(seeds[0, 0, d], gi.PRIOR_LO_FILL[d], gi.PRIOR_HI_FILL[d])
    obs = orc.synth(fs, orc.ga_decode(g, gi.PRIOR_LO_FILL, gi.PRIOR_HI_FILL)[None])
    r = orc.ga_invert(fs, obs, gi.PRIOR_LO_FILL, gi.PRIOR_HI_FILL, cfg, seeds=seeds, nthreads=1)
    assert np.array_equal(r["genes"][0], g) and r["chi2"][0] == 0.0
    assert r["best"].shape == (1, 10)


def test_uncertainty_in_ten_dimensions(orc):
    fs = _fill(_specs(64)[0])
    truth = np.array([[1200.0, 55.0, 35.0, 0.5, 30.0, 0.2, 7.0, 0.35, 0.65, 0.7]])
    obs = orc.synth(fs, truth) + 1e-4 * gi.draw_noise(1, 64, seed=51)
    w = np.full((1, 4), 1e4)
    p, c2 = orc.lm_polish(fs, obs, truth, gi.PRIOR_LO_FILL, gi.PRIOR_HI_FILL, iters=60, w=w)
    sig = orc.lm_uncertainty(fs, obs, p, w=w)[0]
    x = p[0]
    h = 2e-4 * np.maximum(np.abs(x), [100.0, 1.0, 1.0, 0.1, 1.0, 0.01, 0.1, 0.01, 0.01, 0.01])

    def chi2(q):
        return orc.chi2(obs[0], orc.synth(fs, q)[0], w[0], m=10)

    H = np.empty((10, 10))
    for a in range(10):
        for b in range(10):
            def f(sa, sb):
                q = x.copy()
                q[a] += sa * h[a]
                q[b] += sb * h[b]
                return chi2(q)
            H[a, b] = (f(1, 1) - f(1, -1) - f(-1, 1) + f(-1, -1)) / (4 * h[a] * h[b])
    sig_fd = np.sqrt(np.diag(np.linalg.inv(H)) * c2[0] / 10)
    assert np.max(np.abs(sig / sig_fd - 1)) < 3e-2, (sig, sig_fd)
