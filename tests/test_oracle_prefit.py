"""Pins of the oracle's Section 5.3 thermodynamic prefit pieces: the L-M
parameter mask, the bound rule around a prefit, and per-pixel GA bounds.

* Held parameters never move, bit for bit, and a Stokes-I-only fit with the
  field held at zero recovers noiseless non-magnetic truth from a generic
  start (the model contains its own synthesis).
* The bound rule is checked on hand-sized cases (clipping, one-sided and
  infinite margins, NaN prefit, empty interval).
* Per-pixel bounds equal to the global ones reproduce the unbounded GA bit
  for bit; a box keeps every decoded answer inside it; seeds are encoded in
  the pixel's own bounds.
"""
import numpy as np

import genesis_inputs as gi

INF = np.inf
PREFIT_MASK = 0x1F8  # v, dlambda_D, a, eta0, S0, S1 free; B, theta, chi held


def test_mask_holds_parameters_bit_for_bit(orc):
    spec = gi.two_line_spec(n_lambda=64)
    truth = gi.draw_truth(4, seed=1)
    obs = orc.synth(spec, truth) + 1e-3 * gi.draw_noise(4, 64, seed=1)
    start = gi.draw_params_uniform(4, seed=2)
    for mask in [0x1F8, 0x007, 0x100, 0x000]:
        p, _ = orc.lm_polish(spec, obs, start, gi.PRIOR_LO, gi.PRIOR_HI, iters=6, free_mask=mask)
        held = [k for k in range(9) if not (mask >> k) & 1]
        assert np.array_equal(p[:, held], start[:, held]), mask
    p0, c0 = orc.lm_polish(spec, obs, start, gi.PRIOR_LO, gi.PRIOR_HI, iters=6, free_mask=0x000)
    c_start = [orc.chi2(obs[i], orc.synth(spec, start[i])[0], orc.weights_invmax(obs[i])) for i in range(4)]
    assert np.allclose(c0, c_start, rtol=1e-15)


def test_stokes_i_prefit_recovers_nonmagnetic_truth(orc):
    spec = gi.two_line_spec()
    truth = gi.draw_truth(8, seed=4)
    truth[:, 0] = 0.0
    truth[:, 1] = 90.0
    truth[:, 2] = 0.0
    obs = orc.synth(spec, truth)
    start = np.tile([0.0, 90.0, 0.0, 0.0, 35.0, 0.2, 5.0, 0.3, 0.7], (8, 1))
    w = np.zeros((8, 4))
    w[:, 0] = 1e3
    p, c2 = orc.lm_polish(spec, obs, start, gi.PRIOR_LO, gi.PRIOR_HI, iters=60, w=w, free_mask=PREFIT_MASK)
    rel = np.abs(p[:, 3:] - truth[:, 3:]) / (gi.PRIOR_HI[3:] - gi.PRIOR_LO[3:])
    assert np.median(rel) < 1e-8 and np.mean(np.max(rel, 1) < 1e-6) >= 0.75, rel.max(1)


def test_prefit_bound_rule_hand_cases(orc):
    lo = np.zeros(9)
    hi = np.full(9, 10.0)
    p = np.array([[5.0, 5.0, 5.0, 0.5, 9.5, np.nan, 5.0, 5.0, 12.0]])
    lower = np.array([1.0, INF, 2.0, 1.0, 1.0, 1.0, 0.0, -1.0, 1.0])
    upper = np.array([1.0, 2.0, INF, 1.0, 1.0, 1.0, 0.0, 3.0, 1.0])
    b = orc.prefit_bounds(p, lo, hi, lower, upper)[0]
    exp_lo = [4.0, 0.0, 3.0, 0.0, 8.5, 0.0, 0.0, 0.0, 0.0]
    exp_hi = [6.0, 7.0, 10.0, 1.5, 10.0, 10.0, 10.0, 10.0, 10.0]
    # k = 5: NaN prefit -> global; k = 6: zero margins -> empty -> global;
    # k = 7: negative lower margin leaves [6, 8], k = 8: prefit beyond hi -> [11, 10] empty -> global
    exp_lo[7], exp_hi[7] = 6.0, 8.0
    assert np.array_equal(b[0], exp_lo), b[0]
    assert np.array_equal(b[1], exp_hi), b[1]


def test_global_pixel_bounds_reproduce_the_plain_ga(orc):
    spec = gi.two_line_spec(n_lambda=64)
    obs = orc.synth(spec, gi.draw_truth(5, seed=6))
    cfg = orc.ga_config(32, 12, seed=3)
    bpx = np.tile(np.stack([gi.PRIOR_LO, gi.PRIOR_HI])[None], (5, 1, 1))
    a = orc.ga_invert(spec, obs, gi.PRIOR_LO, gi.PRIOR_HI, cfg)
    b = orc.ga_invert(spec, obs, gi.PRIOR_LO, gi.PRIOR_HI, cfg, bounds_px=bpx)
    assert np.array_equal(a["genes"], b["genes"]) and np.array_equal(a["best"], b["best"])


def test_pixel_box_confines_answers_and_seeds(orc):
    spec = gi.two_line_spec(n_lambda=64)
    truth = gi.draw_truth(6, seed=8)
    obs = orc.synth(spec, truth)
    bpx = np.empty((6, 2, 9))
    bpx[:, 0] = np.maximum(gi.PRIOR_LO, truth - 0.1 * (gi.PRIOR_HI - gi.PRIOR_LO))
    bpx[:, 1] = np.minimum(gi.PRIOR_HI, truth + 0.1 * (gi.PRIOR_HI - gi.PRIOR_LO))
    cfg = orc.ga_config(32, 10, seed=4)
    r = orc.ga_invert(spec, obs, gi.PRIOR_LO, gi.PRIOR_HI, cfg, bounds_px=bpx, nthreads=2)
    assert np.all(r["best"] >= bpx[:, 0]) and np.all(r["best"] <= bpx[:, 1])
    # a seed in the last slot, ngen = 0: its genes are encoded in the pixel's box
    seeds = truth[:, None, :3].copy()
    cfg0 = orc.ga_config(32, 0, seed=4)
    r0 = orc.ga_invert(spec, obs, gi.PRIOR_LO, gi.PRIOR_HI, cfg0, bounds_px=bpx, seeds=seeds, nthreads=1)
    for i in range(6):
        g = np.array([orc.sobol_u32(32, d) >> 16 for d in range(9)], dtype=np.uint16)
        for d in range(3):
            g[d] = orc.ga_encode(seeds[i, 0, d], bpx[i, 0, d], bpx[i, 1, d])
        dec = orc.ga_decode(g, bpx[i, 0], bpx[i, 1])
        c_seed = orc.chi2(obs[i], orc.synth(spec, dec[None])[0], orc.weights_invmax(obs[i]))
        assert r0["chi2"][i] <= c_seed
