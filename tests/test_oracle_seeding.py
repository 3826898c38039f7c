"""Pins of the oracle's Section 5.5 seeding and polarity restriction.

* The seed encoding is the nearest gene: a round trip through the decode is
  the identity on all 65536 genes, and brute force over every gene finds
  none closer to a random value.
* Placement: with zero generations, a seeded individual whose synthesis is
  the observation wins with chi2 = 0, and its genes are the encoded seed in
  (B, psi, chi) and the Sobol point of its slot elsewhere.
* Polarity: the inclination of every individual stays in the pixel's half.
"""
import numpy as np
import pytest

import genesis_inputs as gi


@pytest.mark.parametrize("lo,hi", [(0.0, 180.0), (0.0, 5000.0), (-4.0, 4.0), (0.5, 40.0)])
def test_encode_inverts_decode(orc, lo, hi):
    g = np.arange(65536, dtype=np.uint16)
    lo9 = np.full(9, lo)
    hi9 = np.full(9, hi)
    for k in range(0, 65536, 4099):
        gg = np.full(9, g[k], dtype=np.uint16)
        x = orc.ga_decode(gg, lo9, hi9)[0]
        assert orc.ga_encode(x, lo, hi) == g[k]
    assert orc.ga_encode(lo - 1.0, lo, hi) == 0 and orc.ga_encode(hi + 1.0, lo, hi) == 65535


def test_encode_is_nearest_gene_brute_force(orc):
    lo, hi = 0.0, 5000.0
    grid = lo + (hi - lo) * (np.arange(65536) / 65535.0)
    rng = np.random.default_rng(3)
    for x in rng.uniform(lo, hi, 200):
        g = orc.ga_encode(x, lo, hi)
        assert abs(grid[g] - x) <= np.min(np.abs(grid - x)) * (1 + 1e-12)


def test_polarity_bounds(orc):
    assert orc.polarity_bounds(1, 0.0, 180.0) == (0.0, 90.0)
    assert orc.polarity_bounds(-1, 0.0, 180.0) == (90.0, 180.0)
    assert orc.polarity_bounds(0, 0.0, 180.0) == (0.0, 180.0)
    assert orc.polarity_bounds(1, 10.0, 60.0) == (10.0, 60.0)
    assert orc.polarity_bounds(-1, 10.0, 60.0) == (10.0, 60.0)  # empty half: full domain
    assert orc.polarity_bounds(-1, 30.0, 120.0) == (90.0, 120.0)


@pytest.mark.parametrize("pol", [None, 1, -1])
def test_seed_lands_in_last_slots(orc, pol):
    spec = gi.two_line_spec(n_lambda=48)
    npop, nseed = 16, 3
    cfg = orc.ga_config(npop, 0, seed=5)
    lo, hi = gi.PRIOR_LO.copy(), gi.PRIOR_HI.copy()
    plo, phi = lo.copy(), hi.copy()
    if pol is not None:
        plo[1], phi[1] = orc.polarity_bounds(pol, lo[1], hi[1])
    seeds = np.array([[[1200.0, 70.0 if pol != -1 else 110.0, 33.0],
                       [800.0, np.nan, 150.0],
                       [2500.0, 20.0 if pol != -1 else 160.0, 90.0]]])
    for s in range(nseed):
        slot = npop - nseed + s
        genes = np.array([orc.sobol_u32(slot + 1, d) >> 16 for d in range(9)], dtype=np.uint16)
        for d in range(3):
            if not np.isnan(seeds[0, s, d]):
                genes[d] = orc.ga_encode(seeds[0, s, d], plo[d], phi[d])
        obs = orc.synth(spec, orc.ga_decode(genes, plo, phi)[None])
        polar = None if pol is None else np.array([pol])
        r = orc.ga_invert(spec, obs, lo, hi, cfg, seeds=seeds, polarity=polar, nthreads=1)
        assert np.array_equal(r["genes"][0], genes), (s, r["genes"][0], genes)
        assert r["chi2"][0] == 0.0


def test_polarity_confines_inclination(orc):
    spec = gi.two_line_spec(n_lambda=64)
    truth = np.array([[1500.0, 140.0, 60.0, 0.3, 30.0, 0.2, 8.0, 0.3, 0.7]] * 2)
    obs = orc.synth(spec, truth)
    cfg = orc.ga_config(32, 30, seed=9)
    r = orc.ga_invert(spec, obs, gi.PRIOR_LO, gi.PRIOR_HI, cfg, polarity=np.array([1, -1]), nthreads=2)
    assert r["best"][0, 1] <= 90.0 and r["best"][1, 1] >= 90.0
    assert r["chi2"][1] < r["chi2"][0]


def test_seeds_from_classification_help(orc):
    """Seeding the GA with the weak-field and related estimates improves the
    short-run fit of weak-field pixels on average (Section 5.5)."""
    spec = gi.two_line_spec(n_lambda=96)
    truth = gi.draw_truth(24, seed=21)
    truth[:, 0] = np.linspace(100.0, 600.0, 24)
    obs = orc.synth(spec, truth) + 1e-3 * gi.draw_noise(24, 96, seed=21)
    cls = orc.classify(spec, obs, 1.0, (0, 8), 0, (20, 60))
    cfg = orc.ga_config(32, 8, seed=2)
    plain = orc.ga_invert(spec, obs, gi.PRIOR_LO, gi.PRIOR_HI, cfg)
    seeded = orc.ga_invert(spec, obs, gi.PRIOR_LO, gi.PRIOR_HI, cfg, seeds=cls["seeds"],
                           polarity=cls["polarity"])
    assert np.median(seeded["chi2"]) < np.median(plain["chi2"])
    ok = cls["polarity"] != 0
    assert np.all(np.where(cls["polarity"][ok] > 0, seeded["best"][ok, 1] <= 90, seeded["best"][ok, 1] >= 90))
