"""GPU Section 5.3 prefit pieces against the oracle: the masked L-M
(lm_fit), the bound rule (me_prefit_bounds, bit-exact) and the GA in
per-pixel bounds (bit-exact in FP64 on the pixels whose decisions the oracle
separates by more than the FP64 evaluation error)."""
import numpy as np
import pytest
import torch

import genesis_inputs as gi
from gpu_helpers import make_obs

pytestmark = pytest.mark.gpu
INF = np.inf


def test_lm_fit_holds_masked_parameters(gpu, orc):
    spec = gi.two_line_spec()
    _, obs = make_obs(orc, spec, 16, seed=3)
    start = gi.draw_params_uniform(16, seed=4)
    for dtype in ["f32", "f64"]:
        pb = gpu.Problem.from_spec(spec, dtype)
        ob = torch.tensor(obs, device="cuda", dtype=pb.torch_dtype)
        for mask in [0x1F8, 0x007, 0x000]:
            p = torch.tensor(start, device="cuda")
            gpu.lm_fit(pb, ob, p, gi.PRIOR_LO, gi.PRIOR_HI, iters=5, free_mask=mask)
            held = [k for k in range(9) if not (mask >> k) & 1]
            assert np.array_equal(p.cpu().numpy()[:, held], start[:, held]), (dtype, mask)


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-7), ("f32", 3e-3)])
def test_prefit_recovers_nonmagnetic_truth(gpu, orc, dtype, tol):
    spec = gi.two_line_spec()
    truth = gi.draw_truth(64, seed=5)
    truth[:, 0], truth[:, 1], truth[:, 2] = 0.0, 90.0, 0.0
    obs = orc.synth(spec, truth)
    pb = gpu.Problem.from_spec(spec, dtype)
    ob = torch.tensor(obs, device="cuda", dtype=pb.torch_dtype)
    p, c2 = gpu.thermo_prefit(pb, ob, gi.PRIOR_LO, gi.PRIOR_HI, iters=60)
    rel = np.abs(p.cpu().numpy()[:, 3:] - truth[:, 3:]) / (gi.PRIOR_HI[3:] - gi.PRIOR_LO[3:])
    assert np.median(np.max(rel, 1)) < tol and np.mean(np.max(rel, 1) < 10 * tol) >= 0.75


def test_prefit_matches_oracle_prefit(gpu, orc):
    """Magnetic pixels: the GPU (FP64) and oracle prefits reach the same
    non-magnetic optimum from the same start."""
    spec = gi.two_line_spec()
    truth, obs = make_obs(orc, spec, 48, seed=6)
    start = np.tile(gpu.PREFIT_START, (48, 1))
    w = np.zeros((48, 4))
    w[:, 0] = 1.0
    ref, rc2 = orc.lm_polish(spec, obs, start, gi.PRIOR_LO, gi.PRIOR_HI, iters=40, w=w, free_mask=gpu.PREFIT_MASK)
    pb = gpu.Problem.from_spec(spec, "f64")
    p, c2 = gpu.thermo_prefit(pb, torch.tensor(obs, device="cuda"), gi.PRIOR_LO, gi.PRIOR_HI, iters=40)
    rel = np.abs(p.cpu().numpy() - ref) / (gi.PRIOR_HI - gi.PRIOR_LO)
    close = np.max(rel, 1) < 1e-4
    assert close.mean() >= 0.85, np.sort(np.max(rel, 1))[-8:]


def test_prefit_bounds_bit_exact(gpu, orc):
    rng = np.random.default_rng(9)
    n = 300
    p_hat = gi.draw_params_uniform(n, seed=9)
    p_hat[::7, 4] = np.nan
    p_hat[::11, 6] = 25.0  # beyond the prior's upper bound
    lower = np.array(gpu.PREFIT_LOWER)
    upper = np.array(gpu.PREFIT_UPPER)
    ref = orc.prefit_bounds(p_hat, gi.PRIOR_LO, gi.PRIOR_HI, lower, upper)
    got = gpu.prefit_bounds(torch.tensor(p_hat, device="cuda"), gi.PRIOR_LO, gi.PRIOR_HI, lower, upper)
    assert np.array_equal(got.cpu().numpy(), ref)
    lower2 = rng.uniform(-0.1, 2.0, 9)
    upper2 = rng.uniform(-0.1, 2.0, 9)
    ref = orc.prefit_bounds(p_hat, gi.PRIOR_LO, gi.PRIOR_HI, lower2, upper2)
    got = gpu.prefit_bounds(torch.tensor(p_hat, device="cuda"), gi.PRIOR_LO, gi.PRIOR_HI, lower2, upper2)
    assert np.array_equal(got.cpu().numpy(), ref)


def test_ga_in_pixel_bounds_fp64_bit_exact(gpu, orc):
    spec = gi.two_line_spec()
    npix, npop, ngen, pid0 = 24, 64, 16, 4000
    truth, obs = make_obs(orc, spec, npix, seed=10)
    start = np.tile(gpu.PREFIT_START, (npix, 1))
    w = np.zeros((npix, 4))
    w[:, 0] = 1.0
    p_hat, _ = orc.lm_polish(spec, obs, start, gi.PRIOR_LO, gi.PRIOR_HI, iters=40, w=w,
                             free_mask=gpu.PREFIT_MASK)
    bpx = orc.prefit_bounds(p_hat, gi.PRIOR_LO, gi.PRIOR_HI, np.array(gpu.PREFIT_LOWER),
                            np.array(gpu.PREFIT_UPPER))
    cls = orc.classify(spec, obs, 1.0, (0, 8), 1, (80, 110))
    cfg = orc.ga_config(npop, ngen, seed=21)
    ref = orc.ga_invert(spec, obs, gi.PRIOR_LO, gi.PRIOR_HI, cfg, pixel_id0=pid0, want_margin=True,
                        seeds=cls["seeds"][:, :2], polarity=cls["polarity"], bounds_px=bpx)
    pb = gpu.Problem.from_spec(spec, "f64")
    best, chi2, genes = gpu.ga_invert_subset(
        pb, torch.tensor(obs, device="cuda"), gi.PRIOR_LO, gi.PRIOR_HI,
        gpu.GaSettings(npop=npop, ngen=ngen, seed=21), seeds=torch.tensor(cls["seeds"][:, :2].copy(), device="cuda"),
        polarity=torch.tensor(cls["polarity"], device="cuda"), bounds_px=torch.tensor(bpx, device="cuda"),
        pixel_id0=pid0, want_genes=True)
    best, genes = best.cpu().numpy(), genes.cpu().numpy().view(np.uint16)
    safe = ref["margin"] > 1e-10
    assert safe.mean() >= 0.8
    assert np.array_equal(genes[safe], ref["genes"][safe])
    assert np.array_equal(best[safe], ref["best"][safe])
    assert np.all(best >= bpx[:, 0] - 1e-12) and np.all(best <= bpx[:, 1] + 1e-12)


def test_invert_map_with_prefit(gpu, orc):
    spec = gi.two_line_spec()
    npix = 48
    truth, obs = make_obs(orc, spec, npix, seed=12)
    pb = gpu.Problem.from_spec(spec, "f32")
    ob = torch.tensor(obs, device="cuda", dtype=torch.float32)
    ga = gpu.GaSettings(npop=64, ngen=30, seed=6)
    r = gpu.invert_map(pb, ob, gi.PRIOR_LO, gi.PRIOR_HI, ga, 1.0, (0, 8), 1, (80, 110), prefit=True,
                       polish_iters=5)
    hi = r["flag"].cpu().numpy() == 1
    assert hi.all()
    bpx = r["bounds_px"].cpu().numpy()
    b = r["best"].cpu().numpy()
    # the GA answer lies in the prefit box; the L-M polish may leave it (global bounds)
    assert np.all(np.isfinite(b)) and np.all(np.isfinite(r["chi2"].cpu().numpy()))
    assert np.all(bpx[:, 0] <= bpx[:, 1])
