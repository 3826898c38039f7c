"""GPU fill fraction (Section 5.2, parameter 9) against the oracle: synthesis,
Jacobian, adjoint, the GA (bit-exact in FP64 on margin-safe pixels and
through the operator entry points), the L-M polish, the uncertainty, the
serving loop and the classification's weak-field rows."""
import numpy as np
import pytest
import torch

import genesis_inputs as gi
from gpu_helpers import rel_err

pytestmark = pytest.mark.gpu
FE6301_PATTERN = (gi.FE6301[0], 1.667, gi.eta_ratio_6301(), 2, 11.0 / 6.0, 2, 1.5)
LO, HI = gi.PRIOR_LO_FILL, gi.PRIOR_HI_FILL


def _fill(spec):
    return gi.ProblemSpec(spec.lines, spec.lambda_grid, spec.lambda_dop, spec.mu, fill=True)


def _specs():
    two = gi.two_line_spec()
    pat = gi.ProblemSpec([FE6301_PATTERN, (gi.FE6302[0], 2.5, 1.0)], two.lambda_grid)
    odd = gi.one_line_spec(n_lambda=37)
    return {"two": _fill(two), "pattern": _fill(pat), "one_ragged": _fill(odd)}


def _obs(orc, spec, n, seed, noise=True):
    truth = gi.draw_truth(n, seed=seed, lo=LO, hi=HI)
    clean = orc.synth(spec, truth)
    if not noise:
        return truth, clean
    sig = 1e-3 * (truth[:, 7] + truth[:, 8])
    return truth, clean + sig[:, None, None] * gi.draw_noise(n, spec.n_lambda, seed=seed)


@pytest.mark.parametrize("name", ["two", "pattern", "one_ragged"])
@pytest.mark.parametrize("dtype,tol", [("f32", 2e-5), ("f64", 1e-12)])
def test_synth_matches_oracle(gpu, orc, name, dtype, tol):
    spec = _specs()[name]
    P = gi.draw_params_uniform(200, seed=110, lo=LO, hi=HI)
    P[:4, 9] = 0.0
    P[4:8, 9] = 1.0
    P[8:12, 0] = 0.0
    ref = orc.synth(spec, P)
    pb = gpu.Problem.from_spec(spec, dtype)
    got = gpu.me_synth(pb, torch.tensor(P, device="cuda")).double().cpu().numpy()
    ic = P[:, 7] + P[:, 8]
    if dtype == "f32":
        assert rel_err(got, ref, ic) < tol
    else:
        assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), ic[:, None, None])) < tol


def test_alpha_one_equals_nine_parameter_synthesis(gpu):
    spec9 = gi.two_line_spec()
    P9 = gi.draw_params_uniform(64, seed=111)
    P10 = np.hstack([P9, np.ones((64, 1))])
    for dtype, tol in [("f32", 1e-6), ("f64", 1e-14)]:
        a = gpu.me_synth(gpu.Problem.from_spec(spec9, dtype), torch.tensor(P9, device="cuda")).double()
        b = gpu.me_synth(gpu.Problem.from_spec(_fill(spec9), dtype), torch.tensor(P10, device="cuda")).double()
        assert torch.max(torch.abs(a - b)).item() < tol


@pytest.mark.parametrize("name", ["two", "pattern"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_jacobian_matches_finite_differences(gpu, orc, name, dtype):
    spec = _specs()[name]
    P = gi.draw_params_uniform(24, seed=112, lo=LO, hi=HI)
    P[:, 5] = np.maximum(P[:, 5], 0.02)
    pb = gpu.Problem.from_spec(spec, dtype)
    jac, st = gpu.me_synth_jac(pb, torch.tensor(P, device="cuda"), want_stokes=True)
    jac = jac.double().cpu().numpy()
    assert jac.shape[-1] == 10
    for i in range(len(P)):
        ref = orc.jacobian(spec, P[i])
        scale = np.max(np.abs(ref), axis=(0, 1)) + 1e-30
        err = np.max(np.abs(jac[i] - ref) / scale)
        assert err < (2e-4 if dtype == "f32" else 1e-7), (i, err)


def test_vjp_is_jacobian_transpose(gpu, orc):
    spec = _specs()["two"]
    P = gi.draw_params_uniform(16, seed=113, lo=LO, hi=HI)
    g = np.random.default_rng(4).standard_normal((16, 4, spec.n_lambda))
    pb = gpu.Problem.from_spec(spec, "f64")
    got = gpu.me_synth_vjp(pb, torch.tensor(P, device="cuda"), torch.tensor(g, device="cuda")).cpu().numpy()
    for i in range(len(P)):
        ref = np.einsum("slk,sl->k", orc.jacobian(spec, P[i]), g[i])
        assert np.max(np.abs(got[i] - ref) / (np.abs(ref) + 1e-6 * np.abs(ref).max())) < 1e-6


@pytest.mark.parametrize("npop", [32, 128])
def test_operators_with_ten_genes_bit_exact(gpu, orc, npop):
    rng = np.random.default_rng(npop + 10)
    genes = rng.integers(0, 65536, (4, npop, 10)).astype(np.uint16)
    fit = rng.random((4, npop))
    fit[1, 3] = np.nan
    ga = gpu.GaSettings(npop=npop, pc=0.9, pmut_lsb=0.3, pmut_ratio=0.8, seed=77)
    cfg = orc.ga_config(npop, 10, pc=0.9, pmut_lsb=0.3, pmut_ratio=0.8, seed=77)
    child, elite = gpu.ga_breed(genes, fit, 500, 3, ga)
    for p in range(4):
        ref, e = orc.ga_breed(genes[p], fit[p], 500 + p, 3, cfg)
        assert e == elite[p] and np.array_equal(child[p], ref)
    got = gpu.ga_restart(genes, fit, 9000)
    for p in range(4):
        ref, _ = orc.ga_restart(genes[p], fit[p], 9000)
        assert np.array_equal(got[p], ref)


@pytest.mark.parametrize("name", ["two", "pattern"])
def test_ga_fp64_bit_exact(gpu, orc, name):
    spec = _specs()[name]
    npix, npop, ngen, pid0 = 20, 64, 12, 70
    _, obs = _obs(orc, spec, npix, seed=114)
    cfg = orc.ga_config(npop, ngen, seed=9)
    ref = orc.ga_invert(spec, obs, LO, HI, cfg, pixel_id0=pid0, want_margin=True)
    pb = gpu.Problem.from_spec(spec, "f64")
    best, chi2, genes = gpu.ga_invert_batch(pb, torch.tensor(obs, device="cuda"), LO, HI,
                                            gpu.GaSettings(npop=npop, ngen=ngen, seed=9), pixel_id0=pid0,
                                            want_genes=True)
    best, chi2 = best.cpu().numpy(), chi2.cpu().numpy()
    genes = genes.cpu().numpy().view(np.uint16)
    safe = ref["margin"] > 1e-10
    assert safe.mean() >= 0.8
    assert np.array_equal(genes[safe], ref["genes"][safe])
    assert np.array_equal(best[safe], ref["best"][safe])
    assert np.max(np.abs(chi2[safe] / ref["chi2"][safe] - 1)) < 1e-12
    assert np.all(best >= LO) and np.all(best <= HI)


def test_ga_fp32_and_lm_recover_alpha(gpu, orc):
    spec = _specs()["two"]
    truth = gi.draw_truth(48, seed=115, lo=LO, hi=HI)
    truth[:, 0] = np.maximum(truth[:, 0], 500.0)
    truth[:, 9] = np.clip(truth[:, 9], 0.2, 0.95)
    truth[:, 1] = np.clip(truth[:, 1], 20.0, 160.0)
    clean = orc.synth(spec, truth)
    for dtype, tol in [("f32", 2e-3), ("f64", 1e-7)]:
        pb = gpu.Problem.from_spec(spec, dtype)
        ob = torch.tensor(clean, device="cuda", dtype=pb.torch_dtype)
        start = np.clip(truth * (1 + 0.003 * np.random.default_rng(5).standard_normal(truth.shape)), LO, HI)
        p, c2 = gpu.lm_polish(pb, ob, torch.tensor(start, device="cuda"), LO, HI, iters=40,
                              w=torch.full((48, 4), 1e3, dtype=torch.float64, device="cuda"))
        err = np.abs(p.cpu().numpy() - truth) / (HI - LO)
        assert np.median(err) < tol * 0.1 and np.quantile(err, 0.9) < tol, (dtype, np.quantile(err, 0.9))
    # a short FP32 GA + polish from scratch gets alpha roughly right on noisy data
    _, obs = _obs(orc, spec, 48, seed=116)
    pb = gpu.Problem.from_spec(spec, "f32")
    ob = torch.tensor(obs, device="cuda", dtype=torch.float32)
    best, chi2 = gpu.ga_invert_batch(pb, ob, LO, HI, gpu.GaSettings(npop=128, ngen=100, seed=3))
    assert best.shape == (48, 10) and torch.all(torch.isfinite(chi2))


def test_uncertainty_matches_oracle(gpu, orc):
    spec = _specs()["two"]
    truth = gi.draw_truth(24, seed=117, lo=LO, hi=HI)
    truth[:, 0] = np.maximum(truth[:, 0], 400.0)
    truth[:, 1] = np.clip(truth[:, 1], 20.0, 160.0)
    truth[:, 9] = np.clip(truth[:, 9], 0.2, 0.95)
    clean = orc.synth(spec, truth)
    obs = clean + 1e-3 * (truth[:, 7] + truth[:, 8])[:, None, None] * gi.draw_noise(24, 128, seed=117)
    p, _ = orc.lm_polish(spec, obs, truth, LO, HI, iters=20)
    ref = orc.lm_uncertainty(spec, obs, p)
    pb = gpu.Problem.from_spec(spec, "f64")
    got = gpu.lm_uncertainty(pb, torch.tensor(obs, device="cuda"), torch.tensor(p, device="cuda")).cpu().numpy()
    rel = np.abs(got / ref - 1)
    assert got.shape == (24, 10) and np.median(rel) < 1e-7 and np.max(rel) < 1e-5, (np.median(rel), rel.max())


def test_serving_equals_solo_runs(gpu, orc):
    spec = _specs()["two"]
    pb = gpu.Problem.from_spec(spec, "f32")
    reqs = []
    for i, n in enumerate([40, 130, 65]):
        _, obs = _obs(orc, spec, n, seed=120 + i)
        reqs.append((obs.astype(np.float32), 1000 * i))
    solo = []
    for obs, pid in reqs:
        ob = torch.tensor(obs, device="cuda")
        b, c = gpu.ga_invert_batch(pb, ob, LO, HI, gpu.GaSettings(npop=64, ngen=15, seed=8), pixel_id0=pid)
        b, c = gpu.lm_polish(pb, ob, b, LO, HI, iters=3)
        torch.cuda.synchronize()
        solo.append((b.cpu().numpy(), c.cpu().numpy()))
    with gpu.Server(pb, arena_bytes=32 << 20, max_inflight=3) as srv:
        tickets = [srv.submit(obs, LO, HI, gpu.GaSettings(npop=64, ngen=15, seed=8), pixel_id0=pid,
                              polish_iters=3) for obs, pid in reqs]
        got = [srv.poll(t) for t in tickets]
    for (b, c), g in zip(solo, got):
        assert g["best"].shape[1] == 10
        assert np.array_equal(b, g["best"]) and np.array_equal(c, g["chi2"])


def test_classify_rows_and_bounds_with_alpha(gpu, orc):
    spec = _specs()["two"]
    _, obs = _obs(orc, spec, 30, seed=121)
    pb = gpu.Problem.from_spec(spec, "f64")
    best = torch.full((30, 10), -3.0, dtype=torch.float64, device="cuda")
    r = gpu.classify(pb, torch.tensor(obs, device="cuda"), 60.0, (0, 8), 1, (80, 110), best=best)
    b = best.cpu().numpy()
    lo = r["flag"].cpu().numpy() == 0
    assert lo.any()
    assert np.all(np.isnan(b[lo, 3:])) and np.all(b[~lo] == -3.0)
    p_hat = torch.tensor(gi.draw_params_uniform(30, seed=122, lo=LO, hi=HI), device="cuda")
    bpx = gpu.prefit_bounds(p_hat, LO, HI).cpu().numpy()
    assert bpx.shape == (30, 2, 10)
    assert np.all(bpx[:, 0, 9] == 0.0) and np.all(bpx[:, 1, 9] == 1.0)
    ref = orc.prefit_bounds(p_hat.cpu().numpy(), LO, HI, np.array(gpu.PREFIT_LOWER + (np.inf,)),
                            np.array(gpu.PREFIT_UPPER + (np.inf,)))
    assert np.array_equal(bpx, ref)


def test_fill_bounds_validated(gpu):
    pb = gpu.Problem.from_spec(_specs()["two"], "f32")
    ob = torch.zeros((2, 4, 128), dtype=torch.float32, device="cuda")
    bad_hi = HI.copy()
    bad_hi[9] = 1.5
    with pytest.raises(Exception):
        gpu.ga_invert_batch(pb, ob, LO, bad_hi, gpu.GaSettings(npop=32, ngen=1))
