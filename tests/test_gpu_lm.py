"""GPU Levenberg-Marquardt polish against the oracle's and the truth."""
import numpy as np
import pytest
import torch

import genesis_inputs as gi
from gpu_helpers import make_obs

pytestmark = pytest.mark.gpu


def test_lm_recovers_noiseless_truth(gpu, orc):
    spec = gi.two_line_spec()
    truth = gi.draw_truth(64, seed=20)
    truth[:, 0] = np.maximum(truth[:, 0], 300.0)      # well-determined field
    truth[:, 5] = np.clip(truth[:, 5], 0.05, 0.45)
    truth[:, 1] = np.clip(truth[:, 1], 15.0, 165.0)
    _, obs = make_obs(orc, spec, 64, 20, noise=False, truth=truth)
    start = truth * (1 + 0.003 * np.random.default_rng(1).standard_normal(truth.shape))
    start = np.clip(start, gi.PRIOR_LO, gi.PRIOR_HI)
    w = np.full((64, 4), 1e3)
    for dtype, tol in [("f32", 2e-3), ("f64", 1e-7)]:
        pb = gpu.Problem.from_spec(spec, dtype)
        ob = torch.tensor(obs, device="cuda", dtype=pb.torch_dtype)
        p, c2 = gpu.lm_polish(pb, ob, torch.tensor(start, device="cuda"), gi.PRIOR_LO, gi.PRIOR_HI,
                              iters=30, w=torch.tensor(w, device="cuda"))
        p = p.cpu().numpy()
        err = np.abs(p - truth) / (gi.PRIOR_HI - gi.PRIOR_LO)
        assert np.median(err) < tol * 0.1 and np.quantile(err, 0.9) < tol, (dtype, np.quantile(err, 0.9))


@pytest.mark.parametrize("start_kind", ["perturbed", "zero_field"])
def test_lm_matches_oracle_polish(gpu, orc, start_kind):
    """From the same starting vectors the GPU and the oracle reach the same
    chi2.  A zero-field start (B = 0) leaves theta and chi without influence
    (all Zeeman components coincide), so only the damping floor keeps those
    rows of the normal equations positive definite."""
    spec = gi.two_line_spec()
    truth, obs = make_obs(orc, spec, 48, seed=21)
    start = np.clip(truth * (1 + 0.02 * np.random.default_rng(2).standard_normal(truth.shape)),
                    gi.PRIOR_LO, gi.PRIOR_HI)
    if start_kind == "zero_field":
        start[:, 0] = 0.0
    p_ref, c_ref = orc.lm_polish(spec, obs, start, gi.PRIOR_LO, gi.PRIOR_HI, iters=10)
    pb = gpu.Problem.from_spec(spec, "f64")
    p, c2 = gpu.lm_polish(pb, torch.tensor(obs, device="cuda"), torch.tensor(start, device="cuda"),
                          gi.PRIOR_LO, gi.PRIOR_HI, iters=10)
    c2 = c2.cpu().numpy()
    # both descend from the same start; they land within 1% of each other
    assert np.median(np.abs(c2 - c_ref) / c_ref) < 1e-3
    assert np.quantile(np.abs(c2 - c_ref) / c_ref, 0.9) < 1e-2
    c0 = np.array([orc.chi2(obs[i], orc.synth(spec, start[i])[0], orc.weights_invmax(obs[i]))
                   for i in range(48)])
    assert np.all(c2 <= c0 * (1 + 1e-12))


def test_lm_fp32_never_worse_and_in_bounds(gpu, orc):
    spec = gi.two_line_spec()
    truth, obs = make_obs(orc, spec, 128, seed=22)
    start = gi.draw_params_uniform(128, seed=23)
    pb = gpu.Problem.from_spec(spec, "f32")
    ob = torch.tensor(obs, device="cuda", dtype=torch.float32)
    st = torch.tensor(start, device="cuda")
    c0 = gpu.me_chi2(pb, ob, st)
    p, c2 = gpu.lm_polish(pb, ob, st, gi.PRIOR_LO, gi.PRIOR_HI, iters=10)
    assert torch.all(c2 <= c0 * (1 + 1e-5))
    pn = p.cpu().numpy()
    assert np.all(pn >= gi.PRIOR_LO) and np.all(pn <= gi.PRIOR_HI)
    assert np.all((pn[:, 2] >= 0) & (pn[:, 2] < 180.0 + 1e-12))


def test_fp32_served_form_against_fp64_oracle_per_parameter(gpu, orc):
    """The FP32 GA + FP32 L-M answer against the FP64 oracle's L-M from the
    same GA best: the same chi2 and, per parameter, differences far below the
    noise-set uncertainties (the error of the FP32 path stated per parameter)."""
    spec = gi.two_line_spec()
    n = 96
    truth, obs = make_obs(orc, spec, n, seed=60)
    obs32 = obs.astype(np.float32)
    sig = 1e-3 * (truth[:, 7] + truth[:, 8])
    w = np.repeat((1 / sig)[:, None], 4, 1)
    pb = gpu.Problem.from_spec(spec, "f32")
    ob = torch.tensor(obs32, device="cuda")
    best, _ = gpu.ga_invert_batch(pb, ob, gi.PRIOR_LO, gi.PRIOR_HI, gpu.GaSettings(npop=128, ngen=100, seed=3))
    p32, c32 = gpu.lm_polish(pb, ob, best, gi.PRIOR_LO, gi.PRIOR_HI, iters=10, w=torch.tensor(w, device="cuda"))
    p64, c64 = orc.lm_polish(spec, obs32.astype(np.float64), best.cpu().numpy(), gi.PRIOR_LO, gi.PRIOR_HI,
                             iters=10, w=w)
    p32, c32 = p32.cpu().numpy(), c32.cpu().numpy()
    ratio = c32 / c64
    assert abs(np.median(ratio) - 1) < 1e-6 and np.quantile(np.abs(ratio - 1), 0.9) < 1e-4
    d = np.abs(p32 - p64)
    d[:, 2] = np.abs((p32[:, 2] - p64[:, 2] + 90) % 180 - 90)
    rel = np.median(d, 0) / (gi.PRIOR_HI - gi.PRIOR_LO)
    assert np.all(rel < 1e-5), rel


@pytest.mark.parametrize("lambda0", [1.0, 1e-3])
def test_lm_single_fp64_step_matches_oracle(gpu, orc, lambda0):
    """One FP64 L-M iteration from the same (p, lambda): the GPU's analytic
    Jacobian, its normal equations and its warp Cholesky against the oracle's
    Richardson Jacobian and serial Cholesky.  In Marquardt's scaled variables
    u = D^(1/2) delta (D = diag J^T W^2 J) the damped matrix C + lambda I has
    unit-diagonal C, so its condition number is at most (9 + lambda) / lambda;
    Jacobians that agree to about 1e-12 then give steps that agree to 1e-8 or
    better.  Measured: 3e-11 (lambda 1) and 5e-12 (lambda 1e-3)."""
    spec = gi.two_line_spec()
    n = 32
    truth = gi.draw_truth(n, seed=70)
    for k, (a, b) in enumerate([(300, 2900), (20, 160), (20, 160), (-2.5, 2.5), (22, 48), (0.05, 0.45), (2, 19),
                                (0.15, 0.95), (0.15, 0.95)]):
        truth[:, k] = np.clip(truth[:, k], a, b)
    _, obs = make_obs(orc, spec, n, 70, noise=False, truth=truth)
    start = truth * (1 + 0.01 * np.random.default_rng(7).standard_normal(truth.shape))
    sig = 1e-3 * (truth[:, 7] + truth[:, 8])
    w = np.repeat((1 / sig)[:, None], 4, 1)
    p_ref, _ = orc.lm_polish(spec, obs, start, gi.PRIOR_LO, gi.PRIOR_HI, iters=1, lambda0=lambda0, w=w)
    pb = gpu.Problem.from_spec(spec, "f64")
    p_g, _ = gpu.lm_polish(pb, torch.tensor(obs, device="cuda"), torch.tensor(start, device="cuda"),
                           gi.PRIOR_LO, gi.PRIOR_HI, iters=1, lambda0=lambda0, w=torch.tensor(w, device="cuda"))
    p_g = p_g.cpu().numpy()
    d_ref, d_gpu = p_ref - start, p_g - start
    # both take the step (a 1% offset on noiseless data always lowers chi2)
    assert np.all(np.any(d_ref != 0, 1)) and np.all(np.any(d_gpu != 0, 1))
    for i in range(n):
        J = orc.jacobian(spec, start[i])
        D = np.einsum("s,sjk->k", w[i] ** 2, J ** 2)
        u_ref, u_gpu = np.sqrt(D) * d_ref[i], np.sqrt(D) * d_gpu[i]
        assert np.max(np.abs(u_gpu - u_ref)) <= 1e-9 * np.max(np.abs(u_ref)), i
