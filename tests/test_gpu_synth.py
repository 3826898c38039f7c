"""GPU synthesis, Jacobian, adjoint and chi2 against the FP64 oracle.

Tolerances: FP32 synthesis within 2e-5 of max(|oracle|, I_c) per sample; FP64
within 1e-12 relative (both as stated for the method's precision modes).
"""
import numpy as np
import pytest
import torch

import genesis_inputs as gi
from gpu_helpers import rel_err

pytestmark = pytest.mark.gpu


def _pb(gpu, spec, dtype):
    return gpu.Problem.from_spec(spec, dtype)


def _specs():
    three = gi.ProblemSpec(lines=[(gi.FE6301[0], 1.667, gi.eta_ratio_6301()),
                                  (gi.FE6302[0], 2.5, 1.0), (6302.2, 1.2, 0.4)],
                           lambda_grid=np.linspace(6301.0, 6303.0, 37))
    four = gi.ProblemSpec(lines=three.lines + [(6301.9, 0.8, 0.2)],
                          lambda_grid=np.linspace(6300.8, 6303.1, 512))
    return {"one": gi.one_line_spec(), "two": gi.two_line_spec(), "three_ragged": three,
            "four_max_lambda": four}


@pytest.mark.parametrize("name", ["one", "two", "three_ragged", "four_max_lambda"])
@pytest.mark.parametrize("dtype,tol", [("f32", 2e-5), ("f64", 1e-12)])
def test_synth_matches_oracle(gpu, orc, name, dtype, tol):
    spec = _specs()[name]
    P = gi.draw_params_uniform(300, seed=100)
    P[:5, 0] = 0.0           # field free
    P[5:10, 5] = 0.0         # no damping
    P[10:15, 1] = 0.0        # longitudinal
    P[15:20, 1] = 90.0       # transverse
    P[20:25, 3] = 3.0        # velocity at the bound
    mu = np.linspace(0.05, 1.0, len(P))
    ref = orc.synth(spec, P, mu_px=mu)
    pb = _pb(gpu, spec, dtype)
    out = gpu.me_synth(pb, torch.tensor(P, device="cuda"), torch.tensor(mu, device="cuda"))
    got = out.double().cpu().numpy()
    ic = P[:, 7] + mu * P[:, 8]
    if dtype == "f32":
        assert rel_err(got, ref, ic) < tol
    else:
        assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), ic[:, None, None])) < tol


def test_synth_zero_models_is_noop(gpu):
    pb = _pb(gpu, gi.two_line_spec(), "f32")
    out = gpu.me_synth(pb, torch.empty((0, 9), dtype=torch.float64, device="cuda"))
    assert out.shape == (0, 4, 128)


def test_synth_full_disc_size_sampled(gpu, orc):
    """The full-disc cube size (3.3M models) in one launch, checked on a sample."""
    spec = gi.two_line_spec()
    n = 3_290_000
    gen = torch.Generator(device="cuda").manual_seed(7)
    lo = torch.tensor(gi.PRIOR_LO, device="cuda")
    hi = torch.tensor(gi.PRIOR_HI, device="cuda")
    P = lo + (hi - lo) * torch.rand((n, 9), generator=gen, device="cuda", dtype=torch.float64)
    pb = _pb(gpu, spec, "f32")
    out = gpu.me_synth(pb, P)
    idx = np.random.default_rng(1).choice(n, 64, replace=False)
    idx[-1] = n - 1
    Ps = P[idx].cpu().numpy()
    ref = orc.synth(spec, Ps)
    got = out[idx].double().cpu().numpy()
    assert rel_err(got, ref, Ps[:, 7] + Ps[:, 8]) < 2e-5
    del out, P
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_jacobian_matches_finite_differences(gpu, orc, dtype):
    spec = gi.two_line_spec(n_lambda=64)
    P = gi.draw_params_uniform(40, seed=101)
    P[:, 5] = np.maximum(P[:, 5], 0.02)
    pb = _pb(gpu, spec, dtype)
    jac, st = gpu.me_synth_jac(pb, torch.tensor(P, device="cuda"), want_stokes=True)
    jac = jac.double().cpu().numpy()
    for i in range(len(P)):
        ref = orc.jacobian(spec, P[i])
        scale = np.max(np.abs(ref), axis=(0, 1)) + 1e-30     # per parameter column
        err = np.max(np.abs(jac[i] - ref) / scale)
        assert err < (2e-4 if dtype == "f32" else 1e-7), (i, err)
    ref_st = orc.synth(spec, P)
    assert rel_err(st.double().cpu().numpy(), ref_st, P[:, 7] + P[:, 8]) < (2e-5 if dtype == "f32" else 1e-12)


def test_vjp_is_jacobian_transpose(gpu, orc):
    spec = gi.two_line_spec(n_lambda=96)
    P = gi.draw_params_uniform(24, seed=102)
    g = np.random.default_rng(3).standard_normal((24, 4, 96))
    pb = _pb(gpu, spec, "f64")
    out = gpu.me_synth_vjp(pb, torch.tensor(P, device="cuda"), torch.tensor(g, device="cuda"))
    got = out.cpu().numpy()
    for i in range(len(P)):
        ref = np.einsum("slk,sl->k", orc.jacobian(spec, P[i]), g[i])
        assert np.max(np.abs(got[i] - ref) / (np.abs(ref) + 1e-6 * np.abs(ref).max())) < 1e-6


def test_autograd_function_gradcheck(gpu):
    spec = gi.one_line_spec(n_lambda=24)
    pb = _pb(gpu, spec, "f64")
    P = torch.tensor(gi.draw_params_uniform(3, seed=103), device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda p: gpu.synth_autograd(pb, p), (P,), eps=1e-6, atol=1e-6,
                                    rtol=1e-5)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_chi2_f64_matches_oracle(gpu, orc, dtype):
    spec = gi.two_line_spec()
    truth = gi.draw_truth(64, seed=104)
    obs = orc.synth(spec, truth) + 1e-3 * gi.draw_noise(64, 128, seed=104)
    if dtype == "f32":
        obs = obs.astype(np.float32).astype(np.float64)   # the cube the GPU sees
    P = gi.draw_params_uniform(64, seed=105)
    w = orc.weights_invmax(obs)
    ref = np.array([orc.chi2(obs[i], orc.synth(spec, P[i])[0], w[i]) for i in range(64)])
    pb = _pb(gpu, spec, dtype)
    ob = torch.tensor(obs, device="cuda", dtype=pb.torch_dtype)
    got = gpu.me_chi2(pb, ob, torch.tensor(P, device="cuda")).cpu().numpy()
    assert np.max(np.abs(got - ref) / ref) < 1e-12
    wu = np.abs(np.random.default_rng(4).standard_normal((64, 4))) + 0.5
    ref = np.array([orc.chi2(obs[i], orc.synth(spec, P[i])[0], wu[i]) for i in range(64)])
    got = gpu.me_chi2(pb, ob, torch.tensor(P, device="cuda"), w=torch.tensor(wu, device="cuda")).cpu().numpy()
    assert np.max(np.abs(got - ref) / ref) < 1e-12


def test_invalid_arguments_rejected(gpu):
    from paper_1208_0302_gb300 import _lib
    spec = gi.two_line_spec()
    bad = gi.ProblemSpec(lines=spec.lines, lambda_grid=np.linspace(6301, 6303, 600))
    pb = _pb(gpu, bad, "f32")
    with pytest.raises(_lib.GenesisError) as e:
        gpu.me_synth(pb, torch.zeros((2, 9), dtype=torch.float64, device="cuda"))
    assert e.value.code == _lib.ME_EINVAL
    pb = _pb(gpu, spec, "f32")
    obs = torch.zeros((4, 4, 128), device="cuda")
    with pytest.raises(_lib.GenesisError):
        gpu.ga_invert_batch(pb, obs, gi.PRIOR_LO, gi.PRIOR_HI, gpu.GaSettings(npop=48, ngen=2))
    lo = gi.PRIOR_LO.copy()
    lo[0] = 5000.0
    with pytest.raises(_lib.GenesisError):
        gpu.ga_invert_batch(pb, obs, lo, gi.PRIOR_HI, gpu.GaSettings(npop=64, ngen=2))
