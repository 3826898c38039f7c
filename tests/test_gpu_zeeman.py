"""Full Zeeman pattern (Section 5; Fe I 6301.5 5P2-5D2) on the GPU against the
oracle: synthesis, Jacobian and whole FP64 GA runs."""
import numpy as np
import pytest
import torch

import genesis_inputs as gi
from gpu_helpers import make_obs, rel_err

pytestmark = pytest.mark.gpu

FULL_6301 = (gi.FE6301[0], 1.667, gi.eta_ratio_6301(), 2, 11 / 6, 2, 1.5)
FULL_6302 = (gi.FE6302[0], 2.5, 1.0, 1, 2.5, 0, 0.0)


def _spec(n=128):
    return gi.ProblemSpec(lines=[FULL_6301, (gi.FE6302[0], 2.5, 1.0)],
                          lambda_grid=np.linspace(6301.0, 6303.0, n))


@pytest.mark.parametrize("dtype,tol", [("f32", 2e-5), ("f64", 1e-12)])
def test_full_pattern_synthesis(gpu, orc, dtype, tol):
    for spec in [_spec(), gi.ProblemSpec(lines=[FULL_6301, FULL_6302], lambda_grid=np.linspace(6301, 6303, 77))]:
        P = gi.draw_params_uniform(200, seed=70)
        ref = orc.synth(spec, P)
        got = gpu.me_synth(gpu.Problem.from_spec(spec, dtype), torch.tensor(P, device="cuda"))
        got = got.double().cpu().numpy()
        ic = P[:, 7] + P[:, 8]
        if dtype == "f32":
            assert rel_err(got, ref, ic) < tol
        else:
            assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), ic[:, None, None])) < tol


def test_full_pattern_jacobian(gpu, orc):
    spec = _spec(64)
    P = gi.draw_params_uniform(20, seed=71)
    P[:, 5] = np.maximum(P[:, 5], 0.02)
    jac = gpu.me_synth_jac(gpu.Problem.from_spec(spec, "f64"), torch.tensor(P, device="cuda")).cpu().numpy()
    for i in range(len(P)):
        ref = orc.jacobian(spec, P[i])
        scale = np.max(np.abs(ref), axis=(0, 1)) + 1e-30
        assert np.max(np.abs(jac[i] - ref) / scale) < 1e-7


def test_full_pattern_ga_fp64_matches_oracle(gpu, orc):
    spec = _spec()
    truth, obs = make_obs(orc, spec, 24, seed=72)
    ref = orc.ga_invert(spec, obs, gi.PRIOR_LO, gi.PRIOR_HI, orc.ga_config(64, 10, seed=7), pixel_id0=5,
                        want_margin=True)
    pb = gpu.Problem.from_spec(spec, "f64")
    best, chi2, genes = gpu.ga_invert_batch(pb, torch.tensor(obs, device="cuda"), gi.PRIOR_LO, gi.PRIOR_HI,
                                            gpu.GaSettings(npop=64, ngen=10, seed=7), pixel_id0=5,
                                            want_genes=True)
    safe = ref["margin"] > 1e-10
    assert safe.mean() > 0.8
    g = genes.cpu().numpy().view(np.uint16)
    assert (g[safe] == ref["genes"][safe]).all()
    assert np.max(np.abs(chi2.cpu().numpy()[safe] - ref["chi2"][safe]) / ref["chi2"][safe]) < 1e-12


def test_full_pattern_ga_fp32_and_polish(gpu, orc):
    spec = _spec()
    truth, obs = make_obs(orc, spec, 256, seed=73)
    pb = gpu.Problem.from_spec(spec, "f32")
    ob = torch.tensor(obs, device="cuda", dtype=torch.float32)
    sig = 1e-3 * (truth[:, 7] + truth[:, 8])
    w = torch.tensor(np.repeat((1 / sig)[:, None], 4, 1), device="cuda")
    best, _ = gpu.ga_invert_batch(pb, ob, gi.PRIOR_LO, gi.PRIOR_HI, gpu.GaSettings(npop=128, ngen=80, seed=3))
    c0 = gpu.me_chi2(pb, ob, best, w=w)
    p, c2 = gpu.lm_polish(pb, ob, best, gi.PRIOR_LO, gi.PRIOR_HI, iters=10, w=w)
    assert torch.all(c2 <= c0 * (1 + 1e-4))
    assert float(c2.median()) < 1.5
    counts = gpu.ga_count_evaluations(pb, ob[:32].contiguous(), gi.PRIOR_LO, gi.PRIOR_HI,
                                      gpu.GaSettings(npop=64, ngen=4, seed=3))
    # 12 components for 6301.5 + 3 for 6302.5 per wavelength point
    assert (counts["weideman"] + counts["mid"] + counts["cf"] + counts["even2"] + counts["far"] ==
            counts["points"] * 15)
    assert min(counts["weideman"], counts["mid"], counts["cf"], counts["even2"], counts["far"]) > 0
    # syntheses: the initial population, every child of every generation and
    # the restarted half at each generation t < ngen with t % nsamp == 0
    # (nsamp = ngen // 4 = 1 here, so t = 1, 2, 3)
    assert counts["syntheses"] == 32 * (64 * (4 + 1) + 3 * 32)
