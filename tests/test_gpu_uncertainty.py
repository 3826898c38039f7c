"""Section 6 uncertainties on the GPU against the oracle."""
import numpy as np
import pytest
import torch

import genesis_inputs as gi
from gpu_helpers import make_obs

pytestmark = pytest.mark.gpu


def test_uncertainty_matches_oracle(gpu, orc):
    spec = gi.two_line_spec()
    truth, obs = make_obs(orc, spec, 32, seed=80)
    truth[:, 0] = np.maximum(truth[:, 0], 400.0)
    truth[:, 1] = np.clip(truth[:, 1], 20.0, 160.0)
    _, obs = make_obs(orc, spec, 32, seed=80, truth=truth)
    p, _ = orc.lm_polish(spec, obs, truth, gi.PRIOR_LO, gi.PRIOR_HI, iters=20)
    ref = orc.lm_uncertainty(spec, obs, p)
    for dtype, tol_med, tol_max in [("f64", 1e-7, 1e-5), ("f32", 2e-3, 0.2)]:
        pb = gpu.Problem.from_spec(spec, dtype)
        got = gpu.lm_uncertainty(pb, torch.tensor(obs, device="cuda", dtype=pb.torch_dtype),
                                 torch.tensor(p, device="cuda")).cpu().numpy()
        rel = np.abs(got / ref - 1)
        assert np.median(rel) < tol_med and np.max(rel) < tol_max, (dtype, np.median(rel), np.max(rel))


def test_uncertainty_singular_parameter_is_infinite(gpu):
    spec = gi.two_line_spec()
    pb = gpu.Problem.from_spec(spec, "f64")
    p = np.array([[0.0, 40.0, 30.0, 0.1, 30.0, 0.2, 5.0, 0.3, 0.7]])   # B = 0: theta, chi have no effect
    obs = gpu.me_synth(pb, torch.tensor(p, device="cuda"))
    sig = gpu.lm_uncertainty(pb, obs, torch.tensor(p, device="cuda")).cpu().numpy()[0]
    assert np.isinf(sig).any()
