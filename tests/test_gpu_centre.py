"""Section 5.1 line centre on the GPU: bit-exact with the oracle."""
import numpy as np
import pytest
import torch

import genesis_inputs as gi
from gpu_helpers import make_obs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_line_centre_bit_exact(gpu, orc, dtype):
    spec = gi.two_line_spec()
    truth, obs = make_obs(orc, spec, 300, seed=91)
    if dtype == "f32":
        obs = obs.astype(np.float32).astype(np.float64)
    pb = gpu.Problem.from_spec(spec, dtype)
    ob = torch.tensor(obs, device="cuda", dtype=pb.torch_dtype)
    for W, lo, hi in [(6, 0, 1 << 30), (10, 70, 120), (3, 0, 40), (64, 0, 1 << 30)]:
        ref_c, ref_i = orc.line_centre(obs, spec.lambda_grid, W, lo, hi)
        lc, idx = gpu.line_centre(pb, ob, W, lo, hi)
        assert np.array_equal(idx.cpu().numpy(), ref_i)
        got = lc.cpu().numpy()
        assert np.array_equal(np.isnan(got), np.isnan(ref_c))
        ok = ~np.isnan(ref_c)
        assert np.array_equal(got[ok], ref_c[ok])
