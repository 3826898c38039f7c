"""Recovered parameters against the seeded truth (the served form: FP32 GA,
then the FP32 L-M polish, then the Section 6 uncertainties).

The data are the two-line setup with noise of 1e-3 I_c per sample, so the
sigma-weighted chi2 is about 1 at the truth.  Section 6 gives
sigma_i^2 = [H^-1]_ii chi2 / M with H = (2/nu) J^T W^2 J, the Hessian of
Eq. chisq; the least-squares covariance of the estimate is (J^T W^2 J)^-1, so
sigma_true^2 = sigma_i^2 2M / (nu chi2).  On pixels whose answer lies in the
global basin (chi2 < 1.5) and whose truth is well determined (B > 300 G, 15 <
theta < 165, every parameter at least 5 % of its range from the bounds) the
scaled errors |p - truth| / sigma_true follow |N(0, 1)|, whose median is
0.674; the paper's own sigma, larger by sqrt(nu chi2 / 2M), bounds the error.
"""
import numpy as np
import pytest
import torch

import genesis_inputs as gi
from gpu_helpers import make_obs

pytestmark = pytest.mark.gpu
NAMES = ["B", "theta", "chi", "v", "dlD", "a", "eta0", "S0", "S1"]


def test_recovery_against_seeded_truth(gpu, orc):
    spec = gi.two_line_spec()
    n = 4096
    truth, obs = make_obs(orc, spec, n, seed=80)
    obs32 = obs.astype(np.float32)
    sig = 1e-3 * (truth[:, 7] + truth[:, 8])
    w = torch.tensor(np.repeat((1 / sig)[:, None], 4, 1), device="cuda")
    pb = gpu.Problem.from_spec(spec, "f32")
    ob = torch.tensor(obs32, device="cuda")
    best, _ = gpu.ga_invert_batch(pb, ob, gi.PRIOR_LO, gi.PRIOR_HI, gpu.GaSettings(npop=128, ngen=200, seed=80))
    p, c2 = gpu.lm_polish(pb, ob, best, gi.PRIOR_LO, gi.PRIOR_HI, iters=10, w=w)
    s = gpu.lm_uncertainty(pb, ob, p, w=w)
    p, c2, s = p.cpu().numpy(), c2.cpu().numpy(), s.cpu().numpy()
    span = gi.PRIOR_HI - gi.PRIOR_LO
    inner = np.all((truth - gi.PRIOR_LO > 0.05 * span) & (gi.PRIOR_HI - truth > 0.05 * span), axis=1)
    well = (truth[:, 0] > 300) & (truth[:, 1] > 15) & (truth[:, 1] < 165) & inner
    good = well & (c2 < 1.5) & np.all(np.isfinite(s) & (s > 0), axis=1)
    # the GA lands in the global basin on nearly every well-determined pixel
    assert good.sum() >= 0.9 * well.sum() and good.sum() > 800, (good.sum(), well.sum())
    d = np.abs(p - truth)
    d[:, 2] = np.minimum(d[:, 2] % 180.0, 180.0 - d[:, 2] % 180.0)
    nu = 4 * spec.n_lambda - 9
    s_true = s * np.sqrt(2 * 9 / (nu * c2))[:, None]
    z = d[good] / s_true[good]
    med = np.median(z, axis=0)
    assert np.all((med > 0.5) & (med < 0.9)), dict(zip(NAMES, med.round(3)))
    # |N(0,1)| has 95 % of its mass below 1.96
    q95 = np.quantile(z, 0.95, axis=0)
    assert np.all(q95 < 3.0), dict(zip(NAMES, q95.round(3)))
    # the paper's sigma bounds the error
    assert np.all(np.median(d[good] / s[good], axis=0) < 0.5)
