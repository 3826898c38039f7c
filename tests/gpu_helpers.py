"""Helpers shared by the GPU parity tests: oracle-made observations."""
import numpy as np

import genesis_inputs as gi


def make_obs(orc, spec, npix, seed, noise=True, truth=None, mu_px=None):
    """Truth, observed cube [npix, 4, n_lambda] (oracle synthesis + noise)."""
    if truth is None:
        truth = gi.draw_truth(npix, seed=seed)
    clean = orc.synth(spec, truth, mu_px=mu_px)
    if not noise:
        return truth, clean
    mu = np.ones(npix) if mu_px is None else mu_px
    sig = 1e-3 * (truth[:, 7] + mu * truth[:, 8])
    return truth, clean + sig[:, None, None] * gi.draw_noise(npix, spec.n_lambda, seed=seed)


def rel_err(gpu, ref, ic):
    """max |gpu - ref| / max(|ref|, I_c) per sample."""
    scale = np.maximum(np.abs(ref), ic[:, None, None])
    return float(np.max(np.abs(gpu - ref) / scale))
