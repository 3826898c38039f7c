"""The larger workloads in the launch configuration the benchmark uses, checked
on properties that hold at any size and on samples the oracle can compute."""
import numpy as np
import pytest
import torch

import genesis_inputs as gi
import oracle as _oracle_mod  # noqa: F401  (built by the orc fixture)

pytestmark = pytest.mark.gpu


def _gpu_cube(gpu, pb, truth, seed, mu=None):
    tp = torch.tensor(truth, device="cuda")
    mp = None if mu is None else torch.tensor(mu, device="cuda")
    clean = gpu.me_synth(pb, tp, mp)
    g = torch.Generator(device="cuda").manual_seed(seed)
    icont = tp[:, 7] + (1.0 if mp is None else mp) * tp[:, 8]
    sig = 1e-3 * icont
    obs = (clean + sig.to(clean.dtype)[:, None, None] *
           torch.randn(clean.shape, generator=g, device="cuda", dtype=clean.dtype)).contiguous()
    w = (1.0 / sig)[:, None].repeat(1, 4).contiguous()
    return obs, w


def test_adjoint_against_central_differences_1000_vectors(gpu, orc):
    """Analytic Jacobians vs central differences of the FP64 oracle with a
    1e-4 relative step on 1000 random parameter vectors (seed 3), per column
    relative to its scale floored at 1e-3 I_c per unit of the parameter's prior
    range (columns that nearly vanish, e.g. d/dchi at B ~ 0, keep an absolute
    bar at the noise level).

    * The differences are a sound reference: they agree with the oracle's
      Richardson-extrapolated Jacobian to 1e-5 of the floored scale.
    * FP32: within 2e-4 for every vector with B >= 100 G.  Below 100 G the
      linear polarization scales as B^2 and the azimuth column,
      d(Q, U)/dchi = (pi / 90) (-U, Q), falls below the floor; 2e-4 of the
      floor would ask for Q and U to about 3e-8 I_c, under the FP32
      resolution of I_c itself (the FP32 Q and U in the line wings differ
      from the oracle's by about 1e-7 I_c).  Near the line cores the
      Jacobian forms T = P - (phi_b + phi_r) / 2 from a Taylor series in v_B
      rather than from the nearly cancelling profiles, so those vectors are
      held to 8e-4 (measured: 1.95e-4 at B >= 100 G, 6.2e-4 below, 8.9e-4
      before the series form; the median over vectors of their worst column
      is 5.1e-5).
    * FP64: within 2e-7 against the Richardson Jacobian (measured 6.9e-8)."""
    spec = gi.two_line_spec()
    P = gi.draw_params_uniform(1000, seed=3)
    P[:, 5] = np.maximum(P[:, 5], 1e-3)
    pt = torch.tensor(P, device="cuda")
    jac = gpu.me_synth_jac(gpu.Problem.from_spec(spec, "f32"), pt).double().cpu().numpy()
    jac64 = gpu.me_synth_jac(gpu.Problem.from_spec(spec, "f64"), pt).cpu().numpy()
    fd = np.empty((1000, 4, 128, 9))
    for k in range(9):
        h = 1e-4 * np.maximum(np.abs(P[:, k]), 1e-2)
        pp, pm = P.copy(), P.copy()
        pp[:, k] += h
        pm[:, k] -= h
        fd[..., k] = (orc.synth(spec, pp) - orc.synth(spec, pm)) / (2 * h[:, None, None])
    rich = np.stack([orc.jacobian(spec, P[i]) for i in range(1000)])
    ic = (P[:, 7] + P[:, 8])[:, None, None, None]
    floor = 1e-3 * ic / (gi.PRIOR_HI - gi.PRIOR_LO)[None, None, None, :]

    def err(a, ref):
        scale = np.maximum(np.max(np.abs(ref), axis=(1, 2), keepdims=True), floor)
        return (np.abs(a - ref) / scale).max(axis=(1, 2, 3))     # worst column of each vector

    assert err(fd, rich).max() < 1e-5
    e32 = err(jac, fd)
    strong = P[:, 0] >= 100.0
    assert e32[strong].max() < 2e-4, (float(e32[strong].max()), int(np.argmax(np.where(strong, e32, 0))))
    assert e32.max() < 8e-4, float(e32.max())
    assert np.median(e32) < 1e-4
    assert err(jac64, rich).max() < 2e-7


def test_float32_map_with_polish_at_full_size(gpu, orc):
    """512x512 float32 two-line map, FP32 GA + 10 L-M, in one launch each;
    on a sample of pixels the oracle recomputes the reported FP64 chi2 of the
    output parameters one by one."""
    spec = gi.two_line_spec()
    pb = gpu.Problem.from_spec(spec, "f32")
    npix = 512 * 512
    truth = gi.draw_truth(npix, seed=3)
    obs, w = _gpu_cube(gpu, pb, truth, seed=33)
    ga = gpu.GaSettings(npop=128, ngen=200, seed=3)
    best, c_ga = gpu.ga_invert_batch(pb, obs, gi.PRIOR_LO, gi.PRIOR_HI, ga)
    c_ga_sigma = gpu.me_chi2(pb, obs, best, w=w)
    p, c2 = gpu.lm_polish(pb, obs, best, gi.PRIOR_LO, gi.PRIOR_HI, iters=10, w=w)
    torch.cuda.synchronize()
    pn = p.cpu().numpy()
    c2n = c2.cpu().numpy()
    assert np.all(np.isfinite(pn)) and np.all(np.isfinite(c2n))
    assert np.all(pn >= gi.PRIOR_LO) and np.all(pn <= gi.PRIOR_HI)
    # the polish never raises chi2 beyond FP32 evaluation noise
    assert np.all(c2n <= c_ga_sigma.cpu().numpy() * (1 + 1e-4))
    # chi2 output is the FP64 chi2 of the output parameters
    assert torch.equal(c2, gpu.me_chi2(pb, obs, p, w=w))
    med = float(np.median(c2n))
    assert 0.9 < med < 1.3, med
    # sampled parity: the oracle's FP64 chi2 of the GPU's answers
    idx = np.random.default_rng(12).choice(npix, 16, replace=False)
    idx[-1] = npix - 1
    o_s = obs[idx].double().cpu().numpy()
    w_s = w[idx].cpu().numpy()
    for k, i in enumerate(idx):
        ref = orc.chi2(o_s[k], orc.synth(spec, pn[i])[0], w_s[k])
        assert abs(c2n[i] / ref - 1) < 1e-10, (i, c2n[i], ref)
    # batch invariance at full size: a sampled slice run on its own
    for a in [0, 131072, npix - 300]:
        b2, _ = gpu.ga_invert_batch(pb, obs[a:a + 300].contiguous(), gi.PRIOR_LO, gi.PRIOR_HI, ga,
                                    pixel_id0=a)
        assert torch.equal(b2, best[a:a + 300])
    del obs, w, best, p
    torch.cuda.empty_cache()


def test_full_disc_sample_with_mu(gpu, orc):
    """Full-disc pixels with per-pixel mu: FP64 GA bit-exact with the oracle on
    a sample, FP32 GA + polish consistent on a larger sample."""
    truth, mu, _ = gi.draw_full_disc(n=2048, seed=5)
    rng = np.random.default_rng(8)
    idx = rng.choice(len(mu), 24, replace=False)
    spec = gi.two_line_spec()
    lo = gi.PRIOR_LO.copy()
    lo[7] = lo[8] = 0.05
    t, m = truth[idx], mu[idx]
    clean = orc.synth(spec, t, mu_px=m)
    ic = t[:, 7] + m * t[:, 8]
    obs = clean + 1e-3 * ic[:, None, None] * gi.draw_noise(len(idx), 128, seed=9)
    cfg = orc.ga_config(64, 12, seed=5)
    ref = orc.ga_invert(spec, obs, lo, gi.PRIOR_HI, cfg, mu_px=m, pixel_id0=777,
                        want_margin=True)
    pb64 = gpu.Problem.from_spec(spec, "f64")
    best, chi2, genes = gpu.ga_invert_batch(pb64, torch.tensor(obs, device="cuda"), lo, gi.PRIOR_HI,
                                            gpu.GaSettings(npop=64, ngen=12, seed=5),
                                            mu_px=torch.tensor(m, device="cuda"), pixel_id0=777,
                                            want_genes=True)
    safe = ref["margin"] > 1e-10
    assert safe.mean() > 0.8
    g = genes.cpu().numpy().view(np.uint16)
    assert (g[safe] == ref["genes"][safe]).all()
    assert np.max(np.abs(chi2.cpu().numpy()[safe] - ref["chi2"][safe]) / ref["chi2"][safe]) < 1e-12
    # FP32 path on 4096 disc pixels
    idx = rng.choice(len(mu), 4096, replace=False)
    pb = gpu.Problem.from_spec(spec, "f32")
    obs32, w = _gpu_cube(gpu, pb, truth[idx], seed=10, mu=mu[idx])
    mp = torch.tensor(mu[idx], device="cuda")
    best, _ = gpu.ga_invert_batch(pb, obs32, lo, gi.PRIOR_HI, gpu.GaSettings(npop=128, ngen=60, seed=5),
                                  mu_px=mp)
    p, c2 = gpu.lm_polish(pb, obs32, best, lo, gi.PRIOR_HI, iters=10, w=w, mu_px=mp)
    assert torch.equal(c2, gpu.me_chi2(pb, obs32, p, w=w, mu_px=mp))
    assert float(c2.median()) < 1.5
