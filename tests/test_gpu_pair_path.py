"""The GA's own FP32 evaluation (the packed pair path) against the FP64 oracle.

ga_invert_batch ranks individuals by Eq. chisq of the Section 5 synthesis
computed two wavelengths at a time, with w(z) from four regions chosen per
pair and voted across the warp.  These tests run that code on the GPU with the
GA's launch shape (a block per pixel, a thread per individual, partial warps
as in the restarts) and compare it with the oracle:

* w(z) itself (me_faddeeva_pairs), point by point, within the branch budget
  1.5e-7 absolute or the series' FP32 floor 1e-6 |w| (the larger), on warps
  wholly inside one region, warps straddling every threshold, pairs whose two
  points lie in different regions and a ragged last warp;
* the Stokes vectors behind the fitness (ga_fitness returns the weighted
  residuals w_s (O - S)), per sample within 2e-5 of max(|oracle|, I_c);
* the fitness value: against the FP64 sum of its own squared residuals within
  the bound of its Kahan-compensated FP32 sum, and against the oracle's chi2
  within the bound that the 2e-5 sample bar implies.
"""
import numpy as np
import pytest
import torch

import genesis_inputs as gi

pytestmark = pytest.mark.gpu

SAMPLE_TOL = 2e-5            # FP32 synthesis, of max(|oracle|, I_c) per sample
WZ_ABS = 1.5e-7              # branch budget of the pair path's convergents and far field
WZ_REL = 1.0e-6              # FP32 rounding floor of Weideman's series, relative to |w|
U32 = 2.0 ** -24
FULL_6301 = (gi.FE6301[0], 1.667, gi.eta_ratio_6301(), 2, 11 / 6, 2, 1.5)
THRESHOLDS = (21.0, 36.0, 80.0, 360.0)   # |z|^2 of the middle shell, 3rd convergent, outer shell, far field


# ------------------------------------------------------------------ w(z)
def _boundary_points(rng):
    """(x, a) points on both sides of every region threshold, a in [0, 0.5]."""
    xs, ys = [], []
    for a in [0.0, 1e-6, 1e-3, 0.05, 0.2, 0.37, 0.5]:
        for r2 in THRESHOLDS:
            x0 = np.sqrt(r2 - a * a)
            d = np.concatenate([-np.geomspace(1e-5, 2.0, 24), np.geomspace(1e-5, 2.0, 24)])
            xs.append(x0 + d)
            ys.append(np.full(d.size, a))
    x = np.concatenate(xs)
    y = np.concatenate(ys)
    return x * np.where(rng.random(x.size) < 0.5, -1.0, 1.0), y


def _wz_case(rng):
    """Pairs (x0, x1) with a common a, arranged so that warps are wholly in
    one region, straddle thresholds, or mix everything; n is ragged."""
    pairs, avals = [], []
    # 1. homogeneous warps just inside / just beyond each threshold
    for a in [0.0, 0.25, 0.5]:
        for r2 in THRESHOLDS:
            for side in (-1.0, 1.0):
                lo, hi = (r2 * 0.97, r2) if side < 0 else (r2 * 1.0000001, r2 * 1.03)
                z2 = rng.uniform(lo, hi, (32, 2))
                x = np.sqrt(np.maximum(z2 - a * a, 0.0)) * rng.choice([-1.0, 1.0], (32, 2))
                pairs.append(x)
                avals.append(np.full(32, a))
    # 2. pairs whose two points lie in different regions (warp of such pairs)
    for r2 in THRESHOLDS:
        a = rng.uniform(0, 0.5, 32)
        inner = np.sqrt(np.maximum(rng.uniform(0.5 * r2, r2, 32) - a * a, 0))
        outer = np.sqrt(rng.uniform(r2, 2.0 * r2, 32) - a * a)
        pairs.append(np.stack([inner, -outer], 1))
        avals.append(a)
    # 3. boundary points shuffled into mixed warps, and sorted by |z| (mostly one region per warp)
    bx, by = _boundary_points(rng)
    m = bx.size // 64 * 64          # whole warps of pairs
    order = rng.permutation(m)
    pairs.append(bx[order].reshape(-1, 2))
    avals.append(by[order][0::2])
    srt = np.argsort(bx[:m] ** 2 + by[:m] ** 2, kind="stable")
    pairs.append(bx[srt].reshape(-1, 2))
    avals.append(np.maximum(by[srt][0::2], by[srt][1::2]))
    # 4. the two-line grid's range of |v| (far wings up to about 75 Doppler widths)
    x = rng.uniform(-80, 80, (320, 2))
    pairs.append(x)
    avals.append(rng.uniform(0, 0.5, 320))
    # 5. a ragged tail: 13 lanes in the far field after a mixed warp
    pairs.append(np.concatenate([rng.uniform(-3, 3, (32, 2)), rng.uniform(25, 70, (13, 2))]))
    avals.append(rng.uniform(0, 0.5, 45))
    x = np.concatenate(pairs).astype(np.float32)
    a = np.concatenate(avals).astype(np.float32)
    assert x.shape[0] % 32 == 13
    return x, a


def _wz_tol(ref):
    return np.maximum(WZ_ABS, WZ_REL * np.abs(ref))


@pytest.mark.parametrize("mode", [0, 1])
def test_wz_pair_path_matches_oracle(gpu, orc, mode):
    """Each of the four formulas, chosen by the warp vote, within its budget
    for every point (the oracle is the Matta-Reichel FP64 evaluation)."""
    x, a = _wz_case(np.random.default_rng(40 + mode))
    got = gpu.faddeeva_pairs(torch.tensor(x, device="cuda"), torch.tensor(a, device="cuda"), mode=mode)
    got = got.cpu().numpy()
    ref = orc.faddeeva(x.astype(np.float64), np.repeat(a.astype(np.float64)[:, None], 2, 1))
    err = np.abs(got - ref)
    bad = err > _wz_tol(ref)
    assert not bad.any(), (x[bad.any(1)][:5], a[bad.any(1)][:5], err[bad][:5])
    # the region thresholds are exercised: points within 3% of each on both sides
    z2 = x.astype(np.float64) ** 2 + a[:, None].astype(np.float64) ** 2
    for r2 in THRESHOLDS:
        assert ((z2 > r2) & (z2 < 1.03 * r2)).sum() >= 32 and ((z2 <= r2) & (z2 > 0.97 * r2)).sum() >= 32


def test_wz_triplet_level_matches_oracle(gpu, orc):
    """Effective triplets: the whole-triplet votes (wholly far, wholly beyond
    the continued-fraction threshold, near a core) and the inside-out
    component tests, through the unit-strength profile sums."""
    rng = np.random.default_rng(44)
    n = 32 * 40 + 13
    a = rng.uniform(0, 0.5, n).astype(np.float32)
    vb = rng.uniform(0, 30, n)
    vb[: 32 * 8] = 0.0                               # field-free triplets
    vb[32 * 8: 32 * 12] = rng.uniform(0, 0.05, 128)  # tiny splitting
    v = rng.uniform(-80, 80, (n, 2))
    # warps whose triplets all sit just beyond (or just inside) t_ext, t_80 or
    # t_far + |v_B|
    for w, r2 in [(20, 36.0), (21, 360.0), (24, 80.0), (22, 36.0), (23, 360.0), (25, 80.0)]:
        s = slice(32 * w, 32 * w + 32)
        t = np.sqrt(np.maximum(r2 - a[s].astype(np.float64) ** 2, 0)) + vb[s]
        side = 1.0 if w in (20, 21, 24) else 0.995
        v[s] = (t * side)[:, None] * rng.uniform(1.0, 1.02, (32, 2)) * rng.choice([-1, 1], (32, 2))
    vb = vb.astype(np.float32)
    v = v.astype(np.float32)
    got = gpu.faddeeva_pairs(torch.tensor(v, device="cuda"), torch.tensor(a, device="cuda"), mode=2,
                             v_b=torch.tensor(vb, device="cuda")).cpu().numpy()
    a2 = np.repeat(a.astype(np.float64)[:, None], 2, 1)
    # the kernel forms x_b = v + v_B and x_r = v - v_B in FP32
    xb = (v + vb[:, None]).astype(np.float64)
    xr = (v - vb[:, None]).astype(np.float64)
    wb, wp, wr = orc.faddeeva(xb, a2), orc.faddeeva(v.astype(np.float64), a2), orc.faddeeva(xr, a2)
    cols = [(wp.real, _wz_tol(wp)), (wp.imag, _wz_tol(wp)),
            (wb.real + wr.real, _wz_tol(wb) + _wz_tol(wr)), (wb.imag + wr.imag, _wz_tol(wb) + _wz_tol(wr)),
            (wr.real - wb.real, _wz_tol(wb) + _wz_tol(wr)), (wr.imag - wb.imag, _wz_tol(wb) + _wz_tol(wr))]
    for c, (ref, tol) in enumerate(cols):
        err = np.abs(got[:, :, c] - ref)
        assert np.all(err <= tol * 1.01 + 1e-12), (c, float(np.max(err / tol)))


# ---------------------------------------------------------- fitness path
def _individuals(npix, npop, npar, seed, lo, hi):
    """Per-pixel populations that put warps in every region mix: uniform
    draws, a -> 0, a = 0.5, narrow lines far in the wings, half-and-half warps,
    identical individuals, field-free and longitudinal/transverse fields."""
    rng = np.random.default_rng(seed)
    P = lo + (hi - lo) * rng.random((npix, npop, npar))
    for p in range(npix):
        k = p % 8
        if k == 1:
            P[p, :, 5] = np.where(np.arange(npop) % 2, 0.0, 1e-6)
        elif k == 2:
            P[p, :, 5] = 0.5
        elif k == 3:
            P[p, :, 4] = 20.0
            P[p, :, 3] = rng.choice([-3.0, 3.0], npop)
        elif k == 4:
            half = (np.arange(npop) % 32) < 16
            P[p, half, 4], P[p, half, 5] = 20.0, 0.0
            P[p, ~half, 4], P[p, ~half, 5] = 50.0, 0.5
        elif k == 5:
            P[p, :] = P[p, 0]
        elif k == 6:
            P[p, :, 0] = np.where(np.arange(npop) % 3 == 0, 0.0, 3000.0)
            P[p, :, 1] = np.where(np.arange(npop) % 2 == 0, 0.0, 90.0)
        elif k == 7:
            P[p, :, 5] = 0.0
            P[p, :, 0] = 3000.0
            P[p, :, 4] = 20.0
    return P.astype(np.float32).astype(np.float64)   # representable in FP32, as the GA's decode


def _specs():
    two = gi.two_line_spec()
    three = gi.ProblemSpec(lines=[(gi.FE6301[0], 1.667, gi.eta_ratio_6301()), (gi.FE6302[0], 2.5, 1.0),
                                  (6302.2, 1.2, 0.4)], lambda_grid=np.linspace(6301.0, 6303.0, 96))
    pat = gi.ProblemSpec(lines=[FULL_6301, (gi.FE6302[0], 2.5, 1.0)], lambda_grid=two.lambda_grid)
    odd = gi.one_line_spec(n_lambda=47)
    fill = gi.ProblemSpec(two.lines, two.lambda_grid, two.lambda_dop, two.mu, fill=True)
    fill_pat = gi.ProblemSpec(pat.lines, gi.two_line_spec(n_lambda=63).lambda_grid, two.lambda_dop, two.mu, fill=True)
    return {"two": two, "three": three, "pattern": pat, "one_odd": odd, "fill": fill, "fill_pattern_odd": fill_pat}


def _run(gpu, orc, spec, npix, npop, nactive, seed, user_w, mu_px=None):
    npar = 10 if spec.fill else 9
    lo = gi.PRIOR_LO_FILL if spec.fill else gi.PRIOR_LO
    hi = gi.PRIOR_HI_FILL if spec.fill else gi.PRIOR_HI
    P = _individuals(npix, npop, npar, seed, lo, hi)
    truth = gi.draw_truth(npix, seed=seed + 1, lo=lo, hi=hi)
    mu = np.ones(npix) if mu_px is None else mu_px
    sig = 1e-3 * (truth[:, 7] + mu * truth[:, 8])
    obs = orc.synth(spec, truth, mu_px=mu_px) + sig[:, None, None] * gi.draw_noise(npix, spec.n_lambda, seed)
    obs32 = obs.astype(np.float32)
    w = np.repeat((1.0 / sig)[:, None], 4, 1) if user_w else None
    pb = gpu.Problem.from_spec(spec, "f32")
    fit, res = gpu.ga_fitness(pb, torch.tensor(obs32, device="cuda"), torch.tensor(P, device="cuda"),
                              nactive=nactive, w=None if w is None else torch.tensor(w, device="cuda"),
                              mu_px=None if mu_px is None else torch.tensor(mu_px, device="cuda"),
                              want_resid=True)
    fit = fit.cpu().numpy()
    res = res.double().cpu().numpy()
    act = P[:, :nactive]
    ref = orc.synth(spec, act.reshape(-1, npar), mu_px=None if mu_px is None else np.repeat(mu_px, nactive))
    ref = ref.reshape(npix, nactive, 4, spec.n_lambda)
    if w is not None:
        wk = w.astype(np.float32).astype(np.float64)          # the kernel's FP32 weights
    else:
        wk = orc.weights_invmax(obs32.astype(np.float64))     # within a few ulp of the kernel's
    return dict(P=P, obs32=obs32.astype(np.float64), w=w, wk=wk, fit=fit, res=res, ref=ref, mu=mu, npar=npar)


def _check_samples(r, nactive):
    gpu_st = r["obs32"][:, None] - r["res"][:, :nactive] / r["wk"][:, None, :, None]
    ic = (r["P"][:, :nactive, 7] + r["mu"][:, None] * r["P"][:, :nactive, 8])[:, :, None, None]
    err = np.abs(gpu_st - r["ref"]) / np.maximum(np.abs(r["ref"]), ic)
    assert np.all(np.isfinite(gpu_st))
    assert float(err.max()) < SAMPLE_TOL, float(err.max())
    # rows beyond nactive are untouched
    assert np.all(np.isnan(r["fit"][:, nactive:])) and np.all(np.isnan(r["res"][:, nactive:]))
    return float(err.max())


def _check_fitness(orc, r, nactive, nl):
    npar = r["npar"]
    nu = 4 * nl - npar
    res = r["res"][:, :nactive]
    fit = r["fit"][:, :nactive]
    w2 = r["wk"] ** 2
    own = np.einsum("pksj->pk", res ** 2) / nu
    # Kahan-compensated FP32 sum: each pair's four squares by FMA (3 roundings),
    # the compensated running total (2 units plus O(n u^2)), the two lanes and
    # the final scaling: 16 units of 2^-24 bound it, whatever the grid size
    bound_sum = 16 * U32
    assert np.all(np.abs(fit - own) <= bound_sum * own + 1e-30), float(np.max(np.abs(fit - own) / own))
    if r["w"] is None:
        bound_sum += 1e-6     # the kernel's FP32 inverse-max weights against the oracle's FP64 ones
    # against the oracle's chi2 at the same individuals: |dchi2| <= (1/nu)
    # sum w^2 (2 |r| e + e^2) with e = 2e-5 max(|S|, I_c) per sample
    ref = r["ref"]
    ic = (r["P"][:, :nactive, 7] + r["mu"][:, None] * r["P"][:, :nactive, 8])[:, :, None, None]
    e = SAMPLE_TOL * np.maximum(np.abs(ref), ic)
    rr = r["obs32"][:, None] - ref
    chi_ref = np.empty(fit.shape)
    wo = np.sqrt(w2)
    for p in range(fit.shape[0]):
        for k in range(nactive):
            chi_ref[p, k] = orc.chi2(r["obs32"][p], ref[p, k], wo[p], npar)
    bound = np.einsum("ps,pksj->pk", w2, (2 * np.abs(rr) + e) * e) / nu + bound_sum * chi_ref
    assert np.all(np.abs(fit - chi_ref) <= bound), float(np.max(np.abs(fit - chi_ref) / bound))


@pytest.mark.parametrize("name", ["two", "three", "pattern", "one_odd", "fill", "fill_pattern_odd"])
@pytest.mark.parametrize("user_w", [True, False])
def test_fitness_path_matches_oracle(gpu, orc, name, user_w):
    """Full warps of 64 individuals per pixel, every region mix."""
    spec = _specs()[name]
    r = _run(gpu, orc, spec, 8, 64, 64, seed=300 + len(name), user_w=user_w)
    _check_samples(r, 64)
    _check_fitness(orc, r, 64, spec.n_lambda)


@pytest.mark.parametrize("npop,nactive", [(32, 16), (64, 45), (128, 97)])
def test_fitness_path_partial_warps(gpu, orc, npop, nactive):
    """Divergent evaluation as in the GA's restarts: npop 32 evaluates 16
    lanes of one warp; ragged counts leave the last warp partial."""
    spec = gi.two_line_spec()
    r = _run(gpu, orc, spec, 8, npop, nactive, seed=400 + nactive, user_w=True)
    _check_samples(r, nactive)
    _check_fitness(orc, r, nactive, spec.n_lambda)


def test_fitness_path_large_population_and_mu(gpu, orc):
    """The npop > 256 instantiation, with a per-pixel mu."""
    spec = gi.two_line_spec()
    mu = np.linspace(0.1, 1.0, 8)
    r = _run(gpu, orc, spec, 8, 512, 512, seed=500, user_w=True, mu_px=mu)
    _check_samples(r, 512)
    _check_fitness(orc, r, 512, spec.n_lambda)


def test_fitness_path_fp64_matches_oracle(gpu, orc):
    """The FP64 GA's evaluation (Kahan-summed rows) at the 1e-12 bar."""
    spec = gi.two_line_spec()
    npix, npop = 4, 64
    P = _individuals(npix, npop, 9, 600, gi.PRIOR_LO, gi.PRIOR_HI)
    truth = gi.draw_truth(npix, seed=601)
    obs = orc.synth(spec, truth) + 1e-3 * gi.draw_noise(npix, spec.n_lambda, 601)
    pb = gpu.Problem.from_spec(spec, "f64")
    fit, res = gpu.ga_fitness(pb, torch.tensor(obs, device="cuda"), torch.tensor(P, device="cuda"), want_resid=True)
    fit = fit.cpu().numpy()
    res = res.cpu().numpy()
    ref = orc.synth(spec, P.reshape(-1, 9)).reshape(npix, npop, 4, spec.n_lambda)
    ic = (P[:, :, 7] + P[:, :, 8])[:, :, None, None]
    assert np.max(np.abs((obs[:, None] - res) - ref) / np.maximum(np.abs(ref), ic)) < 1e-12
    w = orc.weights_invmax(obs)
    for p in range(npix):
        for k in range(0, npop, 7):
            c = orc.chi2(obs[p], ref[p, k], w[p])
            assert abs(fit[p, k] - c) <= 1e-12 * c


def test_fitness_invalid_arguments(gpu):
    from paper_1208_0302_gb300 import _lib
    spec = gi.two_line_spec()
    pb = gpu.Problem.from_spec(spec, "f32")
    obs = torch.zeros((2, 4, 128), device="cuda")
    P = torch.zeros((2, 48, 9), dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.GenesisError) as e:
        gpu.ga_fitness(pb, obs, P)
    assert e.value.code == _lib.ME_EINVAL
    P = torch.zeros((2, 32, 9), dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.GenesisError):
        gpu.ga_fitness(pb, obs, P, nactive=33)
    x = torch.zeros((4, 2), device="cuda")
    with pytest.raises(_lib.GenesisError):
        gpu.faddeeva_pairs(x, torch.zeros(4, device="cuda"), mode=3)
