"""GPU pixel selection, weak-field fallback, seeds, selection and the
seeded / polarity-restricted / subset GA against the oracle.

me_classify repeats the oracle's FP64 sums in the same order, so every
output but the angles (atan2) must be bit-identical; the angles agree to
1e-12 degree.  me_select must equal numpy's nonzero.  The seeded, polarity-
restricted GA is compared bit for bit in FP64 on the pixels whose decisions
the oracle separates by more than the FP64 evaluation error, with the seeds
and polarity taken from the oracle's classification as inputs to both sides.
"""
import numpy as np
import pytest
import torch

import genesis_inputs as gi
from gpu_helpers import make_obs

pytestmark = pytest.mark.gpu
QUIET, LINE, CORE = (0, 8), 1, (80, 110)
EXACT = ["flag", "polarity", "p", "sigma_p", "B_par", "B_perp", "B"]


def _mixed_map(orc, spec, npix, seed):
    truth = gi.draw_truth(npix, seed=seed)
    truth[::3, 0] = np.linspace(2.0, 30.0, len(truth[::3]))  # every third pixel near-field-free
    truth, obs = make_obs(orc, spec, npix, seed, truth=truth)
    return truth, obs


def _gpu_classify(gpu, spec, obs, dtype, thresh, quiet=QUIET, line=LINE, core=CORE, best=None):
    pb = gpu.Problem.from_spec(spec, dtype)
    ob = torch.tensor(obs, device="cuda", dtype=pb.torch_dtype)
    r = gpu.classify(pb, ob, thresh, quiet, line, core, best=best)
    w = r["weak"].cpu().numpy()
    return {"flag": r["flag"].cpu().numpy(), "polarity": r["polarity"].cpu().numpy(),
            "p": r["p"].cpu().numpy(), "sigma_p": r["sigma_p"].cpu().numpy(), "B": w[:, 0],
            "theta": w[:, 1], "chi": w[:, 2], "B_par": w[:, 3], "B_perp": w[:, 4],
            "seeds": r["seeds"].cpu().numpy()}


def _angle_diff(a, b):
    return np.abs((a - b + 90.0) % 180.0 - 90.0)


def _compare_classify(got, ref):
    for k in EXACT:
        assert np.array_equal(got[k], ref[k].astype(got[k].dtype)), k
    assert np.max(_angle_diff(got["chi"], ref["chi"])) < 1e-12
    assert np.max(np.abs(got["theta"] - ref["theta"])) < 1e-12
    assert np.array_equal(got["seeds"][:, :, 0], ref["seeds"][:, :, 0])
    assert np.max(np.abs(got["seeds"][:, :, 1] - ref["seeds"][:, :, 1])) < 1e-12
    assert np.max(_angle_diff(got["seeds"][:, :, 2], ref["seeds"][:, :, 2])) < 1e-12


@pytest.mark.parametrize("dtype,npix", [("f64", 37), ("f32", 37), ("f32", 1), ("f64", 130)])
def test_classify_matches_oracle(gpu, orc, dtype, npix):
    spec = gi.two_line_spec()
    _, obs = _mixed_map(orc, spec, npix, seed=npix)
    if dtype == "f32":
        obs = obs.astype(np.float32).astype(np.float64)
    for thresh in [1.0, 10.0, 60.0]:
        ref = orc.classify(spec, obs, thresh, QUIET, LINE, CORE)
        got = _gpu_classify(gpu, spec, obs, dtype, thresh)
        _compare_classify(got, ref)
    assert 0 < ref["flag"].sum() < npix or npix == 1


@pytest.mark.parametrize("quiet,line,core", [((0, 128), 0, (0, 127)), ((120, 128), 1, (95, 95)),
                                             ((3, 4), 0, (0, 1)), ((0, 64), 1, (126, 127))])
def test_classify_window_edges(gpu, orc, quiet, line, core):
    spec = gi.two_line_spec()
    _, obs = _mixed_map(orc, spec, 19, seed=5)
    ref = orc.classify(spec, obs, 3.0, quiet, line, core)
    got = _gpu_classify(gpu, spec, obs, "f64", 3.0, quiet, line, core)
    _compare_classify(got, ref)


def test_classify_writes_weak_field_rows(gpu, orc):
    spec = gi.two_line_spec()
    _, obs = _mixed_map(orc, spec, 48, seed=8)
    ref = orc.classify(spec, obs, 10.0, QUIET, LINE, CORE)
    best = torch.full((48, 9), -7.0, dtype=torch.float64, device="cuda")
    _gpu_classify(gpu, spec, obs, "f64", 10.0, best=best)
    b = best.cpu().numpy()
    lo = ref["flag"] == 0
    assert lo.any() and (~lo).any()
    assert np.all(b[~lo] == -7.0)
    assert np.array_equal(b[lo, 0], ref["B"][lo])
    assert np.max(np.abs(b[lo, 1] - ref["theta"][lo])) < 1e-12
    assert np.all(np.isnan(b[lo, 3:]))


def test_classify_rejects_bad_windows(gpu):
    spec = gi.two_line_spec()
    pb = gpu.Problem.from_spec(spec, "f32")
    ob = torch.zeros((4, 4, 128), dtype=torch.float32, device="cuda")
    for quiet, line, core in [((5, 5), 0, CORE), ((0, 129), 0, CORE), ((0, 8), 2, CORE), ((0, 8), 0, (10, 9)),
                              ((0, 8), 0, (0, 128)), ((-1, 8), 0, CORE)]:
        with pytest.raises(Exception):
            gpu.classify(pb, ob, 1.0, quiet, line, core)


@pytest.mark.parametrize("npix", [0, 1, 5, 2047, 2048, 2049, 70001])
def test_select_matches_nonzero(gpu, npix):
    rng = np.random.default_rng(npix)
    for kind in ["random", "ones", "zeros", "mixed_values"]:
        if kind == "random":
            f = (rng.random(npix) < 0.3).astype(np.int32)
        elif kind == "ones":
            f = np.ones(npix, dtype=np.int32)
        elif kind == "zeros":
            f = np.zeros(npix, dtype=np.int32)
        else:
            f = rng.integers(-1, 3, npix).astype(np.int32)
        ft = torch.tensor(f, device="cuda")
        for want in [1, 0]:
            idx, cnt = gpu.select(ft, want)
            n = int(cnt.item())
            ref = np.nonzero(f == want)[0]
            assert n == len(ref)
            assert np.array_equal(idx[:n].cpu().numpy(), ref)


def test_ga_subset_seeded_fp64_bit_exact(gpu, orc):
    """FP64 GA on a subset of a map with seeds and polarity: each pixel's
    result is the oracle's whole-map result for it (random streams keyed by
    the pixel number), and pixels outside the subset are untouched."""
    spec = gi.two_line_spec()
    npix, npop, ngen, pid0 = 30, 64, 16, 321
    _, obs = _mixed_map(orc, spec, npix, seed=12)
    cls = orc.classify(spec, obs, 10.0, QUIET, LINE, CORE)
    seeds, pol = cls["seeds"][:, :3].copy(), cls["polarity"]
    seeds[4, 1, 1] = np.nan  # a partial seed keeps the Sobol gene
    cfg = orc.ga_config(npop, ngen, seed=77)
    ref = orc.ga_invert(spec, obs, gi.PRIOR_LO, gi.PRIOR_HI, cfg, pixel_id0=pid0, want_margin=True,
                        seeds=seeds, polarity=pol)
    sub = np.array([0, 2, 3, 4, 7, 11, 12, 13, 20, 28, 29], dtype=np.int32)
    pb = gpu.Problem.from_spec(spec, "f64")
    ob = torch.tensor(obs, device="cuda")
    index = torch.full((npix,), -5, dtype=torch.int32, device="cuda")
    index[:len(sub)] = torch.tensor(sub, device="cuda")
    count = torch.tensor([len(sub)], dtype=torch.int32, device="cuda")
    best, chi2, genes = gpu.ga_invert_subset(
        pb, ob, gi.PRIOR_LO, gi.PRIOR_HI, gpu.GaSettings(npop=npop, ngen=ngen, seed=77), index=index,
        count=count, seeds=torch.tensor(seeds, device="cuda"), polarity=torch.tensor(pol, device="cuda"),
        pixel_id0=pid0, want_genes=True)
    best, chi2 = best.cpu().numpy(), chi2.cpu().numpy()
    genes = genes.cpu().numpy().view(np.uint16)
    safe = ref["margin"][sub] > 1e-10
    assert safe.mean() >= 0.8
    assert np.array_equal(genes[sub][safe], ref["genes"][sub][safe])
    assert np.array_equal(best[sub][safe], ref["best"][sub][safe])
    assert np.max(np.abs(chi2[sub][safe] / ref["chi2"][sub][safe] - 1)) < 1e-12
    out = np.setdiff1d(np.arange(npix), sub)
    assert np.all(np.isnan(best[out])) and np.all(np.isnan(chi2[out]))
    ok = pol[sub] != 0
    psi = best[sub][ok, 1]
    assert np.all(np.where(pol[sub][ok] > 0, psi <= 90.0, psi >= 90.0))


def test_ga_and_lm_subset_match_whole_map_fp32(gpu, orc):
    """FP32: without seeds, a subset run reproduces the whole-map run's rows
    bit for bit (GA and L-M), via the device-side count from me_select."""
    spec = gi.two_line_spec()
    npix = 40
    _, obs = make_obs(orc, spec, npix, seed=31)
    pb = gpu.Problem.from_spec(spec, "f32")
    ob = torch.tensor(obs, device="cuda", dtype=torch.float32)
    ga = gpu.GaSettings(npop=64, ngen=20, seed=3)
    full, fchi = gpu.ga_invert_batch(pb, ob, gi.PRIOR_LO, gi.PRIOR_HI, ga, pixel_id0=9)
    fpol, fpchi = gpu.lm_polish(pb, ob, full, gi.PRIOR_LO, gi.PRIOR_HI, iters=5)
    flag = torch.tensor((np.arange(npix) % 3 != 1).astype(np.int32), device="cuda")
    index, count = gpu.select(flag, 1)
    best, chi2 = gpu.ga_invert_subset(pb, ob, gi.PRIOR_LO, gi.PRIOR_HI, ga, index=index, count=count,
                                      pixel_id0=9)
    sel = np.nonzero(flag.cpu().numpy())[0]
    assert torch.equal(best[sel], full[sel]) and torch.equal(chi2[sel], fchi[sel])
    keep = best.clone()
    p2, c2 = gpu.lm_polish_subset(pb, ob, best, gi.PRIOR_LO, gi.PRIOR_HI, index=index, count=count, iters=5,
                                  chi2=chi2)
    assert torch.equal(p2[sel], fpol[sel]) and torch.equal(c2[sel], fpchi[sel])
    out = np.setdiff1d(np.arange(npix), sel)
    assert torch.all(torch.isnan(p2[out])) and torch.equal(keep[out].isnan(), p2[out].isnan())


def test_invert_map_pipeline(gpu, orc):
    """Section 2 pipeline: weak-field rows below the threshold, seeded GA +
    L-M above it; the composed call equals its steps run one by one."""
    spec = gi.two_line_spec()
    npix = 60
    truth, obs = _mixed_map(orc, spec, npix, seed=44)
    pb = gpu.Problem.from_spec(spec, "f32")
    ob = torch.tensor(obs, device="cuda", dtype=torch.float32)
    ga = gpu.GaSettings(npop=64, ngen=30, seed=5)
    r = gpu.invert_map(pb, ob, gi.PRIOR_LO, gi.PRIOR_HI, ga, 10.0, QUIET, LINE, CORE, nseed=4, polish_iters=5)
    ref = orc.classify(spec, obs.astype(np.float32).astype(np.float64), 10.0, QUIET, LINE, CORE)
    flag = r["flag"].cpu().numpy()
    assert np.array_equal(flag, ref["flag"])
    assert int(r["count"].item()) == int(flag.sum()) and 0 < flag.sum() < npix
    best = r["best"].cpu().numpy()
    lo = flag == 0
    assert np.array_equal(best[lo, 0], ref["B"][lo]) and np.all(np.isnan(best[lo, 3:]))
    assert np.all(np.isnan(r["chi2"].cpu().numpy()[lo]))
    # the same steps by hand
    b2 = torch.full((npix, 9), float("nan"), dtype=torch.float64, device="cuda")
    c2 = torch.full((npix,), float("nan"), dtype=torch.float64, device="cuda")
    cls = gpu.classify(pb, ob, 10.0, QUIET, LINE, CORE, best=b2)
    idx, cnt = gpu.select(cls["flag"], 1)
    gpu.ga_invert_subset(pb, ob, gi.PRIOR_LO, gi.PRIOR_HI, ga, index=idx, count=cnt,
                         seeds=cls["seeds"].contiguous(), polarity=cls["polarity"], best=b2, chi2=c2)
    gpu.lm_polish_subset(pb, ob, b2, gi.PRIOR_LO, gi.PRIOR_HI, index=idx, count=cnt, iters=5, chi2=c2)
    assert torch.equal(torch.nan_to_num(b2, 1e300), torch.nan_to_num(r["best"], 1e300))
    assert np.all(np.isfinite(r["chi2"].cpu().numpy()[~lo]))
