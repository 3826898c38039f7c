"""Torch-facing calls of the GENESIS GB300 library.

Each function marshals CUDA tensors into the C ABI of ``include/genesis.h``
and enqueues the work on torch's current CUDA stream.  No computation of the
method happens here; PyTorch provides device memory and streams only.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L

NPAR = L.ME_NPAR          # parameters without the fill fraction
NPAR_MAX = L.ME_NPAR_MAX  # with it (Section 5.2): Problem(fill=True)
F32, F64 = L.ME_F32, L.ME_F64
ALL_FREE = (1 << NPAR_MAX) - 1


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def _need(t, dtype, shape=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


class Problem:
    """Line list, wavelength grid and precision (me_problem)."""

    def __init__(self, lines, lambda_grid, lambda_dop, mu=1.0, dtype="f32", fill=False):
        self.lines = [tuple(map(float, ln)) for ln in lines]
        self.fill = bool(fill)
        self.npar = NPAR + (1 if self.fill else 0)
        self.lam = np.ascontiguousarray(lambda_grid, dtype=np.float64)
        self.lambda_dop = float(lambda_dop)
        self.mu = float(mu)
        self.dtype = {"f32": F32, "f64": F64}[dtype]
        self.torch_dtype = torch.float32 if self.dtype == F32 else torch.float64
        s = L.MeProblem()
        s.n_lines = len(self.lines)
        for i, ln in enumerate(self.lines):
            # (lambda0, g_eff, eta_ratio) or, for a full Zeeman pattern,
            # (lambda0, g_eff, eta_ratio, j_lower, g_lower, j_upper, g_upper)
            if len(ln) > 3:
                s.line[i] = L.MeLine(ln[0], ln[1], ln[2], 1, int(ln[3]), int(ln[5]), ln[4], ln[6])
            else:
                s.line[i] = L.MeLine(ln[0], ln[1], ln[2], 0, 0, 0, 0.0, 0.0)
        s.n_lambda = len(self.lam)
        s.lambda_A = self.lam.ctypes.data_as(C.POINTER(C.c_double))
        s.lambda_dop_A = self.lambda_dop
        s.mu = self.mu
        s.dtype = self.dtype
        s.fill_fraction = 1 if self.fill else 0
        self._s = s

    @classmethod
    def from_spec(cls, spec, dtype="f32"):
        return cls(spec.lines, spec.lambda_grid, spec.lambda_dop, spec.mu, dtype, getattr(spec, "fill", False))

    @property
    def n_lambda(self):
        return len(self.lam)

    def ref(self):
        return C.byref(self._s)


def bounds(lo, hi) -> L.MeBounds:
    """me_bounds from 9 or 10 lower/upper values (a missing alpha row is [0, 1])."""
    if len(lo) not in (NPAR, NPAR_MAX) or len(hi) != len(lo):
        raise ValueError("bounds need 9 or 10 entries")
    b = L.MeBounds()
    for d in range(NPAR_MAX):
        b.lo[d] = float(lo[d]) if d < len(lo) else 0.0
        b.hi[d] = float(hi[d]) if d < len(hi) else 1.0
    return b


@dataclass
class GaSettings:
    npop: int = 128
    ngen: int = 200
    nsamp: int | None = None
    pc: float = 0.9
    pmut_lsb: float = 0.05
    pmut_ratio: float = 0.7
    seed: int = 0

    def to_c(self, weight_mode: int) -> L.GaConfig:
        nsamp = self.ngen // 4 if self.nsamp is None else self.nsamp
        return L.GaConfig(int(self.npop), int(self.ngen), int(nsamp), float(self.pc),
                          float(self.pmut_lsb), float(self.pmut_ratio), int(self.seed),
                          int(weight_mode))


def me_synth(pb: Problem, params, mu_px=None):
    """Stokes [n, 4, n_lambda] of params [n, 9] (float64 CUDA)."""
    n = params.shape[0]
    _need(params, torch.float64, (n, pb.npar), "params")
    _need(mu_px, torch.float64, (n,), "mu_px")
    out = torch.empty((n, 4, pb.n_lambda), dtype=pb.torch_dtype, device=params.device)
    L.check(L.load().me_synth(pb.ref(), _ptr(params), _ptr(mu_px), n, _ptr(out), _stream()))
    return out


def me_synth_jac(pb: Problem, params, mu_px=None, want_stokes=False):
    """Jacobian [n, 4, n_lambda, 9] (and Stokes if asked)."""
    n = params.shape[0]
    _need(params, torch.float64, (n, pb.npar), "params")
    _need(mu_px, torch.float64, (n,), "mu_px")
    jac = torch.empty((n, 4, pb.n_lambda, pb.npar), dtype=pb.torch_dtype, device=params.device)
    st = torch.empty((n, 4, pb.n_lambda), dtype=pb.torch_dtype, device=params.device) if want_stokes else None
    L.check(L.load().me_synth_jac(pb.ref(), _ptr(params), _ptr(mu_px), n, _ptr(st), _ptr(jac), _stream()))
    return (jac, st) if want_stokes else jac


def me_synth_vjp(pb: Problem, params, grad_stokes, mu_px=None):
    """J^T grad_stokes -> [n, 9] float64."""
    n = params.shape[0]
    _need(params, torch.float64, (n, pb.npar), "params")
    _need(grad_stokes, pb.torch_dtype, (n, 4, pb.n_lambda), "grad_stokes")
    _need(mu_px, torch.float64, (n,), "mu_px")
    out = torch.empty((n, pb.npar), dtype=torch.float64, device=params.device)
    L.check(L.load().me_synth_vjp(pb.ref(), _ptr(params), _ptr(mu_px), n, _ptr(grad_stokes),
                                  _ptr(out), _stream()))
    return out


def me_chi2(pb: Problem, obs, params, w=None, mu_px=None):
    """FP64 chi2 [npix] of params against obs (Eq. chisq)."""
    npix = obs.shape[0]
    _need(obs, pb.torch_dtype, (npix, 4, pb.n_lambda), "obs")
    _need(params, torch.float64, (npix, pb.npar), "params")
    _need(w, torch.float64, (npix, 4), "w")
    _need(mu_px, torch.float64, (npix,), "mu_px")
    out = torch.empty(npix, dtype=torch.float64, device=obs.device)
    L.check(L.load().me_chi2(pb.ref(), _ptr(obs), _ptr(w), _ptr(mu_px), npix, _ptr(params),
                             _ptr(out), _stream()))
    return out


def ga_invert_batch(pb: Problem, obs, lo, hi, ga: GaSettings, w=None, mu_px=None, pixel_id0=0,
                    want_genes=False):
    """Algorithm 1 per pixel on the GPU -> (best [npix, 9], chi2 [npix][, genes])."""
    npix = obs.shape[0]
    _need(obs, pb.torch_dtype, (npix, 4, pb.n_lambda), "obs")
    _need(w, torch.float64, (npix, 4), "w")
    _need(mu_px, torch.float64, (npix,), "mu_px")
    dev = obs.device
    best = torch.empty((npix, pb.npar), dtype=torch.float64, device=dev)
    chi2 = torch.empty(npix, dtype=torch.float64, device=dev)
    genes = torch.empty((npix, pb.npar), dtype=torch.int16, device=dev) if want_genes else None
    cfg = ga.to_c(L.ME_W_USER if w is not None else L.ME_W_INVMAX)
    b = bounds(lo, hi)
    L.check(L.load().ga_invert_batch(pb.ref(), _ptr(obs), _ptr(w), _ptr(mu_px), npix,
                                     int(pixel_id0), C.byref(b), C.byref(cfg), _ptr(best),
                                     _ptr(chi2), _ptr(genes), _stream()))
    if want_genes:
        return best, chi2, genes
    return best, chi2


def ga_count_evaluations(pb: Problem, obs, lo, hi, ga: GaSettings, w=None, mu_px=None, pixel_id0=0):
    """Work counts of one ga_invert_batch run (same arithmetic, counting build)."""
    npix = obs.shape[0]
    _need(obs, pb.torch_dtype, (npix, 4, pb.n_lambda), "obs")
    _need(w, torch.float64, (npix, 4), "w")
    _need(mu_px, torch.float64, (npix,), "mu_px")
    best = torch.empty((npix, pb.npar), dtype=torch.float64, device=obs.device)
    counts = torch.zeros(6, dtype=torch.int64, device=obs.device)
    cfg = ga.to_c(L.ME_W_USER if w is not None else L.ME_W_INVMAX)
    b = bounds(lo, hi)
    L.check(L.load().ga_count_evaluations(pb.ref(), _ptr(obs), _ptr(w), _ptr(mu_px), npix,
                                          int(pixel_id0), C.byref(b), C.byref(cfg), _ptr(best),
                                          _ptr(counts), _stream()))
    c = counts.cpu().numpy()
    syn = int(c[0])
    points = syn * pb.n_lambda
    return {"syntheses": syn, "points": points, "weideman": int(c[1]), "mid": int(c[4]), "far": int(c[3]),
            "even2": int(c[5]), "cf": int(c[2]) - int(c[1]) - int(c[3]) - int(c[4]) - int(c[5]), "best": best}


def ga_fitness(pb: Problem, obs, params, nactive=None, w=None, mu_px=None, want_resid=False):
    """The GA's fitness of individuals params [npix, npop, M] (float64 CUDA,
    each value representable in the problem's precision): (fitness [npix,
    npop] float64, residuals [npix, npop, 4, n_lambda] or None).  Threads
    k < nactive evaluate (default: all); rows beyond are NaN."""
    npix, npop = params.shape[0], params.shape[1]
    _need(obs, pb.torch_dtype, (npix, 4, pb.n_lambda), "obs")
    _need(params, torch.float64, (npix, npop, pb.npar), "params")
    _need(w, torch.float64, (npix, 4), "w")
    _need(mu_px, torch.float64, (npix,), "mu_px")
    nactive = npop if nactive is None else int(nactive)
    fit = torch.full((npix, npop), float("nan"), dtype=torch.float64, device=params.device)
    res = (torch.full((npix, npop, 4, pb.n_lambda), float("nan"), dtype=pb.torch_dtype, device=params.device)
           if want_resid else None)
    L.check(L.load().ga_fitness(pb.ref(), _ptr(obs), _ptr(w), _ptr(mu_px), npix, npop, nactive, _ptr(params),
                                _ptr(fit), _ptr(res), _stream()))
    return fit, res


def faddeeva_pairs(x, a, mode=0, v_b=None):
    """The pair path's FP32 w(z): x [n, 2] float32 CUDA, a [n] (and v_b [n]
    for mode 2).  Modes 0 and 1: complex [n, 2]; mode 2: float [n, 2, 6]
    profile sums (see include/genesis.h)."""
    n = x.shape[0]
    _need(x, torch.float32, (n, 2), "x")
    _need(a, torch.float32, (n,), "a")
    _need(v_b, torch.float32, (n,), "v_b")
    out = torch.empty((n, 2, 6 if mode == 2 else 2), dtype=torch.float32, device=x.device)
    L.check(L.load().me_faddeeva_pairs(_ptr(x), _ptr(a), _ptr(v_b), n, int(mode), _ptr(out), _stream()))
    if mode == 2:
        return out
    return torch.complex(out[..., 0].double(), out[..., 1].double())


def zeeman_components(line):
    """The library's Zeeman components of one line tuple (see Problem): list
    of (shifts, strengths) for sigma_b, pi, sigma_r."""
    if len(line) > 3:
        ml = L.MeLine(line[0], line[1], line[2], 1, int(line[3]), int(line[5]), line[4], line[6])
    else:
        ml = L.MeLine(line[0], line[1], line[2], 0, 0, 0, 0.0, 0.0)
    n = np.zeros(3, dtype=np.int32)
    sh = np.zeros((3, L.ME_MAX_COMP))
    st = np.zeros((3, L.ME_MAX_COMP))
    L.check(L.load().me_zeeman_components(C.byref(ml), n.ctypes.data, sh.ctypes.data, st.ctypes.data))
    return [(sh[g, :n[g]].copy(), st[g, :n[g]].copy()) for g in range(3)]


def lm_polish(pb: Problem, obs, params, lo, hi, iters=10, lambda0=1e-3, w=None, mu_px=None):
    """L-M refinement; returns (params [npix, 9], chi2 [npix]) (params updated in a copy)."""
    npix = obs.shape[0]
    _need(obs, pb.torch_dtype, (npix, 4, pb.n_lambda), "obs")
    _need(params, torch.float64, (npix, pb.npar), "params")
    _need(w, torch.float64, (npix, 4), "w")
    _need(mu_px, torch.float64, (npix,), "mu_px")
    p = params.clone()
    chi2 = torch.empty(npix, dtype=torch.float64, device=obs.device)
    b = bounds(lo, hi)
    L.check(L.load().lm_polish(pb.ref(), _ptr(obs), _ptr(w), _ptr(mu_px), npix, C.byref(b),
                               int(iters), float(lambda0), _ptr(p), _ptr(chi2), _stream()))
    return p, chi2


def lm_uncertainty(pb: Problem, obs, params, w=None, mu_px=None):
    """Section 6 sigma_i = sqrt([H^-1]_ii chi2 / M), H = (2/nu) J^T W^2 J -> [npix, 9]."""
    npix = obs.shape[0]
    _need(obs, pb.torch_dtype, (npix, 4, pb.n_lambda), "obs")
    _need(params, torch.float64, (npix, pb.npar), "params")
    _need(w, torch.float64, (npix, 4), "w")
    _need(mu_px, torch.float64, (npix,), "mu_px")
    out = torch.empty((npix, pb.npar), dtype=torch.float64, device=obs.device)
    L.check(L.load().lm_uncertainty(pb.ref(), _ptr(obs), _ptr(w), _ptr(mu_px), npix, _ptr(params),
                                    _ptr(out), _stream()))
    return out


def line_centre(pb: Problem, obs, half_width, i_lo=0, i_hi=1 << 30):
    """Section 5.1 centre-of-symmetry line centre -> (lambda_c [npix] f64, index [npix] i32)."""
    npix = obs.shape[0]
    _need(obs, pb.torch_dtype, (npix, 4, pb.n_lambda), "obs")
    lc = torch.empty(npix, dtype=torch.float64, device=obs.device)
    idx = torch.empty(npix, dtype=torch.int32, device=obs.device)
    L.check(L.load().me_line_centre(pb.ref(), _ptr(obs), npix, int(half_width), int(i_lo), int(i_hi),
                                    _ptr(lc), _ptr(idx), _stream()))
    return lc, idx


# ------------------------------------------------- selection and seeding

def classify(pb: Problem, obs, p_thresh, quiet, line, core, best=None):
    """Section 2 selection, weak-field fallback and Section 5.5 seeds.
    quiet = (lo, hi) half-open quiet window, core = (lo, hi) inclusive line
    window (grid indices).  Returns dict of device tensors: flag, polarity
    (int32 [npix]), p, sigma_p (f64 [npix]), weak (f64 [npix, 5] = B, theta,
    chi, B_par, B_perp) and seeds (f64 [npix, 4, 3]).  If best (f64 [npix, 9])
    is given, the rows of pixels below the threshold receive the weak-field
    answer (B, theta, chi, NaN...)."""
    npix = obs.shape[0]
    _need(obs, pb.torch_dtype, (npix, 4, pb.n_lambda), "obs")
    _need(best, torch.float64, (npix, pb.npar), "best")
    dev = obs.device
    flag = torch.empty(npix, dtype=torch.int32, device=dev)
    polarity = torch.empty(npix, dtype=torch.int32, device=dev)
    pol = torch.empty((npix, 2), dtype=torch.float64, device=dev)
    weak = torch.empty((npix, 5), dtype=torch.float64, device=dev)
    seeds = torch.empty((npix, 4, 3), dtype=torch.float64, device=dev)
    L.check(L.load().me_classify(pb.ref(), _ptr(obs), npix, float(p_thresh), int(quiet[0]), int(quiet[1]),
                                 int(line), int(core[0]), int(core[1]), _ptr(flag), _ptr(polarity), _ptr(pol),
                                 _ptr(weak), _ptr(seeds), _ptr(best), _stream()))
    return {"flag": flag, "polarity": polarity, "p": pol[:, 0], "sigma_p": pol[:, 1], "weak": weak,
            "seeds": seeds}


def select(flag, want=1):
    """Pixels with flag == want, in increasing order -> (index int32 [npix],
    count int32 [1]); both stay on the device."""
    npix = flag.shape[0]
    _need(flag, torch.int32, (npix,), "flag")
    lib = L.load()
    index = torch.empty(max(npix, 1), dtype=torch.int32, device=flag.device)
    count = torch.empty(1, dtype=torch.int32, device=flag.device)
    nbytes = int(lib.me_select_scratch_bytes(npix))
    scratch = torch.empty(max(nbytes, 4), dtype=torch.uint8, device=flag.device)
    L.check(lib.me_select(_ptr(flag), npix, int(want), _ptr(index), _ptr(count), _ptr(scratch), nbytes,
                          _stream()))
    return index[:npix], count


def select_static(flag, want=1):
    """select() through me_select_static: no scratch, no allocation in the
    library (the shared tile array limits npix to ME_SELECT_STATIC_MAX_PIX;
    overlapping calls race)."""
    npix = flag.shape[0]
    _need(flag, torch.int32, (npix,), "flag")
    index = torch.empty(max(npix, 1), dtype=torch.int32, device=flag.device)
    count = torch.empty(1, dtype=torch.int32, device=flag.device)
    L.check(L.load().me_select_static(_ptr(flag), npix, int(want), _ptr(index), _ptr(count), _stream()))
    return index[:npix], count


def ga_invert_subset(pb: Problem, obs, lo, hi, ga: GaSettings, index=None, count=None, seeds=None,
                     polarity=None, bounds_px=None, w=None, mu_px=None, pixel_id0=0, best=None, chi2=None,
                     want_genes=False):
    """ga_invert_batch on the pixels index[:count] of a map, seeded and
    polarity-restricted (Section 5.5), optionally in per-pixel bounds
    (Section 5.3).  best/chi2 (map-sized) are written in place for those
    pixels and returned."""
    npix = obs.shape[0]
    _need(obs, pb.torch_dtype, (npix, 4, pb.n_lambda), "obs")
    _need(w, torch.float64, (npix, 4), "w")
    _need(mu_px, torch.float64, (npix,), "mu_px")
    _need(index, torch.int32, None, "index")
    _need(count, torch.int32, (1,), "count")
    _need(polarity, torch.int32, (npix,), "polarity")
    _need(bounds_px, torch.float64, (npix, 2, pb.npar), "bounds_px")
    nseed = 0
    if seeds is not None:
        _need(seeds, torch.float64, None, "seeds")
        if seeds.dim() != 3 or seeds.shape[0] != npix or seeds.shape[2] != 3:
            raise ValueError("seeds must have shape (npix, nseed, 3)")
        nseed = seeds.shape[1]
    if index is not None and count is None and index.shape[0] != npix:
        raise ValueError("an index without count must hold npix entries")
    if index is not None and index.shape[0] < npix and count is not None:
        raise ValueError("index must hold npix entries")
    dev = obs.device
    if best is None:
        best = torch.full((npix, pb.npar), float("nan"), dtype=torch.float64, device=dev)
    if chi2 is None:
        chi2 = torch.full((npix,), float("nan"), dtype=torch.float64, device=dev)
    _need(best, torch.float64, (npix, pb.npar), "best")
    _need(chi2, torch.float64, (npix,), "chi2")
    genes = torch.zeros((npix, pb.npar), dtype=torch.int16, device=dev) if want_genes else None
    cfg = ga.to_c(L.ME_W_USER if w is not None else L.ME_W_INVMAX)
    b = bounds(lo, hi)
    L.check(L.load().ga_invert_subset(pb.ref(), _ptr(obs), _ptr(w), _ptr(mu_px), npix, int(pixel_id0),
                                      C.byref(b), C.byref(cfg), _ptr(seeds), nseed, _ptr(polarity),
                                      _ptr(bounds_px), _ptr(index), _ptr(count), _ptr(best), _ptr(chi2),
                                      _ptr(genes), _stream()))
    if want_genes:
        return best, chi2, genes
    return best, chi2


def lm_fit(pb: Problem, obs, params, lo, hi, index=None, count=None, iters=10, lambda0=1e-3, w=None,
           mu_px=None, chi2=None, free_mask=ALL_FREE):
    """L-M on the pixels index[:count] of a map with the parameters outside
    free_mask held; params (map-sized) and chi2 are updated in place for
    those pixels and returned."""
    npix = obs.shape[0]
    _need(obs, pb.torch_dtype, (npix, 4, pb.n_lambda), "obs")
    _need(params, torch.float64, (npix, pb.npar), "params")
    _need(w, torch.float64, (npix, 4), "w")
    _need(mu_px, torch.float64, (npix,), "mu_px")
    _need(index, torch.int32, None, "index")
    _need(count, torch.int32, (1,), "count")
    if index is not None and index.shape[0] < npix:
        raise ValueError("index must hold npix entries")
    _need(chi2, torch.float64, (npix,), "chi2")
    b = bounds(lo, hi)
    L.check(L.load().lm_fit(pb.ref(), _ptr(obs), _ptr(w), _ptr(mu_px), npix, C.byref(b), int(iters),
                            float(lambda0), int(free_mask), _ptr(index), _ptr(count), _ptr(params), _ptr(chi2),
                            _stream()))
    return params, chi2


def lm_polish_subset(pb: Problem, obs, params, lo, hi, index=None, count=None, iters=10, lambda0=1e-3,
                     w=None, mu_px=None, chi2=None):
    """lm_fit with every parameter free."""
    return lm_fit(pb, obs, params, lo, hi, index=index, count=count, iters=iters, lambda0=lambda0, w=w,
                  mu_px=mu_px, chi2=chi2)


# Section 5.3 prefit: Stokes I, non-magnetic (B, theta, chi held at 0, 90, 0)
PREFIT_MASK = 0x1F8
PREFIT_START = (0.0, 90.0, 0.0, 0.0, 35.0, 0.2, 5.0, 0.3, 0.7)
# margins of the bound rule (B theta chi v dlD a eta0 S0 S1): Zeeman broadening
# only widens the profile, so the non-magnetic fit bounds the Doppler width
# and damping from above and the line strength from below
PREFIT_LOWER = (float("inf"),) * 3 + (1.0, float("inf"), float("inf"), 3.0, 0.15, 0.15)
PREFIT_UPPER = (float("inf"),) * 3 + (1.0, 3.0, 0.15, float("inf"), 0.15, 0.15)


def thermo_prefit(pb: Problem, obs, lo, hi, index=None, count=None, iters=40, lambda0=1e-3, mu_px=None,
                  start=PREFIT_START):
    """Section 5.3 thermodynamic prefit: L-M fit of Stokes I alone with the
    field held at zero, from a generic start -> (params [npix, M], chi2).
    With the fill fraction, alpha is held at 1 (at B = 0 it has no effect)."""
    npix = obs.shape[0]
    dev = obs.device
    start = tuple(start) + ((1.0,) if pb.fill and len(start) == NPAR else ())
    params = torch.tensor(start, dtype=torch.float64, device=dev).repeat(npix, 1).contiguous()
    w = torch.zeros((npix, 4), dtype=torch.float64, device=dev)
    w[:, 0] = 1.0
    chi2 = torch.full((npix,), float("nan"), dtype=torch.float64, device=dev)
    return lm_fit(pb, obs, params, lo, hi, index=index, count=count, iters=iters, lambda0=lambda0, w=w,
                  mu_px=mu_px, chi2=chi2, free_mask=PREFIT_MASK)


def prefit_bounds(p_hat, lo, hi, lower=PREFIT_LOWER, upper=PREFIT_UPPER):
    """Per-pixel search bounds [npix, 2, M] around a prefit (me_prefit_bounds);
    M = p_hat's columns (a 10th margin defaults to infinite: alpha unbounded)."""
    npix, m = p_hat.shape
    if m not in (NPAR, NPAR_MAX):
        raise ValueError("p_hat must have 9 or 10 columns")
    _need(p_hat, torch.float64, (npix, m), "p_hat")
    out = torch.empty((npix, 2, m), dtype=torch.float64, device=p_hat.device)
    pad = (float("inf"),) * (m - len(lower))
    lw = np.ascontiguousarray(tuple(lower) + pad, dtype=np.float64)
    up = np.ascontiguousarray(tuple(upper) + pad, dtype=np.float64)
    if lw.shape != (m,) or up.shape != (m,):
        raise ValueError("lower and upper must hold one margin per parameter")
    b = bounds(lo, hi)
    L.check(L.load().me_prefit_bounds(_ptr(p_hat), npix, m, C.byref(b), C.c_void_p(lw.ctypes.data),
                                      C.c_void_p(up.ctypes.data), _ptr(out), _stream()))
    return out


def invert_map(pb: Problem, obs, lo, hi, ga: GaSettings, p_thresh, quiet, line, core, nseed=4,
               polarity=True, prefit=False, prefit_iters=40, polish_iters=10, lambda0=1e-3, w=None,
               polish_w=None, mu_px=None, pixel_id0=0):
    """The Section 2 pipeline on a map, asynchronous on the current stream:
    classification (weak-field answer below the threshold), selection of the
    pixels above it, optionally the Section 5.3 prefit and its per-pixel
    bounds, the seeded, polarity-restricted GA and the L-M polish on those.
    Returns dict(best [npix, 9], chi2 [npix] (NaN for weak-field pixels),
    flag, polarity, index, count, weak, seeds[, prefit, bounds_px])."""
    npix = obs.shape[0]
    dev = obs.device
    best = torch.full((npix, pb.npar), float("nan"), dtype=torch.float64, device=dev)
    chi2 = torch.full((npix,), float("nan"), dtype=torch.float64, device=dev)
    cls = classify(pb, obs, p_thresh, quiet, line, core, best=best)
    index, count = select(cls["flag"], 1)
    sd = cls["seeds"][:, :nseed].contiguous() if nseed > 0 else None
    pol = cls["polarity"] if polarity else None
    extra = {}
    bpx = None
    if prefit:
        p_hat, _ = thermo_prefit(pb, obs, lo, hi, index=index, count=count, iters=prefit_iters, mu_px=mu_px)
        bpx = prefit_bounds(p_hat, lo, hi)
        extra = {"prefit": p_hat, "bounds_px": bpx}
    ga_invert_subset(pb, obs, lo, hi, ga, index=index, count=count, seeds=sd, polarity=pol, bounds_px=bpx, w=w,
                     mu_px=mu_px, pixel_id0=pixel_id0, best=best, chi2=chi2)
    if polish_iters > 0:
        lm_polish_subset(pb, obs, best, lo, hi, index=index, count=count, iters=polish_iters, lambda0=lambda0,
                         w=polish_w if polish_w is not None else w, mu_px=mu_px, chi2=chi2)
    return dict(cls, best=best, chi2=chi2, index=index, count=count, **extra)


# ------------------------------------------------------------------ serving

def _host_f64(a, shape, name):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != shape:
        raise ValueError(f"{name} must have shape {shape}, got {a.shape}")
    return a


class Server:
    """Continuous-batching serving loop (serve_create / submit / poll / destroy).

    Requests are host arrays; the library copies them on submit, admits them
    as in-flight slots and arena memory free up, and runs them concurrently.
    """

    def __init__(self, pb: Problem, arena_bytes=1 << 30, max_inflight=8, max_queue=4096,
                 small_pixels=0, fail_next_admissions=0):
        self.pb = pb
        self._npar = pb.npar
        cfg = L.ServeConfig(int(arena_bytes), int(max_inflight), int(max_queue), int(small_pixels),
                            int(fail_next_admissions))
        h = C.c_void_p()
        L.check(L.load().serve_create(pb.ref(), C.byref(cfg), C.byref(h)))
        self._h = h
        self._npix = {}

    def submit(self, obs, lo, hi, ga: GaSettings, w=None, mu_px=None, pixel_id0=0, polish_iters=0,
               lambda0=1e-3, polish_w=None):
        npix = obs.shape[0]
        dt = np.float32 if self.pb.dtype == F32 else np.float64
        ob = np.ascontiguousarray(obs, dtype=dt)
        if ob.shape != (npix, 4, self.pb.n_lambda):
            raise ValueError("obs must be [npix, 4, n_lambda]")
        wv = _host_f64(w, (npix, 4), "w")
        mv = _host_f64(mu_px, (npix,), "mu_px")
        pw = _host_f64(polish_w, (npix, 4), "polish_w")
        rq = L.ServeRequest()
        rq.obs = ob.ctypes.data
        rq.w = None if wv is None else wv.ctypes.data
        rq.mu_px = None if mv is None else mv.ctypes.data
        rq.npix = npix
        rq.pixel_id0 = int(pixel_id0)
        rq.ga = ga.to_c(L.ME_W_USER if wv is not None else L.ME_W_INVMAX)
        rq.bounds = bounds(lo, hi)
        rq.polish_iters = int(polish_iters)
        rq.lambda0 = float(lambda0)
        rq.polish_w = None if pw is None else pw.ctypes.data
        t = C.c_uint64()
        L.check(L.load().serve_submit(self._h, C.byref(rq), C.byref(t)))
        self._npix[t.value] = npix
        return t.value

    def poll(self, ticket, timeout_ms=-1):
        """Result dict of a finished request; raises GenesisError with code
        ME_EPENDING / ME_ETIMEOUT if it is not done, or the request's error."""
        npix = self._npix.get(ticket, 0)
        best = np.empty((npix, self._npar))
        chi2 = np.empty(npix)
        res = L.ServeResult(best.ctypes.data if npix else None, chi2.ctypes.data if npix else None,
                            0, 0, 0)
        rc = L.load().serve_poll(self._h, int(ticket), C.byref(res), int(timeout_ms))
        if rc in (L.ME_EPENDING, L.ME_ETIMEOUT):
            L.check(rc)
        self._npix.pop(ticket, None)
        L.check(rc)
        return {"best": best, "chi2": chi2, "status": res.status, "queue_ns": res.queue_ns,
                "latency_ns": res.latency_ns}

    def stats(self):
        st = L.ServeStats()
        L.check(L.load().serve_stats(self._h, C.byref(st)))
        return {"queued": st.queued, "running": st.running, "arena_used": st.arena_used,
                "arena_bytes": st.arena_bytes}

    def close(self):
        if self._h:
            L.check(L.load().serve_destroy(self._h))
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ---------------------------------------------------------- operator checks

def _u16_to_dev(a, device):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint16).view(np.int16)).to(device)


def _dev_to_u16(t):
    return t.cpu().numpy().view(np.uint16)


def ga_breed(genes_u16, fitness, pixel_id0, gen, ga: GaSettings, device="cuda"):
    """One breeding step of nprob populations (numpy uint16 [nprob, npop, M],
    M = 9 or 10; float64 [nprob, npop]) -> (child uint16, elite int)."""
    g = np.ascontiguousarray(genes_u16, dtype=np.uint16)
    nprob, npop, _ = g.shape
    gd = _u16_to_dev(g, device)
    fd = torch.as_tensor(np.ascontiguousarray(fitness, dtype=np.float64)).to(device)
    child = torch.empty_like(gd)
    elite = torch.empty(nprob, dtype=torch.int32, device=device)
    cfg = ga.to_c(L.ME_W_INVMAX)
    L.check(L.load().ga_breed(_ptr(gd), _ptr(fd), nprob, npop, g.shape[2], int(pixel_id0), int(gen),
                              C.byref(cfg), _ptr(child), _ptr(elite), _stream()))
    return _dev_to_u16(child), elite.cpu().numpy()


def ga_restart(genes_u16, fitness, sobol_next, device="cuda"):
    g = np.ascontiguousarray(genes_u16, dtype=np.uint16)
    nprob, npop, _ = g.shape
    gd = _u16_to_dev(g, device)
    fd = torch.as_tensor(np.ascontiguousarray(fitness, dtype=np.float64)).to(device)
    L.check(L.load().ga_restart(_ptr(gd), _ptr(fd), nprob, npop, g.shape[2], int(sobol_next), _stream()))
    return _dev_to_u16(gd)


def philox(ctr_u32, key, device="cuda"):
    c = np.ascontiguousarray(ctr_u32, dtype=np.uint32).reshape(-1, 4)
    cd = torch.from_numpy(c.view(np.int32)).to(device)
    out = torch.empty_like(cd)
    L.check(L.load().me_philox(_ptr(cd), c.shape[0], int(key), _ptr(out), _stream()))
    return out.cpu().numpy().view(np.uint32)


def sobol(first, n, ndim, device="cuda"):
    out = torch.empty((n, ndim), dtype=torch.int32, device=device)
    L.check(L.load().me_sobol(int(first), int(n), int(ndim), _ptr(out), _stream()))
    return out.cpu().numpy().view(np.uint32)


# ------------------------------------------------------------- autograd

class MeSynthFunction(torch.autograd.Function):
    """Stokes = me_synth(params); backward uses the analytic adjoint me_synth_vjp."""

    @staticmethod
    def forward(ctx, params, pb, mu_px):
        ctx.pb = pb
        ctx.save_for_backward(params, mu_px if mu_px is not None else torch.empty(0))
        ctx.has_mu = mu_px is not None
        return me_synth(pb, params.detach().contiguous(), mu_px)

    @staticmethod
    def backward(ctx, grad):
        params, mu = ctx.saved_tensors
        g = me_synth_vjp(ctx.pb, params.detach().contiguous(), grad.contiguous().to(ctx.pb.torch_dtype),
                         mu if ctx.has_mu else None)
        return g, None, None


def synth_autograd(pb: Problem, params, mu_px=None):
    return MeSynthFunction.apply(params, pb, mu_px)


def fp32_peak(packed=True, nblocks=None, iters=4096, repeats=3):
    """Measured FP32 FMA-pipe throughput (me_fp32_peak) in TFLOP/s: the best of
    `repeats` launches timed with CUDA events on the current stream after one
    warm-up launch; nblocks defaults to 8 blocks of 256 threads per SM."""
    dev = torch.cuda.current_device()
    if nblocks is None:
        nblocks = 8 * torch.cuda.get_device_properties(dev).multi_processor_count
    out = torch.empty(nblocks * 256, dtype=torch.float32, device="cuda")
    flops = C.c_double(0.0)
    lib = L.load()
    L.check(lib.me_fp32_peak(int(packed), int(nblocks), int(iters), _ptr(out), C.byref(flops), _stream()))
    best = float("inf")
    st = torch.cuda.current_stream()
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        L.check(lib.me_fp32_peak(int(packed), int(nblocks), int(iters), _ptr(out), None, _stream()))
        e1.record(st)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return flops.value / (best / 1e3) / 1e12
