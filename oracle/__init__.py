"""Plain FP64 CPU oracle for the GENESIS Milne-Eddington GA inversion.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The C sources in this directory share no
code with the CUDA path; this module compiles them with gcc into
``oracle/liboracle.so`` and exposes them through ctypes with numpy arrays.

Every function cites the passage of Harker & Mighell (2012) it follows:
    faddeeva        Section 5 (Voigt / Faraday-Voigt profiles, Hui et al. 1978)
    synth, synth_lu Section 5 (Unno-Rachkovsky ME solution, K = 1 + eta0 Phi)
    weights_invmax  Section 5.4 (inverse-max weighting)
    chi2            Section 5, Eq. chisq
    philox, sobol   Section 5.6 (Sobol initialisation); Philox drives S, R, M
    ga_breed        Section 3, Algorithm 1 (S, E, R, M, elitism)
    ga_restart      Section 5.6 (worst half replaced every N_samp generations)
    ga_invert       Algorithm 1 run per pixel
    jacobian, lm_polish   Levenberg-Marquardt (Section 1, Section 5.3)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["me.c", "rng.c", "ga.c", "lm.c", "zeeman.c"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NPAR = 9
MAX_LINES = 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction) if out of date."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES] + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-pthread", "-o", tmp] + [os.path.join(_HERE, s) for s in _SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(C.Structure):
    _fields_ = [("n_lines", C.c_int),
                ("lambda0", C.c_double * MAX_LINES),
                ("g", C.c_double * MAX_LINES),
                ("eta_ratio", C.c_double * MAX_LINES),
                ("pattern", C.c_int * MAX_LINES),
                ("j_lower", C.c_int * MAX_LINES),
                ("j_upper", C.c_int * MAX_LINES),
                ("g_lower", C.c_double * MAX_LINES),
                ("g_upper", C.c_double * MAX_LINES),
                ("lambda_dop", C.c_double),
                ("n_lambda", C.c_int),
                ("lam", C.POINTER(C.c_double)),
                ("fill", C.c_int)]


class _GaConfig(C.Structure):
    _fields_ = [("npop", C.c_int), ("ngen", C.c_int), ("nsamp", C.c_int),
                ("pc", C.c_double), ("pmut_lsb", C.c_double), ("pmut_ratio", C.c_double),
                ("seed", C.c_uint64)]


_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_U16 = np.ctypeslib.ndpointer(dtype=np.uint16, flags="C_CONTIGUOUS")
_U32 = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_I32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def _optional(arr_type):
    """ndpointer that also accepts None (NULL)."""
    def from_param(cls, obj):
        if obj is None:
            return None
        return arr_type.from_param(obj)
    return type("Opt" + arr_type.__name__, (arr_type,), {"from_param": classmethod(from_param)})


_DN = _optional(_D)
_U16N = _optional(_U16)
_I32N = _optional(_I32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            P = C.POINTER(_Problem)
            L.or_faddeeva_batch.argtypes = [C.c_int, _D, _D, _D, _D]
            L.or_wigner3j.argtypes = [C.c_int] * 6
            L.or_wigner3j.restype = C.c_double
            L.or_zeeman_components.argtypes = [C.c_int, C.c_double, C.c_int, C.c_double,
                                               np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS"),
                                               _D, _D]
            L.or_zeeman_components.restype = C.c_int
            L.or_synth.argtypes = [P, _D, C.c_double, _D]
            L.or_synth_lu.argtypes = [P, _D, C.c_double, _D]
            L.or_synth_batch.argtypes = [P, _D, C.c_int, _DN, C.c_double, _D, C.c_int]
            L.or_weights_invmax.argtypes = [_D, C.c_int, _D]
            L.or_chi2.argtypes = [_D, _D, _D, C.c_int, C.c_int]
            L.or_chi2.restype = C.c_double
            L.or_philox4x32.argtypes = [_U32, _U32, _U32]
            L.or_sobol_u32.argtypes = [C.c_uint64, C.c_int]
            L.or_sobol_u32.restype = C.c_uint32
            L.or_sobol_directions.argtypes = [C.c_int, _U32]
            L.or_ga_decode.argtypes = [_U16, _D, _D, C.c_int, _D]
            L.or_ga_breed.argtypes = [_U16, _D, C.c_int, C.c_int, C.c_uint64, C.c_int,
                                      C.POINTER(_GaConfig), _U16]
            L.or_ga_breed.restype = C.c_int
            L.or_ga_restart.argtypes = [_U16, _D, C.c_int, C.c_int, C.c_uint64, _I32]
            L.or_ga_invert.argtypes = [P, _D, _DN, _DN, C.c_double, C.c_int, C.c_uint64,
                                       _D, _D, C.POINTER(_GaConfig), _DN, C.c_int, _I32N,
                                       _DN, _D, _D, _U16N, _DN, C.c_int]
            L.or_ga_encode.argtypes = [C.c_double, C.c_double, C.c_double]
            L.or_ga_encode.restype = C.c_uint16
            L.or_polarity_bounds.argtypes = [C.c_int, C.c_double, C.c_double, C.POINTER(C.c_double),
                                             C.POINTER(C.c_double)]
            L.or_ga_invert.restype = C.c_int
            L.or_jacobian.argtypes = [P, _D, C.c_double, _D]
            L.or_lm_polish.argtypes = [P, _D, _DN, _DN, C.c_double, C.c_int, _D, _D,
                                       C.c_int, C.c_double, C.c_uint, _D, _D, C.c_int]
            L.or_prefit_bounds.argtypes = [_D, C.c_int, C.c_int, _D, _D, _D, _D, _D]
            L.or_lm_polish.restype = C.c_int
            L.or_line_centre.argtypes = [_D, C.c_int, C.c_int, C.c_int, _D, C.c_int, C.c_int, C.c_int,
                                         _D, _I32]
            L.or_classify.argtypes = [P, _D, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int,
                                      C.c_int, _I32, _I32, _D, _D, _D]
            L.or_lm_uncertainty.argtypes = [P, _D, _DN, _DN, C.c_double, C.c_int, _D, _D]
            _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def nthreads_default() -> int:
    return max(1, os.cpu_count() or 1)


class Problem:
    """ctypes view of a line list + wavelength grid (keeps the grid alive)."""

    def __init__(self, lines, lambda_grid, lambda_dop, fill=False):
        if not 1 <= len(lines) <= MAX_LINES:
            raise ValueError("1..4 lines")
        self.lam = _f64(lambda_grid)
        s = _Problem()
        s.n_lines = len(lines)
        for i, ln in enumerate(lines):
            s.lambda0[i], s.g[i], s.eta_ratio[i] = ln[0], ln[1], ln[2]
            if len(ln) > 3:   # full pattern: (..., j_lower, g_lower, j_upper, g_upper)
                s.pattern[i] = 1
                s.j_lower[i], s.g_lower[i], s.j_upper[i], s.g_upper[i] = int(ln[3]), ln[4], int(ln[5]), ln[6]
        s.lambda_dop = float(lambda_dop)
        s.n_lambda = len(self.lam)
        s.lam = self.lam.ctypes.data_as(C.POINTER(C.c_double))
        s.fill = 1 if fill else 0
        self.s = s
        self.n_lambda = len(self.lam)
        self.npar = NPAR + (1 if fill else 0)

    @classmethod
    def from_spec(cls, spec):
        """From any object with .lines [(lambda0, g, eta_ratio)], .lambda_grid,
        .lambda_dop (and optionally .fill: the fill fraction is parameter 9)."""
        return cls(spec.lines, spec.lambda_grid, spec.lambda_dop, getattr(spec, "fill", False))

    def ref(self):
        return C.byref(self.s)


def _problem(pb):
    return pb if isinstance(pb, Problem) else Problem.from_spec(pb)


def ga_config(npop, ngen, nsamp=None, pc=0.9, pmut_lsb=0.05, pmut_ratio=0.7, seed=0):
    if nsamp is None:
        nsamp = ngen // 4
    return _GaConfig(int(npop), int(ngen), int(nsamp), float(pc), float(pmut_lsb),
                     float(pmut_ratio), int(seed))


# ------------------------------------------------------------------ profiles

def faddeeva(x, y):
    """w(x + i y) (Section 5 profiles; Matta & Reichel trapezoid)."""
    x, y = np.broadcast_arrays(_f64(x), _f64(y))
    shape = x.shape
    x, y = _f64(x.ravel()), _f64(y.ravel())
    re = np.empty_like(x)
    im = np.empty_like(x)
    lib().or_faddeeva_batch(len(x), x, y, re, im)
    return (re + 1j * im).reshape(shape)


def wigner3j(j1, j2, j3, m1, m2, m3):
    return lib().or_wigner3j(int(j1), int(j2), int(j3), int(m1), int(m2), int(m3))


def zeeman_components(j_lower, g_lower, j_upper, g_upper):
    """[(shifts, strengths)] for the sigma_b, pi, sigma_r groups (Section 5
    full Zeeman pattern), shifts in Larmor units toward longer wavelength."""
    n = np.zeros(3, dtype=np.int32)
    sh = np.zeros((3, 9))
    st = np.zeros((3, 9))
    rc = lib().or_zeeman_components(int(j_lower), float(g_lower), int(j_upper), float(g_upper), n, sh, st)
    if rc:
        raise ValueError("invalid transition")
    return [(sh[g, :n[g]].copy(), st[g, :n[g]].copy()) for g in range(3)]


# ----------------------------------------------------------------- synthesis

def synth(pb, params, mu=1.0, mu_px=None, nthreads=None):
    """Stokes [n,4,n_lambda] of params [n,M] (Section 5 ME solution)."""
    pb = _problem(pb)
    p = _f64(np.atleast_2d(params))
    if p.shape[1] != pb.npar:
        raise ValueError(f"params must have {pb.npar} columns")
    n = p.shape[0]
    out = np.empty((n, 4, pb.n_lambda))
    mp = None if mu_px is None else _f64(mu_px)
    lib().or_synth_batch(pb.ref(), p, n, mp, float(mu), out, nthreads or nthreads_default())
    return out


def synth_lu(pb, params, mu=1.0):
    """Stokes [4,n_lambda] of one model, solving K x = e directly."""
    pb = _problem(pb)
    out = np.empty((4, pb.n_lambda))
    lib().or_synth_lu(pb.ref(), _f64(params), float(mu), out)
    return out


def weights_invmax(obs):
    """Section 5.4 inverse-max weights of obs [...,4,n_lambda] -> [...,4]."""
    obs = _f64(obs)
    flat = obs.reshape(-1, 4, obs.shape[-1])
    w = np.empty((flat.shape[0], 4))
    for i in range(flat.shape[0]):
        row = np.empty(4)
        lib().or_weights_invmax(_f64(flat[i]), obs.shape[-1], row)
        w[i] = row
    return w.reshape(obs.shape[:-2] + (4,))


def chi2(obs, model, w, m=NPAR):
    """Eq. chisq for one pixel."""
    obs, model = _f64(obs), _f64(model)
    return lib().or_chi2(obs, model, _f64(w), obs.shape[-1], int(m))


# ----------------------------------------------------------------------- RNG

def philox(ctr, key):
    """Philox4x32-10 of counter [4] under key [2] -> [4] uint32."""
    out = np.empty(4, dtype=np.uint32)
    lib().or_philox4x32(np.ascontiguousarray(ctr, dtype=np.uint32),
                        np.ascontiguousarray(key, dtype=np.uint32), out)
    return out


def sobol_u32(n, dim):
    return int(lib().or_sobol_u32(int(n), int(dim)))


def sobol_directions(dim):
    v = np.empty(32, dtype=np.uint32)
    lib().or_sobol_directions(int(dim), v)
    return v


# ------------------------------------------------------------------------ GA

def ga_decode(genes, lo, hi):
    """Eq. decode of uint16 genes [..., m] -> parameters."""
    g = np.ascontiguousarray(genes, dtype=np.uint16)
    flat = g.reshape(-1, g.shape[-1])
    out = np.empty(flat.shape)
    for i in range(flat.shape[0]):
        row = np.empty(flat.shape[1])
        lib().or_ga_decode(np.ascontiguousarray(flat[i]), _f64(lo), _f64(hi), flat.shape[1], row)
        out[i] = row
    return out.reshape(g.shape)


def ga_breed(genes, f, pixel_id, gen, cfg):
    """One generation of S, R, M and elitism; returns (child genes, elite index)."""
    genes = np.ascontiguousarray(genes, dtype=np.uint16)
    npop, m = genes.shape
    child = np.empty_like(genes)
    e = lib().or_ga_breed(genes, _f64(f), npop, m, int(pixel_id), int(gen), C.byref(cfg), child)
    return child, e


def ga_restart(genes, f, sobol_next):
    """Replace the worst half of genes (in place copy) with Sobol points."""
    genes = np.array(genes, dtype=np.uint16, order="C")
    npop, m = genes.shape
    rep = np.empty(npop // 2, dtype=np.int32)
    lib().or_ga_restart(genes, _f64(f), npop, m, int(sobol_next), rep)
    return genes, rep


def ga_invert(pb, obs, lo, hi, cfg, w=None, mu=1.0, mu_px=None, pixel_id0=0,
              nthreads=None, want_margin=False, seeds=None, polarity=None, bounds_px=None):
    """Algorithm 1 per pixel; returns dict(best, chi2, genes[, margin]).
    seeds [npix][nseed][3] (B, psi, chi) and polarity [npix] of Section 5.5;
    bounds_px [npix][2][9] per-pixel bounds (Section 5.3)."""
    pb = _problem(pb)
    obs = _f64(obs)
    npix = obs.shape[0]
    nseed = 0
    if seeds is not None:
        seeds = _f64(np.asarray(seeds, dtype=np.float64).reshape(npix, -1, 3))
        nseed = seeds.shape[1]
    if polarity is not None:
        polarity = np.ascontiguousarray(polarity, dtype=np.int32).reshape(npix)
    m = pb.npar
    best = np.empty((npix, m))
    c2 = np.empty(npix)
    genes = np.empty((npix, m), dtype=np.uint16)
    margin = np.empty(npix) if want_margin else None
    rc = lib().or_ga_invert(pb.ref(), obs, None if w is None else _f64(w),
                            None if mu_px is None else _f64(mu_px), float(mu), npix,
                            int(pixel_id0), _f64(lo), _f64(hi), C.byref(cfg), seeds, nseed,
                            polarity, None if bounds_px is None else _f64(bounds_px), best, c2, genes,
                            margin, nthreads or nthreads_default())
    if rc != 0:
        raise ValueError("or_ga_invert rejected its arguments")
    out = {"best": best, "chi2": c2, "genes": genes}
    if want_margin:
        out["margin"] = margin
    return out


# ------------------------------------------------------------------- L-M

def jacobian(pb, params, mu=1.0):
    """d stokes / d p as [4, n_lambda, M] (central differences + Richardson)."""
    pb = _problem(pb)
    jac = np.empty((4 * pb.n_lambda, pb.npar))
    lib().or_jacobian(pb.ref(), _f64(params), float(mu), jac)
    return jac.reshape(4, pb.n_lambda, pb.npar)


def lm_polish(pb, obs, params, lo, hi, iters=10, lambda0=1e-3, w=None, mu=1.0,
              mu_px=None, nthreads=None, free_mask=0x3FF):
    """Levenberg-Marquardt polish; returns (params [npix,M], chi2 [npix]).
    Parameters outside free_mask (bit k = parameter k) are held."""
    pb = _problem(pb)
    obs = _f64(obs)
    npix = obs.shape[0]
    p = np.array(params, dtype=np.float64, order="C").reshape(npix, pb.npar)
    c2 = np.empty(npix)
    rc = lib().or_lm_polish(pb.ref(), obs, None if w is None else _f64(w),
                            None if mu_px is None else _f64(mu_px), float(mu), npix,
                            _f64(lo), _f64(hi), int(iters), float(lambda0), int(free_mask), p, c2,
                            nthreads or nthreads_default())
    if rc != 0:
        raise ValueError("or_lm_polish rejected its arguments")
    return p, c2


def lm_uncertainty(pb, obs, params, w=None, mu=1.0, mu_px=None):
    """Section 6 sigma_i = sqrt([H^-1]_ii chi2 / M), H = (2/nu) J^T W^2 J."""
    pb = _problem(pb)
    obs = _f64(obs)
    npix = obs.shape[0]
    out = np.empty((npix, pb.npar))
    lib().or_lm_uncertainty(pb.ref(), obs, None if w is None else _f64(w),
                            None if mu_px is None else _f64(mu_px), float(mu), npix,
                            _f64(np.reshape(params, (npix, pb.npar))), out)
    return out


def line_centre(obs, lambda_grid, half_width, i_lo=0, i_hi=1 << 30):
    """Section 5.1 centre-of-symmetry line centre of each pixel's Stokes I
    (obs [npix, 4, n_lambda]) -> (lambda_c [npix], index [npix])."""
    obs = _f64(obs)
    npix, _, nl = obs.shape
    lc = np.empty(npix)
    idx = np.empty(npix, dtype=np.int32)
    lib().or_line_centre(obs, npix, 4 * nl, nl, _f64(lambda_grid), int(half_width), int(i_lo),
                         int(i_hi), lc, idx)
    return lc, idx


def classify(pb, obs, p_thresh, quiet, line, core):
    """Section 2 selection, weak-field fallback and Section 5.5 seeds.
    quiet = (lo, hi) half-open quiet window, core = (lo, hi) inclusive line
    window.  Returns dict(flag, polarity, p, sigma_p, B, theta, chi, B_par,
    B_perp, seeds [npix][4][3] = (B, psi, chi) of the weak-field, integral,
    centre-of-gravity and non-magnetic seeds)."""
    pb = _problem(pb)
    obs = _f64(obs)
    npix = obs.shape[0]
    flag = np.empty(npix, dtype=np.int32)
    pol = np.empty(npix, dtype=np.int32)
    pp = np.empty((npix, 2))
    weak = np.empty((npix, 5))
    seeds = np.empty((npix, 4, 3))
    lib().or_classify(pb.ref(), obs, npix, float(p_thresh), int(quiet[0]), int(quiet[1]), int(line),
                      int(core[0]), int(core[1]), flag, pol, pp, weak, seeds)
    return {"flag": flag, "polarity": pol, "p": pp[:, 0], "sigma_p": pp[:, 1], "B": weak[:, 0],
            "theta": weak[:, 1], "chi": weak[:, 2], "B_par": weak[:, 3], "B_perp": weak[:, 4], "seeds": seeds}


def ga_encode(x, lo, hi):
    """Nearest gene of a seed value (the inverse of the decode)."""
    return int(lib().or_ga_encode(float(x), float(lo), float(hi)))


def polarity_bounds(pol, lo, hi):
    """Inclination domain of Section 5.5's polarity restriction."""
    a, b = C.c_double(), C.c_double()
    lib().or_polarity_bounds(int(pol), float(lo), float(hi), C.byref(a), C.byref(b))
    return a.value, b.value


def prefit_bounds(p_hat, lo, hi, lower, upper):
    """Per-pixel bounds [npix][2][M] around a thermodynamic prefit (Section 5.3);
    M = the number of columns of p_hat."""
    p_hat = np.asarray(p_hat, dtype=np.float64)
    m = p_hat.shape[-1]
    p = _f64(p_hat.reshape(-1, m))
    out = np.empty((p.shape[0], 2, m))
    lib().or_prefit_bounds(p, p.shape[0], m, _f64(lo), _f64(hi), _f64(lower), _f64(upper), out)
    return out
