"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module holds no arithmetic of the inversion method: it defines the line
list (Table 1 of Harker & Mighell 2012), wavelength grids, prior ranges and
parameter bounds, and draws truth parameter vectors, standard-normal noise and
request streams from seeded generators.  Synthesising the observed Stokes
profiles from the truth is left to the caller (the oracle in tests, the CUDA
``me_synth`` in the benchmark), as is scaling the noise by sigma = 1e-3 I_c.

Workloads (the paper's SOLIS/VSM cube is not available; these stand in for it):
    c1  16x16 px, Fe I 6302.5 only (g = 2.5), 64 points over 6302.0-6303.0 A,
        FP64 cube, population 64, 100 generations, Philox seed 0
    c2  256x256 px, Fe I 6301.5 + 6302.5 in one K, 128 points over
        6301.0-6303.0 A, population 128, 200 generations
    c3  512x512 px, the c2 setup with a float32 cube (+ 10 L-M iterations)
    c4  serving stream: requests of 64-4096 px (log-uniform), 30% of pixels
        magnetised with B log-uniform 10-3000 G, the rest B ~ U(0, 50) G,
        population 64/128, 100/200/300 generations, float32
    c5  2048x2048 grid, on-disc mask r <= 1024 px, mu = sqrt(1 - r^2),
        limb-darkened quiet sun, ~40 spot clusters, float32
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

NPAR = 9
PARAM_NAMES = ("B", "theta", "chi", "vlos", "dlambdaD", "a", "eta0", "S0", "S1")
PARAM_UNITS = ("G", "deg", "deg", "km/s", "mA", "", "", "", "")

# Table 1: Fe I multiplet 816 (wavelength A, g_eff, excitation eV, log gf)
FE6301 = (6301.5091, 1.667, 3.654, -0.718)
FE6302 = (6302.5017, 2.500, 3.686, -1.235)
BOLTZMANN_EV = 8.617333262e-5


def eta_ratio_6301(temperature_k: float = 5000.0) -> float:
    """eta0(6301.5)/eta0(6302.5) from Table 1's gf values and excitation
    potentials under a Boltzmann population at temperature_k (a problem
    constant, not part of the inversion)."""
    dgf = FE6301[3] - FE6302[3]
    dchi = FE6301[2] - FE6302[2]
    return 10.0 ** dgf * math.exp(-dchi / (BOLTZMANN_EV * temperature_k))


# prior ranges (uniform per pixel) = GA bounds
PRIOR_LO = np.array([0.0, 0.0, 0.0, -3.0, 20.0, 0.0, 1.0, 0.1, 0.1])
PRIOR_HI = np.array([3000.0, 180.0, 180.0, 3.0, 50.0, 0.5, 20.0, 1.0, 1.0])
# with the fill fraction alpha in [0, 1] as a 10th parameter
PRIOR_LO_FILL = np.append(PRIOR_LO, 0.0)
PRIOR_HI_FILL = np.append(PRIOR_HI, 1.0)


@dataclass
class ProblemSpec:
    """Line list + wavelength grid; lines are (lambda0 [A], g_eff, eta_ratio).
    fill: the magnetic fill fraction alpha is a 10th parameter."""
    lines: list
    lambda_grid: np.ndarray
    lambda_dop: float = FE6302[0]   # Doppler-width parameter quoted at 6302.5 A
    mu: float = 1.0
    fill: bool = False

    @property
    def n_lambda(self) -> int:
        return len(self.lambda_grid)

    @property
    def n_lines(self) -> int:
        return len(self.lines)


@dataclass
class Workload:
    name: str
    spec: ProblemSpec
    nx: int
    ny: int
    npop: int
    ngen: int
    dtype: str          # "f64" or "f32" cube / GA precision
    lm_iters: int = 0
    seed: int = 0
    lo: np.ndarray = field(default_factory=lambda: PRIOR_LO.copy())
    hi: np.ndarray = field(default_factory=lambda: PRIOR_HI.copy())

    @property
    def npix(self) -> int:
        return self.nx * self.ny


def one_line_spec(n_lambda=64, lo=6302.0, hi=6303.0) -> ProblemSpec:
    return ProblemSpec(lines=[(FE6302[0], FE6302[1], 1.0)],
                       lambda_grid=np.linspace(lo, hi, n_lambda))


# Table 1's lines with their levels for the full Zeeman pattern: (lambda0,
# g_eff, eta_ratio, J_lower, g_lower, J_upper, g_upper); Fe I 6301.5 is
# 5P2 - 5D2 (LS Lande factors 11/6 and 3/2), Fe I 6302.5 5P1 - 5D0.
def fe6301_full_line():
    return (FE6301[0], FE6301[1], eta_ratio_6301(), 2, 11.0 / 6.0, 2, 1.5)


def two_line_pattern_spec(n_lambda=128, lo=6301.0, hi=6303.0) -> ProblemSpec:
    """The two-line grid with Fe I 6301.5 as its full Zeeman pattern (four
    components per sigma_b, pi, sigma_r group) and 6302.5 as its normal
    triplet."""
    return ProblemSpec(lines=[fe6301_full_line(), (FE6302[0], FE6302[1], 1.0)],
                       lambda_grid=np.linspace(lo, hi, n_lambda))


def two_line_spec(n_lambda=128, lo=6301.0, hi=6303.0) -> ProblemSpec:
    return ProblemSpec(lines=[(FE6301[0], FE6301[1], eta_ratio_6301()),
                              (FE6302[0], FE6302[1], 1.0)],
                       lambda_grid=np.linspace(lo, hi, n_lambda))


def workload(name: str) -> Workload:
    if name == "c1":
        return Workload("c1", one_line_spec(), 16, 16, 64, 100, "f64", seed=0)
    if name == "c2":
        return Workload("c2", two_line_spec(), 256, 256, 128, 200, "f64", seed=0)
    if name == "c3":
        return Workload("c3", two_line_spec(), 512, 512, 128, 200, "f32", lm_iters=10, seed=0)
    if name == "c5":
        return Workload("c5", two_line_spec(), 2048, 2048, 128, 300, "f32", lm_iters=10, seed=0)
    raise KeyError(name)


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=(int(seed) << 16) + int(stream)))


def draw_truth(npix: int, seed: int = 0, lo=PRIOR_LO, hi=PRIOR_HI) -> np.ndarray:
    """Truth parameters [npix, len(lo)], uniform per pixel within [lo, hi]."""
    r = _rng(seed, 1)
    u = r.random((npix, len(lo)))
    return lo + (hi - lo) * u


def draw_noise(npix: int, n_lambda: int, seed: int = 0) -> np.ndarray:
    """Standard-normal noise [npix, 4, n_lambda] (scale by 1e-3 I_c)."""
    r = _rng(seed, 2)
    return r.standard_normal((npix, 4, n_lambda))


def draw_params_uniform(n: int, seed: int, lo=PRIOR_LO, hi=PRIOR_HI) -> np.ndarray:
    """Random parameter vectors for parity / finite-difference checks."""
    r = _rng(seed, 3)
    return lo + (hi - lo) * r.random((n, len(lo)))


# ------------------------------------------------------------------ c4

@dataclass
class Request:
    arrival_s: float
    npix: int
    npop: int
    ngen: int
    truth: np.ndarray     # [npix, 9]
    seed: int


def draw_requests(n_requests: int, rate_hz: float, seed: int = 4,
                  max_pixels: int = 4096) -> list:
    """Poisson arrivals of slit-scan / map-tile requests (workload c4)."""
    r = _rng(seed, 4)
    t = 0.0
    out = []
    for k in range(n_requests):
        t += r.exponential(1.0 / rate_hz)
        npix = int(math.floor(math.exp(r.uniform(math.log(64), math.log(max_pixels)))))
        npop = int(r.choice([64, 128]))
        ngen = int(r.choice([100, 200, 300]))
        p = PRIOR_LO + (PRIOR_HI - PRIOR_LO) * r.random((npix, NPAR))
        mag = r.random(npix) < 0.3
        bmag = np.exp(r.uniform(math.log(10.0), math.log(3000.0), npix))
        bweak = r.uniform(0.0, 50.0, npix)
        p[:, 0] = np.where(mag, bmag, bweak)
        out.append(Request(t, npix, npop, ngen, p, seed * 100003 + k))
    return out


# ------------------------------------------------------------------ c5

def disc_geometry(n: int = 2048):
    """On-disc mask and mu of an n x n full-disc grid (radius n/2 px)."""
    c = (n - 1) / 2.0
    yy, xx = np.mgrid[0:n, 0:n]
    r = np.hypot(xx - c, yy - c) / (n / 2.0)
    mask = r <= 1.0
    mu = np.sqrt(np.clip(1.0 - r * r, 0.0, 1.0))
    return mask, mu


def draw_full_disc(n: int = 2048, seed: int = 5, n_spots: int = 40):
    """Truth [npix_on_disc, 9] and mu [npix_on_disc] of the synthetic full disc.

    Quiet sun: S0 ~ U(0.25, 0.35), S1 ~ U(0.65, 0.75) (limb darkening then comes
    from I_c = S0 + mu S1), weak field B log-uniform in 1-50 G.  About n_spots
    clusters with Gaussian radius 10-40 px carry B 1500-3000 G and S0, S1 scaled
    by 0.3-0.6 in the core, blended by the Gaussian weight.
    """
    r = _rng(seed, 5)
    mask, mu = disc_geometry(n)
    iy, ix = np.nonzero(mask)
    npix = len(iy)
    p = PRIOR_LO + (PRIOR_HI - PRIOR_LO) * r.random((npix, NPAR))
    p[:, 0] = np.exp(r.uniform(0.0, math.log(50.0), npix))
    p[:, 7] = r.uniform(0.25, 0.35, npix)
    p[:, 8] = r.uniform(0.65, 0.75, npix)
    c = (n - 1) / 2.0
    for _ in range(n_spots):
        rad = r.uniform(0.0, 0.85) * n / 2.0
        ang = r.uniform(0.0, 2 * math.pi)
        cx, cy = c + rad * math.cos(ang), c + rad * math.sin(ang)
        sig = r.uniform(10.0, 40.0)
        bcore = r.uniform(1500.0, 3000.0)
        dark = r.uniform(0.3, 0.6)
        wgt = np.exp(-((ix - cx) ** 2 + (iy - cy) ** 2) / (2 * sig * sig))
        sel = wgt > 1e-3
        wv = wgt[sel]
        p[sel, 0] = (1 - wv) * p[sel, 0] + wv * bcore
        p[sel, 7] *= (1 - wv) + wv * dark
        p[sel, 8] *= (1 - wv) + wv * dark
    return p, mu[mask], mask
