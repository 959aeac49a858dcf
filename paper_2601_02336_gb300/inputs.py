"""Seeded synthetic inputs shared by the GPU library's callers and the oracle's.

This module holds workload recipes only: sizes, prior boxes, sampler
settings, the analytic noise PSD, detector placements, noise draws and
parameter sets. It holds none of the method's arithmetic (no waveform, no
likelihood, no sampler step), so the CUDA path and the oracle can both take
their inputs from it without sharing any computation.

Workloads (stand-ins for the paper's simulated-BBH and GW150914 analyses,
Sec. 6; the paper's IMRPhenomD waveform, design PSD file and strain data are
replaced by TaylorF2, an analytic PSD and Gaussian noise):

  tiny    -- 4-D TaylorF2, one detector, 433 bins, 128 particles.
  bbh11   -- 11-D aligned-spin TaylorF2, 3 detectors, 8 s at 1/8 Hz (8033 bins),
             2048 particles, tree depth 6.
  bbh11_long -- same model, 16 s at 1/16 Hz to 2048 Hz (32449 bins), 16384
             particles, tree depth 8, dense covariance metric.
  batch64 -- 64 events of the 11-D model, 4/8/16/32 s, uneven particle counts.
  bns     -- low-mass 11-D TaylorF2, 128 s at 1/128 Hz (259585 bins), 8192 particles.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# Physical parameter indices of the aligned-spin model.
MC, Q, CHI1, CHI2, DL, COSI, PHIC, PSI, RA, SINDEC, TC = range(11)
NPHYS = 11
PRIOR_UNIFORM, PRIOR_POWER2 = 0, 1
BOUND_REFLECT, BOUND_PERIODIC = 0, 1
METRIC_IDENTITY, METRIC_COVARIANCE = 0, 1

TWO_PI = 2.0 * math.pi


@dataclasses.dataclass
class Workload:
    name: str
    phys: List[int]                 # physical parameter of each free dimension
    lo: List[float]
    hi: List[float]
    prior: List[int]
    boundary: List[int]
    fixed: List[float]              # values of all 11 physical parameters
    n_det: int
    fixed_response: bool            # one detector with F+ = 1, Fx = 0, no delay
    f_min: float
    df: float
    n_bins: int
    n_particles: int
    max_depth: int
    alpha: float = 0.5
    n_mut: int = 2
    metric: int = METRIC_IDENTITY
    eps_scale: float = 0.5
    snr_target: Optional[float] = 20.0   # None: keep the injected distance
    theta_inj: Optional[List[float]] = None

    @property
    def n_dim(self):
        return len(self.phys)

    @property
    def f_max(self):
        return self.f_min + (self.n_bins - 1) * self.df


def _fixed_default():
    f = [0.0] * NPHYS
    f[DL] = 400.0
    f[COSI] = 1.0
    return f


_PHYS11 = [MC, Q, CHI1, CHI2, DL, COSI, PHIC, PSI, RA, SINDEC, TC]
_BOUND11 = [BOUND_REFLECT] * 6 + [BOUND_PERIODIC] * 3 + [BOUND_REFLECT] * 2
_PRIOR11 = [PRIOR_UNIFORM] * 4 + [PRIOR_POWER2] + [PRIOR_UNIFORM] * 6


def _box11(mc=(20.0, 40.0), q=(0.125, 1.0), chi=(-0.99, 0.99)):
    lo = [mc[0], q[0], chi[0], chi[0], 100.0, -1.0, 0.0, 0.0, 0.0, -1.0, -0.1]
    hi = [mc[1], q[1], chi[1], chi[1], 5000.0, 1.0, TWO_PI, math.pi, TWO_PI, 1.0, 0.1]
    return lo, hi


def tiny():
    fixed = _fixed_default()
    return Workload(
        name="tiny", phys=[MC, Q, TC, PHIC], lo=[10.0, 0.5, -0.05, 0.0],
        hi=[12.0, 1.0, 0.05, TWO_PI], prior=[PRIOR_UNIFORM] * 4,
        boundary=[BOUND_REFLECT, BOUND_REFLECT, BOUND_REFLECT, BOUND_PERIODIC], fixed=fixed,
        n_det=1, fixed_response=True, f_min=20.0, df=0.25, n_bins=433, n_particles=128,
        max_depth=5, alpha=0.5, n_mut=2, snr_target=None, theta_inj=[11.0, 0.75, 0.0, math.pi])


def bbh11(n_particles=2048):
    lo, hi = _box11()
    return Workload(
        name="bbh11", phys=list(_PHYS11), lo=lo, hi=hi, prior=list(_PRIOR11),
        boundary=list(_BOUND11), fixed=_fixed_default(), n_det=3, fixed_response=False,
        f_min=20.0, df=0.125, n_bins=8033, n_particles=n_particles, max_depth=6)


def bbh11_long(n_particles=16384):
    lo, hi = _box11()
    return Workload(
        name="bbh11_long", phys=list(_PHYS11), lo=lo, hi=hi, prior=list(_PRIOR11),
        boundary=list(_BOUND11), fixed=_fixed_default(), n_det=3, fixed_response=False,
        f_min=20.0, df=1.0 / 16.0, n_bins=32449, n_particles=n_particles, max_depth=8,
        metric=METRIC_COVARIANCE)


def bns(n_particles=8192):
    lo, hi = _box11(mc=(1.1, 1.3), q=(0.5, 1.0), chi=(-0.05, 0.05))
    return Workload(
        name="bns", phys=list(_PHYS11), lo=lo, hi=hi, prior=list(_PRIOR11),
        boundary=list(_BOUND11), fixed=_fixed_default(), n_det=3, fixed_response=False,
        f_min=20.0, df=1.0 / 128.0, n_bins=259585, n_particles=n_particles, max_depth=8)


def batch64(seed=3):
    """64 events: durations 4/8/16/32 s (16 each), 20-1024 Hz at df = 1/T,
    particle counts log-uniform in [512, 8192]."""
    rng = np.random.Generator(np.random.Philox(seed))
    out = []
    for i in range(64):
        T = [4, 8, 16, 32][i // 16]
        n = int(round(math.exp(rng.uniform(math.log(512), math.log(8192)))))
        w = bbh11(n_particles=n)
        w.name = f"batch64_{i}"
        w.df = 1.0 / T
        w.n_bins = (1024 - 20) * T + 1
        w.max_depth = 8
        out.append(w)
    return out


@dataclasses.dataclass
class MixtureWorkload:
    """A target without a waveform: a sum of diagonal Gaussians in a box."""
    name: str
    lo: List[float]
    hi: List[float]
    logw: List[float]
    mu: List[List[float]]
    sigma: List[List[float]]
    n_particles: int
    max_depth: int
    alpha: float = 0.5
    n_mut: int = 2
    metric: int = METRIC_COVARIANCE
    eps_scale: float = 0.5

    @property
    def n_dim(self):
        return len(self.lo)


def bimodal11(n_particles=4096):
    """The bimodal 11-D target of App. A (Eq. A1): N(1_11, 0.01 I) + N(-1_11, 0.01 I),
    both normalised, so Z = 2 / prior volume; uniform prior box [-5, 5]^11 (the
    paper does not state the prior); alpha = 0.95 as in the paper's runs (Sec. 6):
    with larger tempering steps the share of each mode drifts before the modes
    separate."""
    d = 11
    return MixtureWorkload(name="bimodal11", lo=[-5.0] * d, hi=[5.0] * d, logw=[0.0, 0.0],
                           mu=[[1.0] * d, [-1.0] * d], sigma=[[0.1] * d, [0.1] * d],
                           n_particles=n_particles, max_depth=6, alpha=0.95)


WORKLOADS = {"tiny": tiny, "bbh11": bbh11, "bbh11_long": bbh11_long, "bns": bns}


# ------------------------------------------------------------------ noise
def psd(f):
    """Analytic one-sided PSD S(f) = 1e-46 [(f/30)^-8 + 1 + (f/150)^2] / Hz."""
    f = np.asarray(f, dtype=np.float64)
    return 1e-46 * ((f / 30.0) ** -8 + 1.0 + (f / 150.0) ** 2)


def frequencies(w: Workload):
    return w.f_min + np.arange(w.n_bins, dtype=np.float64) * w.df


def psd_array(w: Workload):
    return np.tile(psd(frequencies(w)), (w.n_det, 1))


def detectors(w: Workload, seed=0):
    """Detector placements: one fixed-response detector, or three L-shaped
    detectors with lat = asin(2U-1), lon = 2 pi U, azimuth = 2 pi U."""
    if w.fixed_response:
        return [dict(fixed_response=1, fplus=1.0, fcross=0.0, delay=0.0)]
    rng = np.random.Generator(np.random.Philox(seed))
    dets = []
    for _ in range(w.n_det):
        u = rng.uniform(size=3)
        dets.append(dict(lat=math.asin(2.0 * u[0] - 1.0), lon=TWO_PI * u[1], azimuth=TWO_PI * u[2]))
    return dets


def noise(w: Workload, seed=0):
    """Gaussian noise with Re, Im ~ N(0, S/(4 df)) per bin: [n_det][n_bins][2]."""
    rng = np.random.Generator(np.random.Philox(1000 + seed))
    sig = np.sqrt(psd_array(w) / (4.0 * w.df))
    z = rng.standard_normal((w.n_det, w.n_bins, 2))
    return z * sig[:, :, None]


# ------------------------------------------------------------- parameters
def prior_draws(w: Workload, n, seed):
    """Parameter vectors drawn from the prior box (input sets, numpy RNG)."""
    rng = np.random.Generator(np.random.Philox(2000 + seed))
    u = rng.uniform(size=(n, w.n_dim))
    lo = np.array(w.lo)
    hi = np.array(w.hi)
    th = lo + u * (hi - lo)
    for i, p in enumerate(w.prior):
        if p == PRIOR_POWER2:
            th[:, i] = np.cbrt(lo[i] ** 3 + u[:, i] * (hi[i] ** 3 - lo[i] ** 3))
    return th


def injection(w: Workload, seed=0):
    """Injected parameters before any distance rescaling."""
    if w.theta_inj is not None:
        return np.array(w.theta_inj, dtype=np.float64)
    return prior_draws(w, 1, 10_000 + seed)[0]


def ball(w: Workload, center, n, seed, rel=1e-3):
    """Gaussian ball around `center` with sigma = rel * prior width, folded into the box."""
    rng = np.random.Generator(np.random.Philox(3000 + seed))
    lo = np.array(w.lo)
    hi = np.array(w.hi)
    th = np.asarray(center)[None, :] + rel * (hi - lo)[None, :] * rng.standard_normal((n, w.n_dim))
    return np.clip(th, lo, hi)


def distance_index(w: Workload):
    return w.phys.index(DL) if DL in w.phys else None
