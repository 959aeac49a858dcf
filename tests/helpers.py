"""Oracle-side construction of models and events from the workload recipes.

Used by the tests only. Data = oracle waveform at the injection + seeded
noise; the distance is rescaled to the target network SNR using the oracle
(SNR^2 = -2 ln L with zero data).
"""
import math

import numpy as np

import oracle
from paper_2601_02336_gb300 import inputs


def oracle_model(w: inputs.Workload):
    return oracle.make_model(oracle.KIND_GW, w.phys, w.lo, w.hi, w.prior, w.boundary, w.fixed)


def gaussmix_model(lo, hi, logw, mu, sigma, boundary=None):
    d = len(lo)
    return oracle.make_model(oracle.KIND_GAUSSMIX, list(range(d)), lo, hi, [0] * d,
                             boundary or [0] * d, None, logw, mu, sigma)


def oracle_event(w: inputs.Workload, seed=0, noise=True, data=None):
    dets = inputs.detectors(w)
    psd = inputs.psd_array(w)
    if data is None:
        data = np.zeros((w.n_det, w.n_bins, 2))
    return oracle.EventHolder(data, psd, w.f_min, w.df, dets)


def snr(w, model, theta):
    ev0 = oracle_event(w)
    lnl = oracle.loglike(model, ev0, theta, grad=False)
    return math.sqrt(-2.0 * lnl[0])


def injection(w: inputs.Workload, seed=0):
    """Injected parameters with the distance rescaled to the target SNR."""
    model = oracle_model(w)
    th = inputs.injection(w, seed).copy()
    k = inputs.distance_index(w)
    if w.snr_target is not None and k is not None:
        rho = snr(w, model, th)
        th[k] = min(max(th[k] * rho / w.snr_target, w.lo[k]), w.hi[k])
    return th


def make_event(w: inputs.Workload, seed=0, with_noise=True):
    """(EventHolder, theta_inj, data) with data = h(theta_inj) + noise."""
    model = oracle_model(w)
    th = injection(w, seed)
    ev0 = oracle_event(w)
    h = oracle.waveform(model, ev0, th)
    data = h + (inputs.noise(w, seed) if with_noise else 0.0)
    return oracle_event(w, data=data), th, data
