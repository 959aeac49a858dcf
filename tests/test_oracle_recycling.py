"""Pins for the oracle's sample recycling (Sec. 5, "Samples recycling"): a pool
of particles from all stages, particle of stage t drawn from
p_t = L^beta_t pi / Z_t, reweighted to the final target through the mixture
(1/T) sum_t p_t, then rejection-sampled to i.i.d. draws."""
import math

import numpy as np
from scipy import stats

import oracle


def test_single_stage_weights_are_flat():
    """T = 1, beta = 1: the mixture is the target itself, every weight is 1 and every particle is kept."""
    lnl = np.random.default_rng(0).normal(-50.0, 10.0, size=500)
    lw = oracle.recycle_weights(lnl, np.array([1.0]), np.array([-7.25]))
    assert np.allclose(lw, 0.0, atol=1e-12)
    assert oracle.rejection_sample(lw, 3).sum() == 500


def _gaussian_ladder(mu, sig, betas, n_per, seed, half_width=50.0):
    """Exact draws from p_t = N(mu, sig^2 / beta_t) (L = exp(-(x - mu)^2 / (2 sig^2)), flat prior on
    [-half_width, half_width], far wider than every p_t) and the closed-form ln Z_t."""
    rng = np.random.default_rng(seed)
    xs, lnz = [], []
    for b in betas:
        xs.append(rng.normal(mu, sig / math.sqrt(b), size=n_per))
        lnz.append(0.5 * math.log(2.0 * math.pi * sig * sig / b) - math.log(2.0 * half_width))
    x = np.concatenate(xs)
    lnl = -0.5 * (x - mu) ** 2 / sig ** 2
    return x, lnl, np.array(lnz)


def test_gaussian_ladder_recovers_target():
    """Pool drawn exactly from a Gaussian ladder: E_pool[w] = 1 (normalisation by Z_t and 1/T), the weighted
    moments are the target's, and the kept draws follow the target (KS)."""
    mu, sig = 0.7, 0.3
    betas = np.array([0.01, 0.04, 0.15, 0.4, 1.0])
    n_per = 40000
    x, lnl, lnz = _gaussian_ladder(mu, sig, betas, n_per, seed=1)
    lw = oracle.recycle_weights(lnl, betas, lnz)
    w = np.exp(lw)
    m = len(w)
    assert abs(w.mean() - 1.0) < 4 * w.std() / math.sqrt(m)
    wn = w / w.sum()
    mean = float((wn * x).sum())
    var = float((wn * (x - mean) ** 2).sum())
    ess = 1.0 / float((wn ** 2).sum())
    assert abs(mean - mu) < 5 * sig / math.sqrt(ess)
    assert abs(var / sig ** 2 - 1.0) < 5 * math.sqrt(2.0 / ess)
    keep = oracle.rejection_sample(lw, 11).astype(bool)
    kept = x[keep]
    assert keep.sum() > n_per  # more i.i.d. draws than the last stage alone holds
    assert abs(keep.mean() - w.mean() / w.max()) < 5 * math.sqrt(keep.mean() / m)
    assert stats.kstest((kept - mu) / sig, "norm").pvalue > 1e-3


def test_weights_invariant_to_likelihood_offset():
    """ln L -> ln L + c with ln Z_t -> ln Z_t + beta_t c leaves every weight unchanged."""
    rng = np.random.default_rng(2)
    lnl = rng.normal(-30.0, 5.0, size=1000)
    betas = np.array([0.1, 0.3, 1.0])
    lnz = np.array([-2.0, -4.5, -9.0])
    c = 123.25
    a = oracle.recycle_weights(lnl, betas, lnz)
    b = oracle.recycle_weights(lnl + c, betas, lnz + betas * c)
    assert np.allclose(a, b, rtol=0, atol=1e-9)


def test_weights_brute_force_small():
    """Three particles, two stages: the weight written out by hand."""
    lnl = np.array([-1.0, -2.5, -0.25])
    betas = np.array([0.5, 1.0])
    lnz = np.array([-0.8, -1.9])
    lw = oracle.recycle_weights(lnl, betas, lnz)
    for i in range(3):
        mix = 0.5 * (math.exp(0.5 * lnl[i] + 0.8) + math.exp(lnl[i] + 1.9))
        expect = math.log(math.exp(lnl[i] + 1.9) / mix)
        assert abs(lw[i] - expect) < 1e-13
