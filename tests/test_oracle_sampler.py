"""Pins for the oracle's sampler: analytic evidences, NUTS stationarity and a
quadrature evidence on a 2-parameter slice of the tiny TaylorF2 workload."""
import math

import numpy as np
import pytest
from scipy import special, stats

import oracle
from paper_2601_02336_gb300 import inputs
from tests import helpers


def _box_mass(mu, sig, lo, hi):
    return 0.5 * (special.erf((hi - mu) / (sig * math.sqrt(2))) - special.erf((lo - mu) / (sig * math.sqrt(2))))


def gauss_lnz(beta, mu, sig, lo, hi):
    """ln int N(x; mu, sig^2)^beta pi(x) dx with a uniform prior on the box (closed form per dim)."""
    out = 0.0
    for m, s, a, b in zip(mu, sig, lo, hi):
        out += (-0.5 * beta * math.log(2 * math.pi * s * s) + 0.5 * math.log(2 * math.pi * s * s / beta)
                + math.log(_box_mass(m, s / math.sqrt(beta), a, b)) - math.log(b - a))
    return out


@pytest.mark.parametrize("metric", [0, 1, 2])
def test_smc_gaussian_evidence(metric):
    """Gaussian likelihood, uniform box prior: ln Z and every stage's ln Z_beta against the closed
    form (Sec. 3.1 Eqs. 7-8), over 8 seeds."""
    mu, sig = [1.0, -2.0, 0.5], [0.5, 1.0, 0.3]
    lo, hi = [-10.0] * 3, [10.0] * 3
    model = helpers.gaussmix_model(lo, hi, [0.0], [mu], [sig])
    truth = gauss_lnz(1.0, mu, sig, lo, hi)
    lnzs, stage_dev = [], []
    for seed in range(8):
        lnz, th, lnl, rec = oracle.smc_run(model, None, 512, 0.5, 2, 5, metric, 0.5, key=100 + seed)
        lnzs.append(lnz)
        cum = np.cumsum([r["dlnz"] for r in rec])
        for r, c in zip(rec, cum):
            stage_dev.append(c - gauss_lnz(r["beta"], mu, sig, lo, hi))
        # final particles follow the posterior
        assert np.allclose(th.mean(0), mu, atol=0.15)
        assert np.allclose(th.std(0), sig, rtol=0.25)
    lnzs = np.array(lnzs)
    se = lnzs.std(ddof=1) / math.sqrt(len(lnzs))
    assert abs(lnzs.mean() - truth) < 4 * se + 0.02, (lnzs.mean(), truth, se)
    assert abs(np.mean(stage_dev)) < 0.1


def test_smc_bimodal_evidence():
    """Two-component mixture in 3-D (the 11-D mixture of App. A, Eq. A1, in a smaller box):
    both normalised components give Z = 2 / volume."""
    d = 3
    lo, hi = [-5.0] * d, [5.0] * d
    model = helpers.gaussmix_model(lo, hi, [0.0, 0.0], [[1.0] * d, [-1.0] * d], [[0.3] * d, [0.3] * d])
    truth = math.log(2.0) - d * math.log(10.0)
    lnzs = []
    for seed in range(6):
        lnz, th, lnl, rec = oracle.smc_run(model, None, 1024, 0.5, 2, 6, 1, 0.5, key=300 + seed)
        lnzs.append(lnz)
        frac = np.mean(th[:, 0] > 0)
        assert 0.3 < frac < 0.7
    lnzs = np.array(lnzs)
    se = lnzs.std(ddof=1) / math.sqrt(len(lnzs))
    assert abs(lnzs.mean() - truth) < 4 * se + 0.03


@pytest.mark.parametrize("dense", [False, True])
def test_nuts_stationarity(dense):
    """Start 20000 independent chains exactly at the target (N(0,1) per dim, box [-10,10]) and apply
    one NUTS transition: the output must still follow the target (KS test per coordinate)."""
    d = 2
    model = helpers.gaussmix_model([-10.0] * d, [10.0] * d, [0.0], [[0.0] * d], [[1.0, 0.3]])
    rng = np.random.default_rng(8)
    n = 20000
    th = rng.standard_normal((n, d)) * np.array([1.0, 0.3])
    lnl, g = oracle.loglike(model, None, th)
    inv_mass = np.array([[1.0, 0.1], [0.1, 0.09]]) if dense else None
    eps = 0.6 if dense else 0.25
    out, l2, g2, st = oracle.nuts_mutate(model, None, 1.0, th, lnl, g, inv_mass, eps, 8, 1, key=9, ctr=0)
    assert stats.kstest(out[:, 0], "norm").pvalue > 1e-3
    assert stats.kstest(out[:, 1] / 0.3, "norm").pvalue > 1e-3
    assert np.mean(st["n_leapfrog"]) > 1.5
    assert np.mean(np.abs(out - th)) > 0.1  # the chains moved
    # returned ln L / grad belong to the returned positions
    l3, g3 = oracle.loglike(model, None, out)
    assert np.allclose(l2, l3, rtol=1e-12, atol=1e-12) and np.allclose(g2, g3, rtol=1e-12, atol=1e-12)


def test_nuts_subset_by_ensemble_index():
    """A particle's transition depends on its position and its index in the ensemble only (the index names
    its random numbers): rows run alone with their indices give the ensemble run's rows exactly, and the
    same rows under other indices give other transitions."""
    d = 2
    model = helpers.gaussmix_model([-10.0] * d, [10.0] * d, [0.0], [[0.0] * d], [[1.0, 0.3]])
    th = np.random.default_rng(12).standard_normal((300, d)) * np.array([1.0, 0.3])
    lnl, g = oracle.loglike(model, None, th)
    full = oracle.nuts_mutate(model, None, 1.0, th, lnl, g, None, 0.25, 6, 2, key=4, ctr=7)
    ids = np.array([299, 0, 17, 150, 151])
    sub = oracle.nuts_mutate(model, None, 1.0, th[ids], lnl[ids], g[ids], None, 0.25, 6, 2, key=4, ctr=7, ids=ids)
    for a, b in zip(sub[:3], full[:3]):
        assert np.array_equal(a, b[ids])
    assert np.array_equal(sub[3]["n_leapfrog"], full[3]["n_leapfrog"][ids])
    other = oracle.nuts_mutate(model, None, 1.0, th[ids], lnl[ids], g[ids], None, 0.25, 6, 2, key=4, ctr=7,
                               ids=ids + 1)
    assert not np.array_equal(other[0], full[0][ids])


def test_nuts_per_particle_metric_stationarity():
    """Each particle with its own (random, fixed) dense metric: one transition from the target still
    yields the target (KS per coordinate)."""
    d = 2
    model = helpers.gaussmix_model([-10.0] * d, [10.0] * d, [0.0], [[0.0] * d], [[1.0, 0.3]])
    rng = np.random.default_rng(18)
    n = 20000
    th = rng.standard_normal((n, d)) * np.array([1.0, 0.3])
    lnl, g = oracle.loglike(model, None, th)
    a = rng.standard_normal((n, d, d)) * 0.5
    minv = np.einsum("nij,nkj->nik", a, a) + np.diag([0.5, 0.05])[None]
    out, l2, g2, st = oracle.nuts_mutate_local(model, None, 1.0, th, lnl, g, minv, 0.4, 8, 1, key=19, ctr=0)
    assert stats.kstest(out[:, 0], "norm").pvalue > 1e-3
    assert stats.kstest(out[:, 1] / 0.3, "norm").pvalue > 1e-3
    assert np.mean(np.abs(out - th)) > 0.1


def test_nuts_long_chain_moments():
    """1-D N(0,1): 200 chains x 500 transitions, mean 0 and variance 1 within Monte-Carlo error."""
    model = helpers.gaussmix_model([-10.0], [10.0], [0.0], [[0.0]], [[1.0]])
    n = 200
    th = np.zeros((n, 1))
    lnl, g = oracle.loglike(model, None, th)
    draws = []
    for t in range(500):
        th, lnl, g, st = oracle.nuts_mutate(model, None, 1.0, th, lnl, g, None, 0.5, 8, 1, key=11, ctr=t)
        if t >= 20:
            draws.append(th[:, 0].copy())
    x = np.array(draws).ravel()
    assert abs(x.mean()) < 0.02
    assert abs(x.var() - 1.0) < 0.03


def test_reflective_boundary_keeps_target():
    """Target N(0,1) truncated to [-0.5, 2]: chains started at the truncated target stay there
    (reflection at the walls preserves the distribution)."""
    model = helpers.gaussmix_model([-0.5], [2.0], [0.0], [[0.0]], [[1.0]])
    a, b = -0.5, 2.0
    dist = stats.truncnorm(a, b)
    th = dist.rvs(size=(20000, 1), random_state=np.random.default_rng(12))
    lnl, g = oracle.loglike(model, None, th)
    out, *_ = oracle.nuts_mutate(model, None, 1.0, th, lnl, g, None, 0.9, 6, 1, key=13, ctr=0)
    assert np.all(out >= a) and np.all(out <= b)
    assert stats.kstest(out[:, 0], dist.cdf).pvalue > 1e-3


def test_periodic_boundary_keeps_target():
    """Von-Mises-like target on a circle built from a wide Gaussian on a periodic coordinate:
    uniform target (flat likelihood) stays uniform under wrapping."""
    model = helpers.gaussmix_model([0.0], [2 * math.pi], [0.0], [[0.0]], [[1e6]], boundary=[1])
    th = np.random.default_rng(14).uniform(0, 2 * math.pi, size=(20000, 1))
    lnl, g = oracle.loglike(model, None, th)
    out, *_ = oracle.nuts_mutate(model, None, 1.0, th, lnl, g, None, 2.5, 4, 1, key=15, ctr=0)
    assert np.all(out >= 0) and np.all(out < 2 * math.pi)
    assert stats.kstest(out[:, 0] / (2 * math.pi), "uniform").pvalue > 1e-3
    assert np.mean(np.abs(out - th)) > 0.5


def _slice_model(w):
    fixed = list(w.fixed)
    fixed[inputs.Q] = 0.75
    fixed[inputs.PHIC] = math.pi
    return oracle.make_model(oracle.KIND_GW, [inputs.MC, inputs.TC], [10.0, -0.05], [12.0, 0.05],
                             [0, 0], [0, 0], fixed)


def _quadrature_lnz(model, ev):
    """Coarse scan of the whole box, then a fine tensor grid over the region within 40 of the peak."""
    def grid(mc0, mc1, tc0, tc1, n):
        mc = np.linspace(mc0, mc1, n)
        tc = np.linspace(tc0, tc1, n)
        M, T = np.meshgrid(mc, tc, indexing="ij")
        lnl = oracle.loglike(model, ev, np.stack([M.ravel(), T.ravel()], 1), grad=False).reshape(n, n)
        return mc, tc, lnl
    mc, tc, lnl = grid(10.0, 12.0, -0.05, 0.05, 401)
    mx = lnl.max()
    idx = np.argwhere(lnl > mx - 40)
    dm, dt = mc[1] - mc[0], tc[1] - tc[0]
    box = (max(10.0, mc[idx[:, 0].min()] - 3 * dm), min(12.0, mc[idx[:, 0].max()] + 3 * dm),
           max(-0.05, tc[idx[:, 1].min()] - 3 * dt), min(0.05, tc[idx[:, 1].max()] + 3 * dt))
    outs = []
    for n in (301, 601):
        a, b, l = grid(*box, n)
        m = l.max()
        outs.append(m + math.log(np.trapezoid(np.trapezoid(np.exp(l - m), b, axis=1), a)) - math.log(2.0 * 0.1))
    return outs


def test_smc_quadrature_slice():
    """ln Z of the tiny workload's data on the (M_c, t_c) slice (q = 0.75, phi_c = pi fixed):
    SMC (dense covariance metric, alpha 0.8, 6 transitions per stage so that the oscillatory
    likelihood is well mixed) against 2-D quadrature, over 6 seeds."""
    w = inputs.tiny()
    ev, th_inj, _ = helpers.make_event(w, seed=0)
    model = _slice_model(w)
    q1, q2 = _quadrature_lnz(model, ev)
    assert abs(q1 - q2) < 1e-3
    lnzs = np.array([oracle.smc_run(model, ev, 512, 0.8, 6, 6, 1, 0.5, key=500 + seed)[0] for seed in range(6)])
    se = lnzs.std(ddof=1) / math.sqrt(len(lnzs))
    assert se < 0.5
    assert abs(lnzs.mean() - q2) < 3 * se + 0.05, (lnzs, q2)
