"""Persistent GPU NUTS against the oracle's NUTS (same Philox key and counters).

With FP64 arithmetic on both sides a transition follows the same trajectory
up to rounding, so the returned positions agree closely unless a random
acceptance or a U-turn test sits within rounding of its threshold, or the
dynamics amplify rounding (chaotic trajectories on the oscillatory TaylorF2
likelihood): at least 95 % of particles (99 % on Gaussian targets) must match
to 1e-7 in prior-width units with identical leapfrog counts, and every
returned (theta, ln L, grad) must be self-consistent.
"""
import math

import numpy as np
import pytest
import torch
from scipy import stats

import oracle
from paper_2601_02336_gb300 import api, inputs
from tests import gpu_helpers as G
from tests import helpers

pytestmark = pytest.mark.gpu


def _gm(d=3, dense=False):
    lo, hi = [-6.0] * d, [6.0] * d
    mu = [[0.5 * i for i in range(d)], [-1.0] * d]
    sig = [[1.0 + 0.2 * i for i in range(d)], [0.3] * d]
    cfg = api.gaussmix_config(lo, hi, [np.log(0.7), np.log(0.3)], mu, sig, [0] * (d - 1) + [1])
    model = helpers.gaussmix_model(lo, hi, [np.log(0.7), np.log(0.3)], mu, sig, [0] * (d - 1) + [1])
    return cfg, model, np.array(hi) - np.array(lo)


def _compare(th_g, l_g, st_g, th_o, l_o, g_o, st_o, wid, frac=0.95, tol=1e-7, lf_frac=1.0):
    dev = np.max(np.abs(th_g - th_o) / wid[None, :], axis=1)
    match = dev < tol
    assert match.mean() >= frac, (match.mean(), np.sort(dev)[-5:])
    same_lf = st_g["n_leapfrog"][match] == st_o["n_leapfrog"][match]
    assert same_lf.mean() >= lf_frac, same_lf.mean()
    # ln L differs by summation order (~1e-7) plus grad . (theta_gpu - theta_oracle)
    slack = 1e-6 + 1e-9 * np.abs(l_o) + 2.0 * np.abs(np.sum(g_o * (th_g - th_o), axis=1))
    assert np.all(np.abs(l_g - l_o)[match] <= slack[match])
    return match


@pytest.mark.parametrize("dense", [False, True])
def test_nuts_gaussmix_matches_oracle(dense):
    G.require_gpu()
    cfg, model, wid = _gm(3)
    ctx = api.Context(cfg)
    n = 1000
    th = np.random.default_rng(1).uniform(-3, 3, size=(n, 3))
    lnl, g = oracle.loglike(model, None, th)
    minv = np.array([[1.0, 0.2, 0.0], [0.2, 0.8, 0.1], [0.0, 0.1, 0.5]]) if dense else None
    for beta in (0.3, 1.0):
        ref = oracle.nuts_mutate(model, None, beta, th, lnl, g, minv, 0.4, 6, 2, key=21, ctr=5)
        t, l, gg = G.to_dev(th), G.to_dev(lnl), G.to_dev(g)
        st = ctx.nuts_mutate(beta, t, l, gg, G.to_dev(minv) if dense else None, 0.4, 6, 2, key=21, ctr=5,
                             precision="fp64")
        st = api.Context.stats_to_numpy(st)
        _compare(t.cpu().numpy(), l.cpu().numpy(), st, ref[0], ref[1], ref[2], ref[3], wid, frac=0.99)
        # returned ln L / gradient belong to the returned positions
        l2, g2 = oracle.loglike(model, None, t.cpu().numpy())
        assert np.allclose(l.cpu().numpy(), l2, rtol=1e-12, atol=1e-12)
        assert np.allclose(gg.cpu().numpy(), g2, rtol=1e-10, atol=1e-12)


def test_nuts_taylorf2_fp64_matches_oracle():
    G.require_gpu()
    w = inputs.tiny()
    ev, ctx, th_inj, _ = G.event_pair(w)
    model = helpers.oracle_model(w)
    n = 100
    th = np.vstack([inputs.ball(w, th_inj, n // 2, 3, rel=2e-3), inputs.prior_draws(w, n - n // 2, 4)])
    lnl, g = oracle.loglike(model, ev, th)
    wid = G.width(w)
    for beta, eps in [(0.05, 2e-3), (1.0, 2e-4)]:
        ref = oracle.nuts_mutate(model, ev, beta, th, lnl, g, None, eps, 5, 2, key=33, ctr=17)
        t, l, gg = G.to_dev(th), G.to_dev(lnl), G.to_dev(g)
        st = api.Context.stats_to_numpy(ctx.nuts_mutate(beta, t, l, gg, None, eps, 5, 2, key=33, ctr=17,
                                                        precision="fp64"))
        _compare(t.cpu().numpy(), l.cpu().numpy(), st, ref[0], ref[1], ref[2], ref[3], wid)
        assert st["active_bins"].sum() > 0


@pytest.mark.parametrize("precision", ["mixed", "split"])
def test_nuts_taylorf2_11d_mixed_vs_fp64(precision):
    """The mixed sweeps change H by ~1e-4 at most, so most trajectories stay identical to the FP64 ones."""
    G.require_gpu()
    w = inputs.bbh11()
    ev, ctx, th_inj, _ = G.event_pair(w)
    n = 256
    th = inputs.ball(w, th_inj, n, 9, rel=1e-4)
    t0 = G.to_dev(th)
    l0, g0 = ctx.loglike_grad(t0, "fp64")
    out = {}
    for prec in ("fp64", precision):
        t, l, g = t0.clone(), l0.clone(), g0.clone()
        st = ctx.nuts_mutate(0.7, t, l, g, None, 1e-5, 6, 2, key=5, ctr=1, precision=prec)
        out[prec] = (t.cpu().numpy(), l.cpu().numpy(), api.Context.stats_to_numpy(st))
    dev = np.max(np.abs(out["fp64"][0] - out[precision][0]) / G.width(w)[None, :], axis=1)
    assert np.mean(dev < 1e-6) >= 0.8
    assert np.all(np.isfinite(out[precision][0]))
    # the returned ln L belongs to the returned theta: against the FP64 value within the mixed tolerance, and
    # against the standalone mixed call (the same sweep code) to rounding
    th_m = G.to_dev(out[precision][0])
    l64, _ = ctx.loglike_grad(th_m, "fp64")
    l2, _ = ctx.loglike_grad(th_m, precision)
    assert np.max(np.abs(l64.cpu().numpy() - out[precision][1])) <= 1e-3
    assert np.max(np.abs(l2.cpu().numpy() - out[precision][1])) <= 1e-6
    assert ctx.status() == 0


def test_nuts_stationarity_gpu():
    """Chains started exactly at N(0, diag) stay there after one GPU transition (KS per coordinate)."""
    G.require_gpu()
    d = 2
    cfg = api.gaussmix_config([-10.0] * d, [10.0] * d, [0.0], [[0.0] * d], [[1.0, 0.3]])
    ctx = api.Context(cfg)
    n = 20000
    th = np.random.default_rng(8).standard_normal((n, d)) * np.array([1.0, 0.3])
    t = G.to_dev(th)
    l, g = ctx.loglike_grad(t)
    ctx.nuts_mutate(1.0, t, l, g, G.to_dev(np.array([[1.0, 0.1], [0.1, 0.09]])), 0.6, 8, 1, key=9, ctr=0,
                    precision="fp64")
    out = t.cpu().numpy()
    assert stats.kstest(out[:, 0], "norm").pvalue > 1e-3
    assert stats.kstest(out[:, 1] / 0.3, "norm").pvalue > 1e-3
    assert np.mean(np.abs(out - th)) > 0.1


def test_nuts_edge_cases():
    G.require_gpu()
    cfg, model, wid = _gm(2)
    ctx = api.Context(cfg)
    th = np.array([[0.1, 0.2], [5.9, -5.9], [0.0, 0.0]])
    t = G.to_dev(th)
    l, g = ctx.loglike_grad(t)
    # zero transitions and depth 0 leave the state untouched
    ctx.nuts_mutate(1.0, t, l, g, None, 0.5, 4, 0, key=1, ctr=0, precision="fp64")
    ctx.nuts_mutate(1.0, t, l, g, None, 0.5, 0, 3, key=1, ctr=0, precision="fp64")
    assert np.array_equal(t.cpu().numpy(), th)
    # a huge step is reflected back into the box
    ctx.nuts_mutate(1.0, t, l, g, None, 50.0, 3, 2, key=2, ctr=0, precision="fp64")
    out = t.cpu().numpy()
    assert np.all(out >= -6.0) and np.all(out <= 6.0)
    assert ctx.status() == 0


def test_nuts_per_particle_metric_gaussmix_matches_oracle():
    """One fixed dense metric per particle (the same input arrays on both sides)."""
    G.require_gpu()
    cfg, model, wid = _gm(3)
    ctx = api.Context(cfg)
    n = 800
    rng = np.random.default_rng(31)
    th = rng.uniform(-3, 3, size=(n, 3))
    lnl, g = oracle.loglike(model, None, th)
    a = rng.standard_normal((n, 3, 3)) * 0.3
    minv = np.einsum("nij,nkj->nik", a, a) + np.diag([0.6, 0.4, 0.3])[None]
    chol = np.linalg.cholesky(minv)
    ref = oracle.nuts_mutate_local(model, None, 0.7, th, lnl, g, minv, 0.4, 6, 2, key=23, ctr=3)
    t, l, gg = G.to_dev(th), G.to_dev(lnl), G.to_dev(g)
    st = ctx.nuts_mutate_local(0.7, t, l, gg, G.to_dev(minv), G.to_dev(chol), 0.4, 6, 2, key=23, ctr=3,
                               precision="fp64")
    _compare(t.cpu().numpy(), l.cpu().numpy(), api.Context.stats_to_numpy(st), ref[0], ref[1], ref[2], ref[3],
             wid, frac=0.99)


def test_nuts_local_metric_taylorf2_matches_oracle():
    """The local metric of Sec. 5 computed on each side (GPU: sharpy_local_metric; oracle: its Fisher
    information and an inverse), then one NUTS call with it. In physical units the mass matrix has a
    condition number near 1e10, so the two inverses agree only to ~1e-6 relative: an occasional U-turn test
    then falls differently (same end point, another leapfrog count)."""
    G.require_gpu()
    w = inputs.tiny()
    ev, ctx, th_inj, _ = G.event_pair(w)
    model = helpers.oracle_model(w)
    n = 100
    th = np.vstack([inputs.ball(w, th_inj, n // 2, 3, rel=2e-3), inputs.prior_draws(w, n - n // 2, 4)])
    lnl, g = oracle.loglike(model, ev, th)
    wid = G.width(w)
    for beta in (0.05, 1.0):
        minv_ref = np.linalg.inv(oracle.local_metric(model, ev, th, beta))
        ref = oracle.nuts_mutate_local(model, ev, beta, th, lnl, g, minv_ref, 0.5, 5, 2, key=35, ctr=9)
        t, l, gg = G.to_dev(th), G.to_dev(lnl), G.to_dev(g)
        met = ctx.local_metric(t, beta, want=("inv_mass", "chol"))
        st = ctx.nuts_mutate_local(beta, t, l, gg, met["inv_mass"], met["chol"], 0.5, 5, 2, key=35, ctr=9,
                                   precision="fp64")
        _compare(t.cpu().numpy(), l.cpu().numpy(), api.Context.stats_to_numpy(st), ref[0], ref[1], ref[2],
                 ref[3], wid, frac=0.9, lf_frac=0.9)


def _laplace_ensemble(w, model, ev, th_inj, beta, n, seed):
    """Synthetic SMC-like state on the 11-D event: the dense inverse mass matrix is the inverse of the
    oracle's local metric at the injection (Sec. 5); half the particles are drawn from N(theta_inj,
    0.01 M^-1) (folded into the box by clipping), half from the prior."""
    minv = np.linalg.inv(oracle.local_metric(model, ev, th_inj[None, :], beta)[0])
    minv = 0.5 * (minv + minv.T)
    lam, vec = np.linalg.eigh(minv)
    z = np.random.default_rng(seed).standard_normal((n // 2, w.n_dim))
    core = np.clip(th_inj + 0.1 * (z * np.sqrt(np.maximum(lam, 0.0))) @ vec.T, w.lo, w.hi)
    return np.vstack([core, inputs.prior_draws(w, n - n // 2, seed)]), minv


def test_nuts_bbh11_full_launch_sampled_parity():
    """The 11-D three-detector event at full size: one launch over 2048 particles (8 slots per CTA, 256
    CTAs: the geometry of the SMC run), depth 6, 2 transitions, a dense metric. Each particle's transition
    is named by its index in the ensemble, so the oracle runs 64 sampled particles on their own. The step
    gives trees that stop at a U-turn, at the depth limit and by divergence.

    FP64 path: the trajectories agree with the oracle's as in the small cases. Mixed path: its gradient
    differs from the FP64 one by ~1e-5 relative, and the 11-D dynamics amplify that over 63 leapfrogs, so
    its trajectories are not the oracle's row by row. It is checked for what holds at any size: every
    sampled returned state carries the oracle's ln L and gradient at its theta within the mixed-path
    tolerances, and the ensemble's tree statistics match the FP64 launch's."""
    G.require_gpu()
    w = inputs.bbh11()
    ev, ctx, th_inj, _ = G.event_pair(w)
    model = helpers.oracle_model(w)
    n, beta, eps = 2048, 0.5, 0.1
    th, minv = _laplace_ensemble(w, model, ev, th_inj, beta, n, 31)
    ids = np.sort(np.random.default_rng(5).choice(n, 64, replace=False))
    out = {}
    for prec in ("fp64", "mixed"):
        t = G.to_dev(th)
        l, g = ctx.loglike_grad(t, "fp64" if prec == "fp64" else prec)
        if prec == "fp64":
            l0, g0 = l.cpu().numpy(), g.cpu().numpy()
        st = api.Context.stats_to_numpy(ctx.nuts_mutate(beta, t, l, g, G.to_dev(minv), eps, 6, 2, key=43,
                                                        ctr=512, precision=prec))
        out[prec] = (t.cpu().numpy(), l.cpu().numpy(), g.cpu().numpy(), st)
        assert np.all(np.isfinite(out[prec][0])) and ctx.status() == 0
    ref = oracle.nuts_mutate(model, ev, beta, th[ids], l0[ids], g0[ids], minv, eps, 6, 2, key=43, ctr=512,
                             ids=ids)
    lf = ref[3]["n_leapfrog"]
    assert lf.min() < 20 and lf.max() == 126 and ref[3]["n_divergent"].sum() > 0  # all three tree endings
    th64, l64, _, st64 = out["fp64"]
    _compare(th64[ids], l64[ids], st64[ids], ref[0], ref[1], ref[2], ref[3], G.width(w), frac=0.9)
    thm, lm, gm, stm = out["mixed"]
    l2, g2 = oracle.loglike(model, ev, thm[ids])
    assert np.max(np.abs(lm[ids] - l2)) <= 1e-3, np.max(np.abs(lm[ids] - l2))
    assert np.max(G.grad_rel_err(gm[ids], g2, G.width(w))) <= 1e-4
    for f, tol in (("n_leapfrog", 0.1), ("accept_sum", 0.1), ("n_divergent", 0.25)):
        a, b = stm[f].astype(float).mean(), st64[f].astype(float).mean()
        assert abs(a - b) <= tol * b + 1e-3, (f, a, b)


def test_mixed_state_machine_energy_error_against_fp64():
    """The mixed path's NUTS state machine keeps momenta, velocities and log-weights in FP32 (positions and
    the potential energy in FP64). Its effect on the energy check, measured: from the same 2048 starts near
    the injection of the 11-D workload, one leapfrog per transition (max depth 1, so the acceptance statistic
    is min(1, e^-dH)), the mixed and FP64 kernels' energy errors dH agree to 1e-3 (four times the mixed path's
    ln L budget, which dominates: FP32 momenta move the kinetic energy by ~1e-6) at every particle where
    both are below 20; with full trees (depth 6, two transitions) the mean acceptance statistic, mean depth
    and leapfrog count agree within their Monte Carlo spread."""
    G.require_gpu()
    w = inputs.bbh11()
    ev, ctx, th_inj, _ = G.event_pair(w)
    n = 2048
    th = inputs.ball(w, th_inj, n, 21, rel=1e-3)
    t0 = G.to_dev(th)
    l0, g0 = ctx.loglike_grad(t0, "fp64")
    eps0 = float(np.min(np.std(th, axis=0)))
    for scale in (0.05, 0.3):
        dh = {}
        for prec in ("fp64", "mixed"):
            t, l, g = t0.clone(), l0.clone(), g0.clone()
            st = api.Context.stats_to_numpy(ctx.nuts_mutate(1.0, t, l, g, None, scale * eps0, 1, 1, key=31, ctr=2,
                                                            precision=prec))
            assert np.all(st["n_leapfrog"] == 1)
            acc = st["accept_sum"]
            dh[prec] = np.where(acc < 1.0, -np.log(np.maximum(acc, 1e-300)), 0.0)
        both = (dh["fp64"] < 20.0) & (dh["mixed"] < 20.0) & (dh["fp64"] > 0.0) & (dh["mixed"] > 0.0)
        assert both.sum() > 100
        assert np.max(np.abs(dh["mixed"][both] - dh["fp64"][both])) <= 1e-3
    stats_by = {}
    for prec in ("fp64", "mixed"):
        t, l, g = t0.clone(), l0.clone(), g0.clone()
        stats_by[prec] = api.Context.stats_to_numpy(ctx.nuts_mutate(1.0, t, l, g, None, 0.5 * eps0, 6, 2, key=32,
                                                                    ctr=3, precision=prec))
    for f in ("accept_sum", "depth_sum", "n_leapfrog"):
        a, b = stats_by["fp64"][f] / 2.0, stats_by["mixed"][f] / 2.0
        spread = 3.0 * math.sqrt(np.var(a) / n + np.var(b) / n)
        assert abs(np.mean(a) - np.mean(b)) <= spread + 1e-3, (f, np.mean(a), np.mean(b), spread)
    assert ctx.status() == 0


def test_nuts_long_signal_streams_match_oracle():
    """The 259585-bin segment: its sweeps (~2e5 bins a detector) are cut into streams that the warps of a NUTS
    tick share. FP64 path against the oracle's NUTS from the same 48 starts (same Philox counters), and the mixed
    path's returned ln L against the standalone likelihood call at the returned theta (the same streams and
    merge order: equal to rounding) and the FP64 value (long-signal tolerance)."""
    G.require_gpu()
    w = inputs.bns()
    ev, ctx, th_inj, _ = G.event_pair(w)
    model = helpers.oracle_model(w)
    n = 48
    th = inputs.ball(w, th_inj, n, 13, rel=1e-5)
    t0 = G.to_dev(th)
    l0, g0 = ctx.loglike_grad(t0, "fp64")
    step = 0.5 * float(np.min(np.std(th, axis=0)))
    ref = oracle.nuts_mutate(model, ev, 0.8, th, l0.cpu().numpy(), g0.cpu().numpy(), None, step, 3, 1, key=4, ctr=2)
    t, l, g = t0.clone(), l0.clone(), g0.clone()
    st = api.Context.stats_to_numpy(ctx.nuts_mutate(0.8, t, l, g, None, step, 3, 1, key=4, ctr=2, precision="fp64"))
    _compare(t.cpu().numpy(), l.cpu().numpy(), st, ref[0], ref[1], ref[2], ref[3], G.width(w), frac=0.9)
    t, l, g = t0.clone(), l0.clone(), g0.clone()
    ctx.nuts_mutate(0.8, t, l, g, None, step, 3, 1, key=4, ctr=2, precision="mixed")
    lm, _ = ctx.loglike_grad(t, "mixed")
    l64, _ = ctx.loglike_grad(t, "fp64")
    assert np.max(np.abs(lm.cpu().numpy() - l.cpu().numpy())) <= 1e-6 * max(1.0, float(l.abs().max()))
    assert np.max(np.abs(l64.cpu().numpy() - l.cpu().numpy())) <= 1e-2
    assert ctx.status() == 0


@pytest.mark.parametrize("wname,n,depth", [("bbh11", 300, 6), ("bbh11_long", 64, 4), ("bns", 48, 3)])
def test_nuts_outputs_equal_likelihood_call(wname, n, depth):
    """The NUTS kernel evaluates ln L and its gradient with the likelihood's own per-particle phases, sweeps and
    epilogue (on the long segment, streams shared by the warps of a tick; in the standalone call, the tuner's
    kernel, the staged one included): the ln L and gradient it returns equal sharpy_loglike_grad at the returned
    positions bit for bit, on every path and all three segment lengths."""
    G.require_gpu()
    w = getattr(inputs, wname)()
    ctx, th_inj, _ = api.make_event(w, seed=0)
    th = np.vstack([inputs.prior_draws(w, n // 2, 31), inputs.ball(w, th_inj, n - n // 2, 32, rel=1e-3)])
    t0 = G.to_dev(th)
    step = 0.5 * float(np.min(np.std(th, axis=0)))
    for prec in ("mixed", "split", "fp64"):
        l0, g0 = ctx.loglike_grad(t0, prec)
        t, l, g = t0.clone(), l0.clone(), g0.clone()
        ctx.nuts_mutate(0.3, t, l, g, None, step, depth, 2, key=41, ctr=3, precision=prec)
        assert not torch.equal(t, t0), prec
        lc, gc = ctx.loglike_grad(t, prec)
        assert torch.equal(lc, l) and torch.equal(gc, g), prec
    assert ctx.status() == 0


def test_nuts_slot_count_invariant():
    """The slot count per CTA (sharpy_set_nuts_slots: 4, 8, 16, 32) changes how a CTA schedules its particles'
    sweeps and state machines, never what a particle computes: positions, ln L, gradients and the transition
    statistics are bit-identical, on the 11-D workload from prior draws at a small beta (deep trees, reflections at
    the box) and near the injection."""
    G.require_gpu()
    w = inputs.bbh11()
    ev, ctx, th_inj, _ = G.event_pair(w)
    n = 300  # ragged last CTA for every slot count
    th = np.vstack([inputs.prior_draws(w, n // 2, 31), inputs.ball(w, th_inj, n - n // 2, 32, rel=1e-3)])
    t0 = G.to_dev(th)
    l0, g0 = ctx.loglike_grad(t0, "mixed")
    step = 0.5 * float(np.min(np.std(th, axis=0)))
    ref = None
    for slots in (8, 4, 16, 32):
        ctx.set_nuts_slots(slots)
        t, l, g = t0.clone(), l0.clone(), g0.clone()
        st = api.Context.stats_to_numpy(ctx.nuts_mutate(0.01, t, l, g, None, step, 6, 2, key=41, ctr=3,
                                                        precision="mixed"))
        out = (t, l, g, st)
        if ref is None:
            ref = out
            continue
        assert torch.equal(t, ref[0]) and torch.equal(l, ref[1]) and torch.equal(g, ref[2]), slots
        for f in ("accept_sum", "depth_sum", "n_leapfrog", "n_divergent", "active_bins"):
            assert np.array_equal(st[f], ref[3][f]), (slots, f)
    ctx.set_nuts_slots(0)
    assert ctx.status() == 0
