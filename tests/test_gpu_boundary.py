"""Boundary calls against the oracle and the failure-detection bound.

- sharpy_prior_sample: the same Philox uniforms (key, counter (particle, ctr,
  1, dimension)) and the same transforms as the oracle's prior draw (Sec. 5
  priors: uniform boxes, d_L ~ d^2). The kernel may contract x = lo + u w into
  an FMA and its cube root rounds differently from the host's, so positions
  agree to a few ulp rather than bit for bit.
- sharpy_prior_logpdf_grad: ln pi and its gradient, -inf outside the box.
- sharpy_nuts_mutate_cov_step: the identity-metric step rule computed on the
  device equals sharpy_nuts_mutate with that step computed on the host.
- sharpy_set_nuts_tick_limit: a lowered tick bound ends the persistent NUTS
  launch with SHARPY_ETIMEOUT in the status word and a valid written-back
  state; nothing faults and the context stays usable.
- stage records carry the device-accumulated running ln Z.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2601_02336_gb300 import _lib, api, inputs
from tests import gpu_helpers as G
from tests import helpers

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("wname", ["tiny", "bbh11"])
def test_prior_sample_matches_oracle(wname):
    G.require_gpu()
    w = getattr(inputs, wname)()
    ctx = api.Context.from_workload(w)
    model = helpers.oracle_model(w)
    for key, ctr, n in ((11, 0, 4099), (2 ** 40 + 5, 7, 333)):
        got = ctx.prior_sample(n, key, ctr).cpu().numpy()
        ref = oracle.prior_sample(model, n, key, ctr)
        lo, hi = np.array(w.lo), np.array(w.hi)
        # rounding of lo + u (hi - lo) (fused or not) is an ulp of the box's scale, not of x near 0
        ulp = np.spacing(np.maximum(np.abs(ref), np.maximum(np.abs(lo), np.abs(hi))[None, :]))
        assert np.all(np.abs(got - ref) <= 4 * ulp), np.max(np.abs(got - ref) / ulp)
        assert np.all(got >= lo) and np.all(got <= hi)


def test_prior_logpdf_grad_matches_oracle():
    G.require_gpu()
    w = inputs.bbh11()
    ctx = api.Context.from_workload(w)
    model = helpers.oracle_model(w)
    th = inputs.prior_draws(w, 1000, 3)
    th[:5, 4] = [100.0, 5000.0, 101.5, 4999.0, 2500.0]  # the d^2 prior's ends
    th[5, 0] = w.lo[0] - 1e-9                            # outside the box
    th[6, 4] = w.hi[4] * 1.01
    lp_g, g_g = ctx.prior_logpdf_grad(G.to_dev(th))
    lp_o, g_o = oracle.prior_logpdf_grad(model, th)
    lp_g, g_g = lp_g.cpu().numpy(), g_g.cpu().numpy()
    assert np.all(np.isneginf(lp_g[5:7])) and np.all(np.isneginf(lp_o[5:7]))
    fin = np.isfinite(lp_o)
    assert np.array_equal(fin, np.isfinite(lp_g))
    np.testing.assert_allclose(lp_g[fin], lp_o[fin], rtol=1e-14, atol=1e-13)
    np.testing.assert_allclose(g_g[fin], g_o[fin], rtol=1e-14, atol=1e-300)


def test_nuts_mutate_cov_step_equals_host_step():
    G.require_gpu()
    w = inputs.tiny()
    ev, ctx, th_inj, _ = G.event_pair(w)
    n = 512
    th0 = inputs.ball(w, th_inj, n, 5)
    lnl0, g0 = ctx.loglike_grad(G.to_dev(th0), "fp64")
    wts = np.random.default_rng(4).uniform(0.1, 1.0, n)
    cov = oracle.weighted_cov(th0, wts)
    cov_d = G.to_dev(cov)
    outs = []
    for mode in ("device", "host"):
        t, l, g = G.to_dev(th0), lnl0.clone(), g0.clone()
        if mode == "device":
            ctx.nuts_mutate_cov_step(0.7, t, l, g, cov_d, 0.5, 5, 2, key=3, ctr=9, precision="fp64")
        else:
            eps = 0.5 * float(np.sqrt(np.diag(cov)).min())
            ctx.nuts_mutate(0.7, t, l, g, None, eps, 5, 2, key=3, ctr=9, precision="fp64")
        outs.append((t, l, g))
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)
    assert ctx.status() == 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nuts_tick_limit_reports_timeout(precision):
    """Failure detection without a fault: the NUTS kernel's loop bound, lowered to a few ticks,
    stops the launch, records SHARPY_ETIMEOUT and writes back each particle's current proposal,
    a point of its own trajectory with that point's ln L; the default bound then runs clean."""
    G.require_gpu()
    w = inputs.tiny()
    ev, ctx, th_inj, _ = G.event_pair(w)
    model = helpers.oracle_model(w)
    n = 256
    th0 = inputs.prior_draws(w, n, 8)
    lnl0, g0 = ctx.loglike_grad(G.to_dev(th0), "fp64")
    ctx.clear_status()
    ctx.set_nuts_tick_limit(3)
    t, l, g = G.to_dev(th0), lnl0.clone(), g0.clone()
    # a short step: trees grow to the depth limit (31 leapfrogs a transition), far beyond the bound
    st = api.Context.stats_to_numpy(ctx.nuts_mutate(0.5, t, l, g, None, 2e-5, 5, 2, key=5, ctr=1,
                                                    precision=precision))
    assert ctx.status() == _lib.ETIMEOUT
    th = t.cpu().numpy()
    assert np.all(np.isfinite(th)) and np.all(th >= np.array(w.lo)) and np.all(th <= np.array(w.hi))
    # at most one evaluated leaf per tick (ticks 0..3), plus leaves that diverge at the box edge
    # without an evaluation
    assert st["n_leapfrog"].max() <= 8
    lref = oracle.loglike(model, ev, th, grad=False)
    np.testing.assert_allclose(l.cpu().numpy(), lref, rtol=1e-6, atol=1e-3)
    ctx.clear_status()
    ctx.set_nuts_tick_limit(0)
    t, l, g = G.to_dev(th0), lnl0.clone(), g0.clone()
    st = api.Context.stats_to_numpy(ctx.nuts_mutate(0.5, t, l, g, None, 2e-5, 5, 2, key=5, ctr=1,
                                                    precision=precision))
    assert ctx.status() == 0
    assert st["n_leapfrog"].max() > 8


def test_stage_records_carry_running_lnz():
    G.require_gpu()
    w = inputs.tiny()
    ctx = api.make_event(w, seed=0)[0]
    lnz, th, ll, rec = ctx.smc_run(w.n_particles, w.alpha, w.n_mut, w.max_depth, w.metric, w.eps_scale, key=17,
                                   precision="mixed")
    run = 0.0
    for r in rec:
        run += r["dlnz"]
        assert r["lnz"] == pytest.approx(run, rel=1e-13, abs=1e-12)
    assert rec[-1]["lnz"] == lnz
