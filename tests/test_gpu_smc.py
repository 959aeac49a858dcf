"""GPU SMC stage kernels against the oracle: bit-exact systematic resampling,
tempering increment, ESS, evidence increment, covariance and gather."""
import numpy as np
import pytest
import torch

import oracle
from paper_2601_02336_gb300 import api, inputs
from tests import gpu_helpers as G
from tests import helpers

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 1000, 2048, 65537])
def test_systematic_bit_exact(n):
    G.require_gpu()
    rng = np.random.default_rng(n)
    for trial in range(5):
        w = rng.uniform(0, 1, n) ** rng.uniform(0.5, 8)
        w[rng.uniform(size=n) < 0.2] = 0.0
        w[rng.integers(n)] = 1.0
        u = float(rng.uniform())
        ref = oracle.systematic_resample(w, u)
        got = api.systematic_resample(G.to_dev(w), u).cpu().numpy()
        assert np.array_equal(got, ref), (n, trial)


def test_systematic_edges():
    G.require_gpu()
    w = np.array([0.0, 1.0, 0.0, 0.5])
    for u in (0.0, 0.25, 0.999999999):
        assert np.array_equal(api.systematic_resample(G.to_dev(w), u).cpu().numpy(),
                              oracle.systematic_resample(w, u))
    with pytest.raises(Exception):
        api.systematic_resample(G.to_dev(np.array([0.5, 1.5])), 0.1)  # weight outside [0, 1]


@pytest.mark.parametrize("n", [1, 64, 2048, 16384])
def test_reweight_resample_matches_oracle(n):
    G.require_gpu()
    w = inputs.bbh11()
    ctx = api.Context.from_workload(w)
    rng = np.random.default_rng(100 + n)
    th = inputs.prior_draws(w, n, 7)
    lnl = -0.5 * rng.chisquare(11, size=n) * 40.0 - 2.0e4
    grad = rng.normal(size=(n, w.n_dim))
    for beta_prev, alpha in [(0.0, 0.5), (0.3, 0.9), (0.9999, 0.5)]:
        bn, dl, ess, wts = oracle.smc_reweight(lnl, beta_prev, alpha)
        cov_ref = oracle.weighted_cov(th, wts)
        u = float(rng.uniform())
        anc_ref = oracle.systematic_resample(wts, u)
        t, l, g = G.to_dev(th), G.to_dev(lnl), G.to_dev(grad)
        out = ctx.reweight_resample(t, l, g, beta_prev, alpha, u)
        torch.cuda.synchronize()
        # the oracle bisects to adjacent doubles; the GPU's Newton stops at 1e-13 relative
        assert float(out["beta_next"]) == pytest.approx(bn, rel=1e-11, abs=1e-15)
        assert float(out["ess"]) == pytest.approx(ess, rel=1e-9)
        assert float(out["dlnz"]) == pytest.approx(dl, rel=1e-10, abs=1e-10)
        anc = out["ancestors"].cpu().numpy()
        assert np.array_equal(anc, anc_ref)
        assert np.allclose(out["cov"].cpu().numpy(), cov_ref, rtol=1e-9, atol=1e-12 * np.abs(cov_ref).max())
        assert np.array_equal(t.cpu().numpy(), th[anc_ref])
        assert np.array_equal(l.cpu().numpy(), lnl[anc_ref])
        assert np.array_equal(g.cpu().numpy(), grad[anc_ref])
        if bn < 1.0:
            assert float(out["ess"]) == pytest.approx(alpha * n, rel=1e-9)


def test_evidence_accumulates():
    G.require_gpu()
    w = inputs.bbh11()
    ctx = api.Context.from_workload(w)
    ctx.reset_evidence()
    n = 512
    rng = np.random.default_rng(3)
    th = G.to_dev(inputs.prior_draws(w, n, 1))
    g = G.to_dev(np.zeros((n, w.n_dim)))
    total, beta = 0.0, 0.0
    for k in range(4):
        lnl = -0.5 * rng.chisquare(11, size=n) * 40.0
        out = ctx.reweight_resample(th, G.to_dev(lnl), g, beta, 0.5, 0.3, want_cov=False)
        bn, dl, ess, _ = oracle.smc_reweight(lnl, beta, 0.5)
        total += dl
        beta = float(out["beta_next"])
    lnz, ns = ctx.log_evidence()
    assert ns == 4
    assert lnz == pytest.approx(total, rel=1e-10)
