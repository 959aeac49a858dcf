"""Sample recycling on the GPU (sharpy_recycle, Sec. 5): weights and kept draws
against the oracle on the same pool, and recycled draws of a full run against the
analytic posterior."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2601_02336_gb300 import api
from tests import gpu_helpers as G
from tests.test_oracle_recycling import _gaussian_ladder

pytestmark = pytest.mark.gpu


def test_recycle_matches_oracle():
    G.require_gpu()
    betas = np.array([0.02, 0.1, 0.35, 1.0])
    x, lnl, lnz = _gaussian_ladder(0.4, 0.2, betas, 5000, seed=21)
    key = 77
    lw_ref = oracle.recycle_weights(lnl, betas, lnz)
    keep_ref = oracle.rejection_sample(lw_ref, key).astype(bool)
    th = G.to_dev(x[:, None])
    lw, kept = api.recycle(th, G.to_dev(lnl), betas, lnz, key)
    lw = lw.cpu().numpy()
    assert np.allclose(lw, lw_ref, rtol=1e-12, atol=1e-12)
    # the kept set: identical except where u_i sits within rounding of w_i / max w
    u = np.array([oracle.uniform2(key, i & 0xffffffff, i >> 32, 7, 0)[0] for i in range(len(x))])
    ratio = np.exp(lw_ref - lw_ref.max())
    sure = np.abs(u - ratio) > 1e-9
    kept = kept.cpu().numpy()[:, 0]
    where = {v: i for i, v in enumerate(x)}  # continuous draws: the values are distinct
    rows = np.array([where[v] for v in kept])
    assert np.all(np.diff(rows) > 0)  # pool order
    keep_gpu = np.zeros(len(x), dtype=bool)
    keep_gpu[rows] = True
    assert np.array_equal(keep_gpu[sure], keep_ref[sure])


def test_recycled_run_matches_posterior():
    """Gaussian likelihood, wide box prior: the recycled pool of a full run gives i.i.d. draws of the
    posterior, more of them than the last stage's particles."""
    G.require_gpu()
    mu, sig = [0.5, -1.0], [0.3, 0.6]
    ctx = api.Context(api.gaussmix_config([-10.0] * 2, [10.0] * 2, [0.0], [mu], [sig]))
    n = 4096
    lnz, th, ll, rec, pth, pll = ctx.smc_run(n, 0.5, 2, 5, 1, 0.5, key=31, precision="fp64", pool_stages=64)
    assert pth.shape[0] == len(rec) * n
    lw, kept = api.recycle_run(pth, pll, rec, n, key=5)
    kept = kept.cpu().numpy()
    assert kept.shape[0] > n
    for j in range(2):
        assert abs(kept[:, j].mean() - mu[j]) < 5 * sig[j] / math.sqrt(kept.shape[0]) + 0.01
        assert abs(kept[:, j].std() / sig[j] - 1.0) < 0.05
