"""Per-particle mass matrices on the GPU (sharpy_local_metric, Sec. 5) against the
oracle's literal Fisher information on the same event arrays."""
import numpy as np
import pytest
import torch

import oracle
from paper_2601_02336_gb300 import api, inputs
from tests import gpu_helpers as G
from tests import helpers

pytestmark = pytest.mark.gpu


def _scaled_err(a, b):
    """max |a - b| / sqrt(b_jj b_kk) per particle (entries span many decades in physical units)."""
    d = np.sqrt(np.abs(np.einsum("nii->ni", b)))
    return np.max(np.abs(a - b) / (d[:, :, None] * d[:, None, :]), axis=(1, 2))


@pytest.mark.parametrize("name", ["tiny", "bbh11"])
@pytest.mark.parametrize("beta", [0.0, 0.37, 1.0])
def test_local_metric_matches_oracle(name, beta):
    G.require_gpu()
    w = inputs.WORKLOADS[name]()
    ev, ctx, th_inj, data = G.event_pair(w, seed=0)
    model = helpers.oracle_model(w)
    th = np.concatenate([inputs.prior_draws(w, 24, 5), inputs.ball(w, th_inj, 24, 6, rel=1e-3)])
    ref = oracle.local_metric(model, ev, th, beta)
    out = ctx.local_metric(G.to_dev(th), beta)
    M = out["mass"].cpu().numpy()
    assert np.max(_scaled_err(M, ref)) < 1e-8
    Mi = out["inv_mass"].cpu().numpy()
    L = out["chol"].cpu().numpy()
    eye = np.eye(w.n_dim)
    for i in range(len(th)):
        s = np.sqrt(np.diag(ref[i]))
        # M M^-1 = I in the scale of M; L L^T = M^-1; L lower triangular
        assert np.allclose((M[i] @ Mi[i]) * (1.0 / s)[:, None] * s[None, :], eye, atol=1e-6)
        assert np.allclose(L[i] @ L[i].T, Mi[i], rtol=1e-9, atol=1e-12 * np.abs(Mi[i]).max())
        assert np.allclose(np.triu(L[i], 1), 0.0)


def test_local_metric_gaussian_mixture():
    G.require_gpu()
    lo, hi = [-4.0, -2.0, -3.0], [4.0, 6.0, 3.0]
    mu, sig = [[0.5, 1.0, 0.0], [-0.5, 2.0, 1.0]], [[0.2, 0.7, 0.4], [0.3, 0.5, 0.6]]
    model = helpers.gaussmix_model(lo, hi, [0.0, -0.3], mu, sig)
    ctx = api.Context(api.gaussmix_config(lo, hi, [0.0, -0.3], mu, sig))
    th = np.random.default_rng(4).uniform(-1.0, 1.5, size=(40, 3))
    ref = oracle.local_metric(model, None, th, 0.8)
    M = ctx.local_metric(G.to_dev(th), 0.8)["mass"].cpu().numpy()
    assert np.allclose(M, ref, rtol=1e-12, atol=0)
