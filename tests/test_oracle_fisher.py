"""Pins for the oracle's Fisher information and per-particle mass matrix (Sec. 5,
"Exploitation of local geometry"): closed forms of single entries, the noiseless
Hessian identity, and the box-prior limit."""
import math

import numpy as np

import oracle
from paper_2601_02336_gb300 import inputs
from tests import helpers


def _zero_event(w):
    return helpers.oracle_event(w, noise=False, data=np.zeros((w.n_det, w.n_bins, 2)))


def _inner(w, h1, h2):
    """<h1|h2> = 4 df Re sum conj(h1) h2 / S over detectors and bins (Eq. 2)."""
    psd = inputs.psd_array(w)
    a = h1[..., 0] - 1j * h1[..., 1]
    b = h2[..., 0] + 1j * h2[..., 1]
    return float(np.sum(4.0 * w.df * (a * b).real / psd))


def test_fisher_closed_form_entries():
    """d h / d d_L = -h / d_L, d h / d phi_c = i h, d h / d t_c = -2 pi i f h: so F_dLdL d_L^2 and F_phiphi
    are <h|h> = -2 ln L(theta; d = 0), F_tt is 4 pi^2 <f h|f h>, and F_(phi, d_L) = 0."""
    w = inputs.bbh11()
    model = helpers.oracle_model(w)
    ev0 = _zero_event(w)
    rng = np.random.default_rng(3)
    th = inputs.prior_draws(w, 3, 4)
    F = oracle.fisher(model, ev0, th)
    hh = -2.0 * oracle.loglike(model, ev0, th, grad=False)
    f = inputs.frequencies(w)
    kd, kp, kt = w.phys.index(inputs.DL), w.phys.index(inputs.PHIC), w.phys.index(inputs.TC)
    for i in range(3):
        h = oracle.waveform(model, ev0, th[i]).reshape(w.n_det, w.n_bins, 2)
        fh = h * f[None, :, None]
        assert math.isclose(F[i, kd, kd] * th[i, kd] ** 2, hh[i], rel_tol=1e-10)
        assert math.isclose(F[i, kp, kp], hh[i], rel_tol=1e-10)
        assert abs(F[i, kp, kd]) < 1e-10 * math.sqrt(F[i, kp, kp] * F[i, kd, kd])
        assert math.isclose(F[i, kt, kt], 4.0 * math.pi ** 2 * _inner(w, fh, fh), rel_tol=1e-10)
        assert np.allclose(F[i], F[i].T, rtol=1e-12, atol=0)
        assert np.linalg.eigvalsh(F[i]).min() > -1e-9 * np.abs(F[i]).max()
    del rng


def test_fisher_is_noiseless_hessian():
    """With data d = h(theta0) and no noise the residual vanishes at theta0, so -d^2 ln L = F there
    (central differences of the exact gradient; tiny workload, f_ISCO above the band)."""
    w = inputs.tiny()
    model = helpers.oracle_model(w)
    ev, th0, _ = helpers.make_event(w, seed=0, with_noise=False)
    F = oracle.fisher(model, ev, th0[None, :])[0]
    d = w.n_dim
    H = np.zeros((d, d))
    for k in range(d):
        step = 1e-5 * (w.hi[k] - w.lo[k])
        tp, tm = th0.copy(), th0.copy()
        tp[k] += step
        tm[k] -= step
        _, gp = oracle.loglike(model, ev, tp[None, :])
        _, gm = oracle.loglike(model, ev, tm[None, :])
        H[:, k] = -(gp[0] - gm[0]) / (2 * step)
    scale = np.sqrt(np.outer(np.diag(F), np.diag(F)))
    assert np.max(np.abs(H - F) / scale) < 1e-5, np.max(np.abs(H - F) / scale)


def test_local_metric_box_limit_and_scaling():
    """beta = 0: the mass matrix is the precision 12 / width^2 of each uniform box (variance of U[a, b]
    is (b - a)^2 / 12), plus 2 / d^2 on the distance (prior proportional to d^2); beta scales F."""
    w = inputs.bbh11()
    model = helpers.oracle_model(w)
    ev0 = _zero_event(w)
    th = inputs.prior_draws(w, 2, 9)
    M0 = oracle.local_metric(model, ev0, th, 0.0)
    wid = np.array(w.hi) - np.array(w.lo)
    kd = w.phys.index(inputs.DL)
    for i in range(2):
        expect = np.diag(12.0 / wid ** 2)
        expect[kd, kd] += 2.0 / th[i, kd] ** 2
        assert np.allclose(M0[i], expect, rtol=1e-14, atol=0)
    F = oracle.fisher(model, ev0, th)
    M = oracle.local_metric(model, ev0, th, 0.3)
    assert np.allclose(M - M0, 0.3 * F, rtol=1e-12, atol=1e-12 * np.abs(F).max())


def test_local_metric_single_gaussian_is_hessian():
    """One Gaussian component: beta F is exactly beta times the Hessian of -ln L, diag(1 / sigma^2)."""
    lo, hi = [-4.0, -2.0], [4.0, 6.0]
    model = helpers.gaussmix_model(lo, hi, [0.0], [[0.5, 1.0]], [[0.2, 0.7]])
    th = np.array([[0.1, 1.5], [-1.0, 3.0]])
    M = oracle.local_metric(model, None, th, 0.6)
    expect = np.diag(0.6 / np.array([0.2, 0.7]) ** 2 + 12.0 / (np.array(hi) - np.array(lo)) ** 2)
    for i in range(2):
        assert np.allclose(M[i], expect, rtol=1e-14, atol=0)
