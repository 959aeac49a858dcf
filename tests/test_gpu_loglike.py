"""GPU likelihood, gradient and waveform against the oracle (same seeded inputs).

Tolerances: FP64 path |d lnL| <= 1e-7 + 1e-10 |lnL| and gradient relative
error <= 1e-8; mixed path |d lnL| <= 1e-3 (<= 1e-2 for the 259585-bin
workload) and gradient relative error <= 1e-4, where the gradient error is
||(g - g_ref) * width|| / ||g_ref * width|| per particle (prior widths put
all components on one scale).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2601_02336_gb300 import api, inputs
from paper_2601_02336_gb300 import _lib
from paper_2601_02336_gb300._lib import SharpyError
from tests import gpu_helpers as G
from tests import helpers

pytestmark = pytest.mark.gpu


def _thetas(w, th_inj, n_prior, n_ball, seed):
    return np.vstack([inputs.prior_draws(w, n_prior, seed), inputs.ball(w, th_inj, n_ball, seed + 1)])


def _check(w, ev, ctx, thetas, lnl_tol, grad_tol, precision):
    model = helpers.oracle_model(w)
    ref_l, ref_g = oracle.loglike(model, ev, thetas)
    l, g = ctx.loglike_grad(G.to_dev(thetas), precision)
    torch.cuda.synchronize()
    l, g = l.cpu().numpy(), g.cpu().numpy()
    dl = np.abs(l - ref_l)
    assert np.all(np.isfinite(l)) and np.all(np.isfinite(g))
    assert np.max(dl - lnl_tol(ref_l)) <= 0, (np.max(dl), ref_l[np.argmax(dl)])
    err = G.grad_rel_err(g, ref_g, G.width(w))
    assert np.max(err) <= grad_tol, (np.max(err), np.argmax(err))
    # forward-only sweep gives the same ln L as the gradient sweep
    l2, _ = ctx.loglike_grad(G.to_dev(thetas), precision, grad=False)
    assert np.allclose(l2.cpu().numpy(), l, rtol=0, atol=1e-9 * max(1.0, np.max(np.abs(l))))
    return dl, err


@pytest.mark.parametrize("name", ["tiny", "bbh11"])
def test_waveform_matches_oracle(name):
    G.require_gpu()
    w = inputs.WORKLOADS[name]()
    ev, ctx, th_inj, _ = G.event_pair(w)
    model = helpers.oracle_model(w)
    thetas = _thetas(w, th_inj, 3, 2, 40)
    h = ctx.waveform(G.to_dev(thetas)).cpu().numpy()
    for i, th in enumerate(thetas):
        ref = oracle.waveform(model, ev, th)
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(h[i] - ref)) <= 1e-9 * scale, i


@pytest.mark.parametrize("name", ["tiny", "bbh11", "bbh11_long"])
def test_loglike_grad_fp64(name):
    G.require_gpu()
    w = inputs.WORKLOADS[name]()
    ev, ctx, th_inj, _ = G.event_pair(w)
    thetas = _thetas(w, th_inj, 21, 19, 50)  # 40 rows: several CTAs and a ragged tail
    _check(w, ev, ctx, thetas, lambda r: 1e-7 + 1e-10 * np.abs(r), 1e-8, "fp64")


@pytest.mark.parametrize("precision", ["mixed", "split"])
@pytest.mark.parametrize("name", ["tiny", "bbh11", "bbh11_long"])
def test_loglike_grad_mixed(name, precision):
    G.require_gpu()
    w = inputs.WORKLOADS[name]()
    ev, ctx, th_inj, _ = G.event_pair(w)
    thetas = _thetas(w, th_inj, 35, 29, 60)
    _check(w, ev, ctx, thetas, lambda r: 1e-3 + 0 * r, 1e-4, precision)


@pytest.mark.parametrize("name", ["tiny", "bbh11", "bbh11_long"])
def test_mixed_precision_budget(name):
    """The reduced-precision paths against the GPU FP64 path on 2048 theta (prior draws and a ball around the
    injection): a budget well inside the 1e-3 tolerance, so that a loss of precision anywhere in the mixed
    arithmetic (double-float coefficients, fixed-point delay term, compensated moments) shows up here first."""
    G.require_gpu()
    w = inputs.WORKLOADS[name]()
    ev, ctx, th_inj, _ = G.event_pair(w)
    t = G.to_dev(_thetas(w, th_inj, 1024, 1024, 90))
    l64, g64 = ctx.loglike_grad(t, "fp64")
    for precision, budget in (("mixed", 2.5e-4), ("split", 2.5e-4)):
        l, g = ctx.loglike_grad(t, precision)
        dl = torch.max(torch.abs(l - l64)).item()
        err = np.max(G.grad_rel_err(g.cpu().numpy(), g64.cpu().numpy(), G.width(w)))
        print(name, precision, "max |dlnL|", dl, "max grad rel", err)
        assert dl <= budget, (precision, dl)
        assert err <= 2.5e-5, (precision, err)


def test_loglike_long_signal_sampled():
    """259585 bins x 3 detectors at full size (sampled particles): mixed within 1e-2, FP64 tight."""
    G.require_gpu()
    w = inputs.bns()
    ev, ctx, th_inj, _ = G.event_pair(w)
    thetas = _thetas(w, th_inj, 9, 7, 70)
    _check(w, ev, ctx, thetas, lambda r: 1e-2 + 0 * r, 1e-4, "mixed")
    _check(w, ev, ctx, thetas, lambda r: 1e-2 + 0 * r, 1e-4, "split")
    _check(w, ev, ctx, thetas[:6], lambda r: 1e-6 + 1e-10 * np.abs(r), 1e-8, "fp64")


def test_gradient_central_differences_gpu():
    """GPU FP64 gradient vs central differences of the GPU FP64 ln L (h = 1e-6 relative), 64 seeded theta
    on the 32449-bin workload; components whose step moves the f_ISCO bin are skipped."""
    G.require_gpu()
    w = inputs.bbh11_long()
    ev, ctx, th_inj, _ = G.event_pair(w)
    thetas = _thetas(w, th_inj, 32, 32, 80)
    l, g = ctx.loglike_grad(G.to_dev(thetas), "fp64")
    g = g.cpu().numpy()
    wid = G.width(w)
    pts, hs = [], []
    for th in thetas:
        for j in range(w.n_dim):
            h = 1e-6 * abs(th[j]) if abs(th[j]) > 1e-3 * wid[j] else 1e-6 * wid[j]
            hs.append(h)
            for s in (1, -1):
                t = th.copy()
                t[j] += s * h
                pts.append(t)
    vals, _ = ctx.loglike_grad(G.to_dev(np.array(pts)), "fp64", grad=False)
    vals = vals.cpu().numpy().reshape(len(thetas), w.n_dim, 2)
    fd = (vals[..., 0] - vals[..., 1]) / (2 * np.array(hs).reshape(len(thetas), w.n_dim))
    kis = lambda t: math.floor((oracle.f_isco(t[0], t[1]) - w.f_min) / w.df)
    checked = 0
    for i, th in enumerate(thetas):
        for j in range(w.n_dim):
            if j in (0, 1):
                tp, tm = th.copy(), th.copy()
                tp[j] += hs[i * w.n_dim + j]
                tm[j] -= hs[i * w.n_dim + j]
                if kis(tp) != kis(th) or kis(tm) != kis(th):
                    continue
            scale = max(abs(g[i, j]), 1e-3 * np.linalg.norm(g[i] * wid) / wid[j], 1e-8)
            noise = 20 * 2.2e-16 * abs(float(l[i])) / hs[i * w.n_dim + j]  # rounding of ln L in the FD
            assert abs(fd[i, j] - g[i, j]) <= 2e-4 * scale + noise, (i, j, fd[i, j], g[i, j])
            checked += 1
    assert checked > 0.9 * len(thetas) * w.n_dim


def test_edge_cases():
    G.require_gpu()
    w = inputs.bbh11()
    ev, ctx, th_inj, _ = G.event_pair(w)
    model = helpers.oracle_model(w)
    # empty batch
    l, g = ctx.loglike_grad(torch.empty((0, w.n_dim), dtype=torch.float64, device="cuda"))
    assert l.shape == (0,)
    # single particle, and a mass above the band: f_ISCO < f_min, no bins -> lnL = -<d|d>/2
    th = th_inj.copy()
    th[0] = 400.0
    for prec in ("fp64", "mixed", "split"):
        l, g = ctx.loglike_grad(G.to_dev(th[None, :]), prec)
        ref = oracle.loglike(model, ev, th[None, :], grad=False)[0]
        assert float(l[0]) == pytest.approx(ref, rel=1e-12)
    # ragged batch sizes across CTA boundaries give identical rows
    thetas = inputs.prior_draws(w, 17, 90)
    full, _ = ctx.loglike_grad(G.to_dev(thetas), "mixed")
    for n in (1, 7, 8, 9, 16, 17):
        part, _ = ctx.loglike_grad(G.to_dev(thetas[:n]), "mixed")
        assert torch.equal(part, full[:n])
    assert ctx.status() == 0


def test_nonfinite_input_sets_status():
    G.require_gpu()
    w = inputs.tiny()
    ev, ctx, th_inj, _ = G.event_pair(w)
    th = th_inj.copy()
    th[0] = float("nan")
    l, g = ctx.loglike_grad(G.to_dev(th[None, :]), "mixed")
    assert not np.isfinite(float(l[0]))
    assert ctx.status() == -4
    ctx.clear_status()
    assert ctx.status() == 0


def test_set_data_rejects_nonfinite():
    G.require_gpu()
    w = inputs.tiny()
    ctx = api.Context.from_workload(w)
    data = np.zeros((1, w.n_bins, 2))
    psd = inputs.psd_array(w)
    psd[0, 10] = np.inf
    with pytest.raises(SharpyError):
        ctx.set_data(data, psd, w.f_min, w.df, inputs.detectors(w))
    with pytest.raises(Exception):
        ctx.loglike_grad(G.to_dev(inputs.prior_draws(w, 2, 1)))


def test_set_data_again_on_the_same_grid():
    """A second event on the same grid reuses the grid tables: its likelihood, gradient and local metric are
    bit-identical to a fresh context's, also when the PSD changes (the metric tables are rebuilt then)."""
    G.require_gpu()
    w = inputs.bbh11()
    dets = inputs.detectors(w)
    psd = inputs.psd_array(w)
    _, _, d0 = helpers.make_event(w, seed=0)
    _, _, d1 = helpers.make_event(w, seed=1)
    th = G.to_dev(inputs.prior_draws(w, 64, 7))
    ctx = api.Context.from_workload(w)
    ctx.set_data(d0, psd, w.f_min, w.df, dets)
    ctx.loglike_grad(th, "mixed")
    ctx.local_metric(th, 0.5, want=("mass",))
    for data, p in ((d1, psd), (d1, psd * 1.5)):
        ctx.set_data(data, p, w.f_min, w.df, dets)
        fresh = api.Context.from_workload(w)
        fresh.set_data(data, p, w.f_min, w.df, dets)
        for prec in ("fp64", "mixed", "split"):
            a, b = ctx.loglike_grad(th, prec), fresh.loglike_grad(th, prec)
            assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]), prec
        ma, mb = ctx.local_metric(th, 0.5, want=("mass",)), fresh.local_metric(th, 0.5, want=("mass",))
        assert torch.equal(ma["mass"], mb["mass"])


def test_autograd_backward_is_the_adjoint():
    G.require_gpu()
    w = inputs.bbh11()
    ev, ctx, th_inj, _ = G.event_pair(w)
    th = G.to_dev(_thetas(w, th_inj, 5, 5, 95)).requires_grad_(True)
    l = api.loglike(th, ctx, "mixed")
    wts = torch.linspace(0.5, 2.0, th.shape[0], dtype=torch.float64, device="cuda")
    (l * wts).sum().backward()
    _, g = ctx.loglike_grad(th.detach(), "mixed")
    assert torch.allclose(th.grad, g * wts[:, None], rtol=1e-12, atol=0)


@pytest.mark.parametrize("wname", ["bbh11", "bns"])
def test_loglike_split_factor_invariant(wname):
    """The likelihood kernel cuts a vector's bins into chunks of 2048 dealt to 8 streams merged in a fixed
    order, so the number of warps sharing a vector (1, 2, 4, 8: the tuner's choice) does not change ln L or
    the gradient, bit for bit, on every path, with and without the gradient; nor does choice 16, the staged
    kernel (one vector per warp, the tables of each 256-bin block brought into shared memory by one bulk copy),
    which the 259585-bin segment's mixed and split paths have (each with records of its own) and the others
    replace by 8. On that segment the streams' merge stays within the long-signal tolerance of the oracle. The
    tuner's pick is one of the candidates."""
    G.require_gpu()
    w = getattr(inputs, wname)()
    ev, ctx, th_inj, _ = G.event_pair(w)
    n = 37  # a ragged last CTA (the staged kernel holds 8 vectors a CTA)
    th = np.vstack([inputs.prior_draws(w, 19, 6), inputs.ball(w, th_inj, n - 19, 7)])
    t = G.to_dev(th)
    for prec in ("fp64", "mixed", "split"):
        ref = None
        for split in (1, 2, 4, 8, 16):
            ctx.set_loglike_split(split)
            l, g = ctx.loglike_grad(t, prec)
            l0, _ = ctx.loglike_grad(t, prec, grad=False)
            if ref is None:
                ref = (l, g, l0)
            else:
                assert torch.equal(l, ref[0]) and torch.equal(g, ref[1]), (prec, split)
                assert torch.equal(l0, ref[2]), (prec, split, "no gradient")
        if wname == "bns" and prec != "fp64":
            lref = oracle.loglike(helpers.oracle_model(w), ev, th[:4], grad=False)
            assert np.max(np.abs(ref[0].cpu().numpy()[:4] - lref)) <= 1e-2, prec
    ctx.set_loglike_split(0)
    for prec in ("mixed", "split"):
        ctx.loglike_grad(t, prec)
        assert ctx.loglike_split(n, prec) in ((1, 2, 4, 8, 16) if wname == "bns" else (1, 2, 4, 8)), prec
    assert ctx.status() == 0


@pytest.mark.parametrize("n_bins", [65535, 65536, 65537, 65536 + 255, 65536 + 2048 * 8 + 1])
def test_staged_kernel_segment_edges(n_bins):
    """The staged kernel at the edges of its domain: segments one bin short of the staging threshold (choice 16
    falls back to 8 warps), exactly at it, one bin and one record past it, and one bin into a stream's second
    chunk. On the mixed and split paths, with and without the gradient, choice 16 gives choice 1's ln L and
    gradient bit for bit, on 9 vectors (a full CTA of 8 and one more)."""
    import dataclasses
    G.require_gpu()
    w = dataclasses.replace(inputs.bns(n_particles=9), n_bins=n_bins, f_min=20.0, df=1.0 / 64.0)
    ctx, th_inj, _ = api.make_event(w, seed=0)
    t = G.to_dev(np.vstack([inputs.prior_draws(w, 4, 6), inputs.ball(w, th_inj, 5, 7)]))
    for prec in ("mixed", "split"):
        for grad in (True, False):
            ctx.set_loglike_split(1)
            l1, g1 = ctx.loglike_grad(t, prec, grad=grad)
            ctx.set_loglike_split(16)
            l16, g16 = ctx.loglike_grad(t, prec, grad=grad)
            assert torch.equal(l1, l16), (prec, grad)
            if grad:
                assert torch.equal(g1, g16), prec
    ctx.set_loglike_split(0)
    assert ctx.status() == 0


def test_staged_kernel_wait_timeout_reports_status():
    """Failure detection without a fault in the staged kernel (choice 16). The test hook leaves out the bulk copy of
    one table block, so the mbarrier waits for it run out after a short poll bound. The call returns; the status word
    reads SHARPY_ETIMEOUT, and the kernel issued no further copies and drained the ones in flight. The same context then
    runs clean: status 0 and ln L and gradient equal, bit for bit, to the 1-warp split kernel's."""
    G.require_gpu()
    w = inputs.bns()
    ctx, th_inj, _ = api.make_event(w, seed=0)
    t = G.to_dev(inputs.ball(w, th_inj, 20, 5, rel=1e-3))
    ctx.set_loglike_split(1)
    ref_l, ref_g = ctx.loglike_grad(t, "mixed")
    assert ctx.status() == 0
    ctx.set_loglike_split(16)
    ctx.set_stage_test_hooks(skip_block=3, wait_polls=64)
    ctx.loglike_grad(t, "mixed")
    torch.cuda.synchronize()
    assert ctx.status() == _lib.ETIMEOUT
    ctx.clear_status()
    ctx.set_stage_test_hooks(-1, 0)
    l, g = ctx.loglike_grad(t, "mixed")
    assert ctx.status() == 0
    assert torch.equal(l, ref_l) and torch.equal(g, ref_g)
    ctx.set_loglike_split(0)
