"""Batched SMC (sharpy_batch_*): several events in one persistent NUTS launch per
stage round, rounds replayed from a captured CUDA graph, slot count picked by
the autotuner. The batch only regroups the work, so every event must give
exactly what a separate sharpy_smc_run with the same key gives: ln Z, the final
particles and the stage records, bit for bit."""
import pytest
import torch

from paper_2601_02336_gb300 import api, inputs
from paper_2601_02336_gb300._lib import SharpyError
from tests import gpu_helpers as G

pytestmark = pytest.mark.gpu


def _uneven_events():
    """Three events of the batched workload recipe (4 s, 4 s and 8 s segments), few particles."""
    ws = inputs.batch64()
    pick = [ws[0], ws[1], ws[16]]
    for w, n in zip(pick, (192, 320, 256)):
        w.n_particles = n
        w.max_depth = 6
    return pick


def _check_against_runs(b, ws, ctxs, keys, res, **kw):
    for e, (w, c, k) in enumerate(zip(ws, ctxs, keys)):
        lnz, th, ll, rec = c.smc_run(w.n_particles, key=k, **kw)
        assert res[e]["lnz"] == lnz, (e, res[e]["lnz"], lnz)
        assert res[e]["n_stages"] == len(rec)
        assert res[e]["beta"] == 1.0
        assert res[e]["n_leapfrog"] == sum(r["n_leapfrog"] for r in rec)
        tb, lb = b.particles(e)
        assert torch.equal(tb, th) and torch.equal(lb, ll)
        st = b.stages(e)
        for f in ("beta", "ess", "dlnz", "eps", "n_leapfrog", "active_bins"):
            assert [s[f] for s in st] == [r[f] for r in rec], f


@pytest.mark.parametrize("precision", ["split", "fp64"])
def test_batch_matches_separate_runs(precision):
    G.require_gpu()
    ws = _uneven_events()
    ctxs = [api.make_event(w, seed=i)[0] for i, w in enumerate(ws)]
    keys = [11, 12, 13]
    kw = dict(alpha=0.5, n_mut=2, max_depth=6, metric=0, eps_scale=0.5, precision=precision, max_stages=200)
    b = api.Batch(ctxs, [w.n_particles for w in ws], **kw)
    res, rounds = b.run(keys)
    assert b.slots in (0, 4, 8, 16, 32)  # 0: every event finished before the tuning round
    assert rounds >= max(r["n_stages"] for r in res)
    _check_against_runs(b, ws, ctxs, keys, res, **kw)
    # a second run replays the cached graph without tuning and repeats itself
    res2, rounds2 = b.run(keys)
    assert [r["lnz"] for r in res2] == [r["lnz"] for r in res]
    # init, prior draw and ln L per event, then 7 kernels per round (eager or replayed)
    assert b.launches == 1 + 2 * len(ws) + 7 * rounds2


@pytest.mark.parametrize("slots", [4, 8, 32])
def test_batch_forced_slots_match_separate_runs(slots):
    """The batched NUTS launch with a forced slot count (32: many sweeps per CTA, each warp runs whole
    particles; 8: few; 4: one sweep and one state machine per warp, on a 16-lane group with the upper half-warp
    idle) against separate runs, bit for bit: a particle's trajectory must not depend on how its CTA schedules
    the sweeps."""
    G.require_gpu()
    ws = _uneven_events()
    ctxs = [api.make_event(w, seed=10 + i)[0] for i, w in enumerate(ws)]
    keys = [21, 22, 23]
    kw = dict(alpha=0.5, n_mut=2, max_depth=6, metric=0, eps_scale=0.5, precision="mixed", max_stages=200)
    b = api.Batch(ctxs, [w.n_particles for w in ws], **kw)
    b.slots = slots
    res, _ = b.run(keys)
    assert b.slots == slots
    _check_against_runs(b, ws, ctxs, keys, res, **kw)


@pytest.mark.parametrize("metric", [1, 2])
def test_batch_dense_metrics_single_detector(metric):
    """Two single-detector events (different noise) with the weighted-covariance metric (1) and the
    per-particle local metric (2)."""
    G.require_gpu()
    ws = [inputs.tiny(), inputs.tiny()]
    ctxs = [api.make_event(w, seed=i)[0] for i, w in enumerate(ws)]
    keys = [5, 6]
    kw = dict(alpha=0.5, n_mut=2, max_depth=5, metric=metric, eps_scale=0.5, precision="fp64", max_stages=200)
    b = api.Batch(ctxs, [w.n_particles for w in ws], **kw)
    res, _ = b.run(keys)
    _check_against_runs(b, ws, ctxs, keys, res, **kw)


def test_batch_rejects_mixed_detector_counts():
    G.require_gpu()
    a = api.make_event(inputs.tiny(), seed=0)[0]
    w = inputs.batch64()[0]
    w.n_particles = 64
    c = api.make_event(w, seed=0)[0]
    with pytest.raises(SharpyError):
        api.Batch([a, c], [64, 64], 0.5, 2, 4, 0, 0.5)


def test_batch_event_lnz_vs_oracle_runs():
    """One event of the batched recipe (4 s segment, 4017 bins, 256 particles, depth 8) run inside a
    two-event batch: ln Z over R = 8 keys against the oracle's full SMC runs of that event
    (tests/golden, written by tests/golden/make_lnz_oracle.py from the oracle alone), within two
    combined standard errors."""
    import json
    import math
    import os

    import numpy as np
    G.require_gpu()
    with open(os.path.join(os.path.dirname(__file__), "golden", "lnz_batch1_oracle.json")) as fh:
        gold = json.load(fh)
    ws = inputs.batch64()
    w, w2 = ws[5], ws[16]
    w.n_particles, w2.n_particles = gold["n_particles"], 192
    assert gold["n_bins"] == w.n_bins and gold["max_depth"] == w.max_depth
    _, ctx, _, _ = G.event_pair(w, seed=gold["event_seed"])
    ctx2 = api.make_event(w2, seed=16)[0]
    b = api.Batch([ctx, ctx2], [w.n_particles, w2.n_particles], alpha=w.alpha, n_mut=w.n_mut,
                  max_depth=w.max_depth, metric=w.metric, eps_scale=w.eps_scale, precision="mixed", max_stages=200)
    got = [b.run([7300 + s, 7400 + s])[0][0]["lnz"] for s in range(8)]
    ref = [r["lnz"] for r in gold["runs"]]
    assert len(ref) >= 6
    se = lambda x: np.std(x, ddof=1) / math.sqrt(len(x))
    assert abs(np.mean(got) - np.mean(ref)) <= 2.0 * math.sqrt(se(got) ** 2 + se(ref) ** 2), (got, ref)
