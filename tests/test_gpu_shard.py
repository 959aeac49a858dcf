"""Particle sharding of one event (multirank.ShardedSMC) on the GPU path: one
GPU holding three shards runs the sharded algorithm (per stage: gather of
the shards' state, the tempering step on the whole ensemble, each shard's
NUTS launch with its rows' ensemble indices, sharpy_set_shard) and must give
the same beta ladder, ln Z and particles, bit for bit, as sharpy_smc_run on
the whole ensemble. Between GPUs the gather is an NCCL all-gather (the same
driver code is checked over gloo ranks on the oracle in
test_multirank_cpu.py)."""
import numpy as np
import pytest
import torch

from paper_2601_02336_gb300 import api, inputs, multirank
from tests import gpu_helpers as G

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("wname,metric,precision", [("tiny", 0, "fp64"), ("tiny", 1, "mixed"),
                                                     ("bbh11", 0, "mixed"), ("tiny", 2, "fp64"),
                                                     ("bbh11", 2, "mixed")])
def test_sharded_run_equals_single_run(wname, metric, precision):
    G.require_gpu()
    w = getattr(inputs, wname)(n_particles=1000) if wname == "bbh11" else inputs.tiny()
    ctx = api.make_event(w, seed=0)[0]
    n = w.n_particles
    key = 515
    lnz, th, ll, rec = ctx.smc_run(n, w.alpha, w.n_mut, w.max_depth, metric, w.eps_scale, key=key,
                                   precision=precision)
    run = multirank.ShardedSMC(multirank.GpuShardBackend(ctx, precision), n, w.alpha, w.n_mut, w.max_depth,
                               metric, w.eps_scale, key, shards_per_rank=3)
    lnz_s = run.run()
    assert [r["beta"] for r in run.records] == [r["beta"] for r in rec]
    assert [r["dlnz"] for r in run.records] == [r["dlnz"] for r in rec]
    assert lnz_s == lnz
    parts = run.state()
    assert [p[0] for p in parts] == multirank.shard_bounds(n, 3)[:3]
    th_s = torch.cat([p[1] for p in parts])
    ll_s = torch.cat([p[2] for p in parts])
    assert torch.equal(th_s, th) and torch.equal(ll_s, ll)
    assert ctx.status() == 0
