"""Stage-boundary checkpoints (api.SMCRunner): the host-driven stage loop draws
the kernels' random numbers, so it reproduces sharpy_smc_run bit for bit, and a
run saved after any stage and restored continues exactly as the uninterrupted
one."""
import pytest
import torch

from paper_2601_02336_gb300 import api, inputs
from tests import gpu_helpers as G

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("metric,precision", [(0, "fp64"), (1, "mixed"), (2, "split")])
def test_runner_matches_native_run_and_resumes(tmp_path, metric, precision):
    G.require_gpu()
    w = inputs.tiny()
    ctx = api.make_event(w, seed=0)[0]
    kw = dict(n_particles=w.n_particles, alpha=w.alpha, n_mut=w.n_mut, max_depth=w.max_depth, metric=metric,
              eps_scale=w.eps_scale, key=71, precision=precision)
    lnz, th, ll, rec = ctx.smc_run(kw["n_particles"], kw["alpha"], kw["n_mut"], kw["max_depth"], metric,
                                   kw["eps_scale"], key=71, precision=precision)
    full = api.SMCRunner(ctx, **kw)
    assert full.run() == lnz
    assert torch.equal(full.theta, th) and torch.equal(full.lnl, ll)
    assert [r["beta"] for r in full.records] == [r["beta"] for r in rec]
    # interrupt after two stages, checkpoint, restore into a fresh runner, finish
    part = api.SMCRunner(ctx, **kw).start()
    part.step().step()
    path = tmp_path / "stage2.npz"
    part.save(path)
    del part
    resumed = api.SMCRunner.load(ctx, path)
    assert resumed.stage == 2
    assert resumed.run() == lnz
    assert torch.equal(resumed.theta, th)
    assert [r["beta"] for r in resumed.records] == [r["beta"] for r in rec]
