"""Multi-rank layouts on CPU (gloo ranks, oracle arithmetic).

1. The benchmark's layout: one independent event per rank, scalars reduced.
2. Particle sharding of one event (multirank.ShardedSMC): two gloo ranks
   (and one rank holding three shards) give the same beta ladder, ancestors,
   particles and ln Z, bit for bit, as one rank holding the whole ensemble,
   which in turn equals the oracle's own SMC run with the same key.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import time

    import torch.distributed as dist

    import oracle
    from paper_2601_02336_gb300 import inputs, multirank
    from tests import helpers
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, ws, lr = multirank.env_rank()
    w = inputs.tiny()
    ev, th_inj, data = helpers.make_event(w, seed=multirank.event_seed(r))
    model = helpers.oracle_model(w)
    th = inputs.ball(w, th_inj, 16, 7 + r, rel=2e-3)
    lnl, g = oracle.loglike(model, ev, th)
    t0 = time.perf_counter()
    _, _, _, st = oracle.nuts_mutate(model, ev, 1.0, th, lnl, g, None, 2e-4, 4, 1,
                                     key=multirank.run_key(5, r, 0), ctr=0)
    secs = time.perf_counter() - t0
    evals = float(st["n_leapfrog"].sum())
    rate, slowest = multirank.aggregate(evals, secs, ws)
    out[r] = (evals, secs, rate, slowest, float(data[0, 0, 0]))
    dist.barrier()
    dist.destroy_process_group()


def _spawn(target, world, *args):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, out) + args) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(600)
        assert p.exitcode == 0
    return dict(out)


def test_two_rank_aggregation():
    out = _spawn(_worker, 2)
    e0, s0, r0, m0, d0 = out[0]
    e1, s1, r1, m1, d1 = out[1]
    assert r0 == pytest.approx(r1) and m0 == pytest.approx(m1)
    assert m0 == pytest.approx(max(s0, s1))
    assert r0 == pytest.approx((e0 + e1) / max(s0, s1))
    assert d0 != d1  # each rank analysed its own event


def test_single_rank_identity():
    from paper_2601_02336_gb300 import multirank
    assert multirank.aggregate(10.0, 2.0, 1) == (5.0, 2.0)
    assert multirank.run_key(100, 1, 2) != multirank.run_key(100, 0, 2)
    assert multirank.shard_bounds(10, 3) == [0, 3, 6, 10]
    with pytest.raises(ValueError):
        multirank.shard_bounds(2, 3)


# ----------------------------------------------------- particle sharding
N_SHARD, KEY_SHARD = 96, 4242


def _sharded_run(shards_per_rank, metric=None):
    import oracle
    from paper_2601_02336_gb300 import inputs, multirank
    from tests import helpers
    from tests.sharded_oracle import OracleShardBackend
    w = inputs.tiny()
    ev, _, _ = helpers.make_event(w, seed=0)
    model = helpers.oracle_model(w)
    prev = oracle.set_threads(1)  # restored below: later tests in this process use all cores
    try:
        run = multirank.ShardedSMC(OracleShardBackend(model, ev), N_SHARD, w.alpha, w.n_mut, 4,
                                   w.metric if metric is None else metric, w.eps_scale, KEY_SHARD,
                                   shards_per_rank=shards_per_rank)
        lnz = run.run()
    finally:
        oracle.set_threads(prev)
    recs = [(r["beta"], r["dlnz"], r["lnz"], np.asarray(r["ancestors"]).tolist()) for r in run.records]
    parts = [(lo, th.tolist(), lnl.tolist()) for lo, th, lnl, _ in run.state()]
    return lnz, recs, parts


def _shard_worker(rank, world, port, out, shards_per_rank):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out[rank] = _sharded_run(shards_per_rank)
    dist.barrier()
    dist.destroy_process_group()


def _assemble(parts_by_rank):
    rows = sorted(p for parts in parts_by_rank for p in parts)
    th = np.concatenate([np.array(t) for _, t, _ in rows])
    lnl = np.concatenate([np.array(l) for _, _, l in rows])
    return th, lnl


def test_particle_sharding_bit_identical():
    import oracle
    from paper_2601_02336_gb300 import inputs
    from tests import helpers
    single = _sharded_run(1)                 # one rank, whole ensemble
    multi = _spawn(_shard_worker, 2, 1)      # two gloo ranks, one shard each
    local3 = _sharded_run(3)                 # one rank, three shards
    lnz1, rec1, parts1 = single
    th1, l1 = _assemble([parts1])
    for lnz, rec, th, l in [(multi[0][0], multi[0][1], *_assemble([multi[0][2], multi[1][2]])),
                            (local3[0], local3[1], *_assemble([local3[2]]))]:
        assert lnz == lnz1
        assert rec == rec1  # beta, increments, running ln Z and ancestors of every stage
        assert np.array_equal(th, th1) and np.array_equal(l, l1)
    assert multi[1][0] == lnz1 and multi[1][1] == rec1  # both ranks hold the same ladder and evidence
    assert len(rec1) >= 2
    # and the unsharded driver is the oracle's own SMC run
    w = inputs.tiny()
    ev, _, _ = helpers.make_event(w, seed=0)
    lnz_o, th_o, l_o, rec_o = oracle.smc_run(helpers.oracle_model(w), ev, N_SHARD, w.alpha, w.n_mut, 4, w.metric,
                                             w.eps_scale, key=KEY_SHARD)
    assert lnz_o == lnz1
    assert [r["beta"] for r in rec_o] == [r[0] for r in rec1]
    assert np.array_equal(th_o, th1) and np.array_equal(l_o, l1)


def test_particle_sharding_local_metric():
    """The per-particle local metric (metric 2, Sec. 5) in the sharded driver: each shard forms its own rows'
    metrics at the new temperature, so three shards on one rank give the one-shard run bit for bit, and that is
    the oracle's own SMC run with metric 2."""
    import oracle
    from paper_2601_02336_gb300 import inputs
    from tests import helpers
    lnz1, rec1, parts1 = _sharded_run(1, metric=2)
    lnz3, rec3, parts3 = _sharded_run(3, metric=2)
    th1, l1 = _assemble([parts1])
    th3, l3 = _assemble([parts3])
    assert lnz3 == lnz1 and rec3 == rec1
    assert np.array_equal(th3, th1) and np.array_equal(l3, l1)
    assert len(rec1) >= 2
    w = inputs.tiny()
    ev, _, _ = helpers.make_event(w, seed=0)
    lnz_o, th_o, l_o, rec_o = oracle.smc_run(helpers.oracle_model(w), ev, N_SHARD, w.alpha, w.n_mut, 4, 2,
                                             w.eps_scale, key=KEY_SHARD)
    assert lnz_o == lnz1
    assert [r["beta"] for r in rec_o] == [r[0] for r in rec1]
    assert np.array_equal(th_o, th1) and np.array_equal(l_o, l1)

