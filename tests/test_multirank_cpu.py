"""The benchmark's multi-GPU layout on CPU: two gloo ranks, one independent event each,
work from the oracle's NUTS, scalars reduced across ranks."""
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


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
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
