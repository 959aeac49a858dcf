"""Multi-GPU layouts.

1. The benchmark's weak-scaling layout: one independent event (SMC run) per
   rank. SMC runs on different events share nothing, so the ranks exchange no
   data on the hot path; only two scalars cross ranks per measurement (the
   summed evaluation count and the maximum elapsed time).

2. Particle sharding of ONE event (Sec. 7: splitting the SMC particles across
   GPUs). The mutation step (Sec. 3, item 3) is independent per particle, so
   shard j of G holds the rows [j N / G, (j + 1) N / G) and mutates them alone;
   its NUTS random numbers are named by the rows' ensemble indices
   (sharpy_set_shard), so a shard computes what a single-GPU run computes for
   those rows. The exchange is one step per stage: an all-gather of the
   particle state (theta, ln L, grad: (2 D + 1) doubles a particle, 3 MB for
   16384 particles at D = 11), after which every rank holds the whole ensemble
   and runs the tempering step on it -- the ESS root (Eqs. 5-6), the evidence
   increment (Eq. 7), the weighted covariance and the integer systematic
   resampling -- with the same kernels on the same inputs, so every rank gets
   the same beta, ln Z and ancestors, bit for bit, as a single-GPU run; it
   then keeps its own rows of the resampled ensemble (the particle migration).
   Replicating the reweight costs each rank one O(N) pass (~0.1 ms at
   N = 16384) and replaces the per-iteration all-reduces of a distributed root
   search, the logsumexp reductions and the exclusive scan of per-rank integer
   weight totals with one collective, whose result does not depend on the
   shard count.

   The driver is backend-agnostic: GpuShardBackend runs every step in the CUDA
   library (NCCL all-gather between GPUs); the tests drive the same code with
   a backend on the CPU oracle over gloo ranks. A rank may hold several shards
   (shards_per_rank), which lets one GPU run the sharded algorithm.
"""
from __future__ import annotations

import os


def env_rank():
    """(rank, world size, local rank) from the torchrun environment (1 process: 0, 1, 0)."""
    g = lambda k, d: int(os.environ.get(k, d))
    return g("RANK", 0), g("WORLD_SIZE", 1), g("LOCAL_RANK", 0)


def event_seed(rank: int) -> int:
    """Seed of the synthetic event analysed by `rank` (each rank: its own injection and noise)."""
    return rank


def run_key(base: int, rank: int, step: int) -> int:
    """Philox key of SMC run `step` on `rank`: disjoint across ranks and steps."""
    return base + 1000 * rank + step


def reduce_scalar(x: float, op: str, world: int, device="cpu") -> float:
    """All-reduce one float across ranks ('sum' or 'max'); identity with one rank."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM if op == "sum" else dist.ReduceOp.MAX)
    return float(t[0])


def aggregate(evals: float, seconds: float, world: int, device="cpu"):
    """Whole-job (evaluations/s, slowest rank's seconds)."""
    total = reduce_scalar(evals, "sum", world, device)
    slowest = reduce_scalar(seconds, "max", world, device)
    return total / slowest, slowest


# ----------------------------------------------------------- particle sharding
RNG_RESAMPLE = 6  # Philox purpose of the stage's resampling uniform (particle 0, step = stage)


def shard_bounds(n: int, g: int):
    """Row boundaries of g shards of n particles: shard j holds [b[j], b[j + 1]); sizes differ by <= 1."""
    if g < 1 or n < g:
        raise ValueError(f"cannot split {n} particles into {g} shards")
    return [j * n // g for j in range(g + 1)]


class GpuShardBackend:
    """ShardedSMC steps on this rank's GPU: one library context holding the event; every step runs in
    the library's kernels (prior draw, likelihood, tempering step, NUTS)."""

    def __init__(self, ctx, precision="mixed"):
        self.ctx = ctx
        self.precision = precision

    def uniform(self, key, c0, c1, c2, c3):
        from . import api
        return api.uniform2(key, c0, c1, c2, c3)[0]

    def prior(self, first, n, key):
        self.ctx.set_shard(first)
        th = self.ctx.prior_sample(n, key, 0)
        lnl, grad = self.ctx.loglike_grad(th, self.precision)
        return th, lnl, grad

    def pack(self, th, lnl, grad):
        import torch
        return torch.cat([th, lnl[:, None], grad], dim=1)

    def unpack(self, packed, d):
        return (packed[:, :d].contiguous(), packed[:, d].contiguous(), packed[:, d + 1:].contiguous())

    def rows(self, state, lo, hi):
        return tuple(a[lo:hi].clone() for a in state)

    def concat(self, blocks):
        import torch
        return torch.cat(blocks, dim=0)

    def to_tensor(self, packed):
        return packed

    def from_tensor(self, t):
        return t

    def begin(self):
        self.ctx.reset_evidence()

    def stage(self, state, beta, alpha, u):
        """Tempering step on the whole ensemble, in place; (beta_next, dlnz, running ln Z, cov, ancestors)."""
        th, lnl, grad = state
        r = self.ctx.reweight_resample(th, lnl, grad, beta, alpha, u)
        lnz, _ = self.ctx.log_evidence()  # the context's device accumulator of the increments (Eq. 8)
        return float(r["beta_next"]), float(r["dlnz"]), lnz, r["cov"], r["ancestors"]

    def mutate(self, first, state, beta, cov, metric, eps_scale, max_depth, n_mut, key, ctr):
        th, lnl, grad = state
        self.ctx.set_shard(first)
        if metric == 0:
            self.ctx.nuts_mutate_cov_step(beta, th, lnl, grad, cov, eps_scale, max_depth, n_mut, key, ctr,
                                          precision=self.precision, stats=False)
        elif metric == 1:
            self.ctx.nuts_mutate(beta, th, lnl, grad, cov, eps_scale, max_depth, n_mut, key, ctr,
                                 precision=self.precision, stats=False)
        elif metric == 2:
            # each row's local metric at the new temperature (Sec. 5) needs only the row: no exchange
            m = self.ctx.local_metric(th, beta, want=("inv_mass", "chol"))
            self.ctx.nuts_mutate_local(beta, th, lnl, grad, m["inv_mass"], m["chol"], eps_scale, max_depth, n_mut,
                                       key, ctr, precision=self.precision, stats=False)
        else:
            raise ValueError("metric must be 0 (identity), 1 (covariance) or 2 (local)")
        return th, lnl, grad

    def finish(self):
        self.ctx.set_shard(0)


class ShardedSMC:
    """One event's SMC run (Sec. 3) with its particles split over the ranks of the default process
    group (world size 1 without one), `shards_per_rank` shards on each rank. Rank r holds shards
    r S .. r S + S - 1. run() returns ln Z; `records` has each stage's beta, dlnz, running ln Z and
    ancestors; `state()` the rank's shards."""

    def __init__(self, backend, n_particles, alpha, n_mut, max_depth, metric, eps_scale, key,
                 shards_per_rank=1, max_stages=500):
        import torch.distributed as dist
        self.b = backend
        self.n, self.alpha, self.n_mut, self.max_depth = int(n_particles), float(alpha), int(n_mut), int(max_depth)
        self.metric, self.eps_scale, self.key, self.max_stages = int(metric), float(eps_scale), int(key), max_stages
        dist_on = dist.is_available() and dist.is_initialized()
        self.rank = dist.get_rank() if dist_on else 0
        self.world = dist.get_world_size() if dist_on else 1
        self.spr = int(shards_per_rank)
        bounds = shard_bounds(self.n, self.world * self.spr)
        self.bounds = bounds
        self.mine = [(bounds[j], bounds[j + 1]) for j in range(self.rank * self.spr, (self.rank + 1) * self.spr)]
        # rows of each rank's block
        self.block = [(bounds[r * self.spr], bounds[(r + 1) * self.spr]) for r in range(self.world)]
        self.records = []
        self.shards = None
        self.lnz = 0.0

    def _gather(self):
        """All-gather of the ranks' particle state, in ensemble order."""
        import torch
        import torch.distributed as dist
        local = self.b.concat([self.b.pack(*s) for s in self.shards])
        if self.world == 1:
            return local
        t = self.b.to_tensor(local)
        rows = max(hi - lo for lo, hi in self.block)
        pad = torch.zeros((rows, t.shape[1]), dtype=t.dtype, device=t.device)
        pad[:t.shape[0]] = t
        parts = [torch.empty_like(pad) for _ in range(self.world)]
        dist.all_gather(parts, pad)
        full = torch.cat([p[:hi - lo] for p, (lo, hi) in zip(parts, self.block)], dim=0)
        return self.b.from_tensor(full)

    def run(self):
        d = None
        self.shards = []
        for lo, hi in self.mine:
            s = self.b.prior(lo, hi - lo, self.key)
            self.shards.append(s)
            d = s[0].shape[1]
        self.b.begin()
        beta, t = 0.0, 0
        while beta < 1.0 and t < self.max_stages:
            t += 1
            state = self.b.unpack(self._gather(), d)
            u = self.b.uniform(self.key, 0, t, RNG_RESAMPLE, 0)
            bn, dl, lnz, cov, anc = self.b.stage(state, beta, self.alpha, u)
            self.shards = [self.b.rows(state, lo, hi) for lo, hi in self.mine]
            self.shards = [self.b.mutate(lo, s, bn, cov, self.metric, self.eps_scale, self.max_depth, self.n_mut,
                                         self.key, t << 8) for (lo, _), s in zip(self.mine, self.shards)]
            self.records.append({"beta": bn, "dlnz": dl, "lnz": lnz, "ancestors": anc})
            beta = bn
            self.lnz = lnz
        self.b.finish()
        return self.lnz

    def state(self):
        """(first row, theta, ln L, grad) of each of this rank's shards."""
        return [(lo,) + tuple(s) for (lo, _), s in zip(self.mine, self.shards)]
