"""ShardedSMC backend on the CPU oracle (test infrastructure): the same
per-stage steps as the oracle's own SMC run (prior draw, literal ln L, ESS
bisection, evidence increment, weighted covariance, integer systematic
resampling, NUTS with the rows' ensemble indices naming their random
numbers), on numpy arrays, exchanged as CPU tensors over gloo."""
import math

import numpy as np
import torch

import oracle


class OracleShardBackend:
    def __init__(self, model, event):
        self.model, self.event = model, event
        self.lnz = 0.0

    def uniform(self, key, c0, c1, c2, c3):
        return oracle.uniform2(key, c0, c1, c2, c3)[0]

    def prior(self, first, n, key):
        th = oracle.prior_sample(self.model, first + n, key)[first:].copy()
        lnl, g = oracle.loglike(self.model, self.event, th)
        return th, lnl, g

    def pack(self, th, lnl, grad):
        return np.concatenate([th, lnl[:, None], grad], axis=1)

    def unpack(self, packed, d):
        return (np.ascontiguousarray(packed[:, :d]), np.ascontiguousarray(packed[:, d]),
                np.ascontiguousarray(packed[:, d + 1:]))

    def rows(self, state, lo, hi):
        return tuple(a[lo:hi].copy() for a in state)

    def concat(self, blocks):
        return np.concatenate(blocks, axis=0)

    def to_tensor(self, packed):
        return torch.from_numpy(np.ascontiguousarray(packed))

    def from_tensor(self, t):
        return t.numpy()

    def begin(self):
        self.lnz = 0.0

    def stage(self, state, beta, alpha, u):
        th, lnl, grad = state
        bn, dl, ess, w = oracle.smc_reweight(lnl, beta, alpha)
        self.lnz += dl
        cov = oracle.weighted_cov(th, w)
        anc = oracle.systematic_resample(w, u)
        th[:], lnl[:], grad[:] = th[anc], lnl[anc], grad[anc]
        return bn, dl, self.lnz, cov, anc

    def mutate(self, first, state, beta, cov, metric, eps_scale, max_depth, n_mut, key, ctr):
        th, lnl, grad = state
        ids = first + np.arange(th.shape[0], dtype=np.int64)
        if metric == 2:
            # each row's local metric at the new temperature (Sec. 5): needs only the row itself
            minv = oracle.local_inv_mass(self.model, self.event, th, beta)
            th, lnl, grad, _ = oracle.nuts_mutate_local(self.model, self.event, beta, th, lnl, grad, minv, eps_scale,
                                                        max_depth, n_mut, key, ctr, ids=ids)
            return th, lnl, grad
        if metric == 0:
            eps = eps_scale * min(math.sqrt(cov[j, j]) for j in range(cov.shape[0]))
            minv = None
        else:
            eps, minv = eps_scale, cov
        th, lnl, grad, _ = oracle.nuts_mutate(self.model, self.event, beta, th, lnl, grad, minv, eps, max_depth,
                                              n_mut, key, ctr, ids=ids)
        return th, lnl, grad

    def finish(self):
        pass
