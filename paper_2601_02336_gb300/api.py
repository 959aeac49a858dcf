"""Python face of libsharpy: tensors in, tensors out, arguments marshalled.

Device memory and streams come from PyTorch; every step of the sampler's hot
path runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import inputs
from ._lib import (FP64, MIXED, MIXED_SPLIT, MODEL_GAUSSMIX, MODEL_TAYLORF2, BatchResult, Config, Detector,
                   NutsStats, SmcOptions, Stage, check, lib)

PRECISION = {"fp64": FP64, "mixed": MIXED, "split": MIXED_SPLIT}
STATS_DTYPE = np.dtype([("accept_sum", "<f8"), ("active_bins", "<f8"), ("depth_sum", "<i4"),
                        ("n_leapfrog", "<i4"), ("n_divergent", "<i4"), ("pad", "<i4")])


def _prec(p):
    return PRECISION[p] if isinstance(p, str) else int(p)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, what):
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError(f"{what} must be a contiguous float64 CUDA tensor")
    return t


def config_from_workload(w: inputs.Workload) -> Config:
    c = Config()
    c.model = MODEL_TAYLORF2
    c.n_dim = w.n_dim
    for i in range(w.n_dim):
        c.phys[i] = w.phys[i]
        c.lo[i] = w.lo[i]
        c.hi[i] = w.hi[i]
        c.prior[i] = w.prior[i]
        c.boundary[i] = w.boundary[i]
    for i in range(11):
        c.fixed[i] = w.fixed[i]
    return c


def gaussmix_config(lo, hi, logw, mu, sigma, boundary=None) -> Config:
    c = Config()
    c.model = MODEL_GAUSSMIX
    c.n_dim = len(lo)
    for i in range(len(lo)):
        c.phys[i] = i
        c.lo[i] = lo[i]
        c.hi[i] = hi[i]
        c.prior[i] = 0
        c.boundary[i] = boundary[i] if boundary else 0
    c.n_comp = len(logw)
    for k in range(len(logw)):
        c.mix_logw[k] = logw[k]
        for i in range(len(lo)):
            c.mix_mu[k][i] = mu[k][i]
            c.mix_sigma[k][i] = sigma[k][i]
    return c


class Context:
    """A sharpy context bound to one CUDA device."""

    def __init__(self, config: Config, device: int = 0):
        self._h = C.c_void_p()
        self.n_dim = config.n_dim
        self.device = device
        self.n_det = 0
        self.n_bins = 0
        check(lib().sharpy_create(C.byref(self._h), C.byref(config), device), "sharpy_create")

    @classmethod
    def from_workload(cls, w: inputs.Workload, device: int = 0):
        return cls(config_from_workload(w), device)

    def close(self):
        if self._h:
            lib().sharpy_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- data
    def set_data(self, data, psd, f_min, df, detectors):
        data = np.ascontiguousarray(data, dtype=np.float64)
        psd = np.ascontiguousarray(psd, dtype=np.float64)
        n_det, n_bins = psd.shape
        dets = (Detector * max(1, n_det))()
        for a, d in enumerate(detectors):
            dets[a] = Detector(d.get("lat", 0.0), d.get("lon", 0.0), d.get("azimuth", 0.0),
                               d.get("fixed_response", 0), d.get("fplus", 0.0), d.get("fcross", 0.0),
                               d.get("delay", 0.0))
        check(lib().sharpy_set_data(self._h, n_det, n_bins, f_min, df,
                                    data.ctypes.data_as(C.c_void_p), psd.ctypes.data_as(C.c_void_p),
                                    dets), "sharpy_set_data")
        self.n_det, self.n_bins = n_det, n_bins

    # ---------------------------------------------------------- likelihood
    def loglike_grad(self, theta, precision="mixed", grad=True, out=None):
        theta = _dev(theta, "theta")
        n = theta.shape[0]
        lnl = torch.empty(n, dtype=torch.float64, device=theta.device) if out is None else out[0]
        g = (torch.empty_like(theta) if out is None else out[1]) if grad else None
        check(lib().sharpy_loglike_grad(self._h, n, _ptr(theta), _ptr(lnl), _ptr(g), _prec(precision),
                                        _stream()), "sharpy_loglike_grad")
        return lnl, g

    def loglike_split(self, n, precision="mixed", grad=True):
        """Warps per vector the likelihood call's tuner picked for n vectors (0: not tuned yet)."""
        return lib().sharpy_loglike_split(self._h, int(n), _prec(precision), 1 if grad else 0)

    def set_loglike_split(self, split):
        """Force 1, 2, 4 or 8 warps per vector, or 16 (the staged kernel of long segments, mixed and split
        paths; 8 where it does not apply), in later likelihood calls (0: tune)."""
        check(lib().sharpy_set_loglike_split(self._h, int(split)), "sharpy_set_loglike_split")

    def set_nuts_slots(self, slots):
        """Force 4, 8, 16 or 32 NUTS particle slots per CTA in later single-event launches (0: tuned/default)."""
        check(lib().sharpy_set_nuts_slots(self._h, int(slots)), "sharpy_set_nuts_slots")

    def set_stage_test_hooks(self, skip_block=-1, wait_polls=0):
        """Failure-detection tests of the staged likelihood kernel: leave out the bulk copy of table block
        `skip_block` (-1: none) and poll each mbarrier wait at most `wait_polls` times (0: the default)."""
        check(lib().sharpy_set_stage_test_hooks(self._h, int(skip_block), int(wait_polls)),
              "sharpy_set_stage_test_hooks")

    def waveform(self, theta):
        theta = _dev(theta, "theta")
        h = torch.empty((theta.shape[0], self.n_det, self.n_bins, 2), dtype=torch.float64,
                        device=theta.device)
        check(lib().sharpy_waveform(self._h, theta.shape[0], _ptr(theta), _ptr(h), _stream()),
              "sharpy_waveform")
        return h

    def prior_sample(self, n, key, ctr=0):
        th = torch.empty((n, self.n_dim), dtype=torch.float64, device=f"cuda:{self.device}")
        check(lib().sharpy_prior_sample(self._h, n, _ptr(th), key, ctr, _stream()), "sharpy_prior_sample")
        return th

    def prior_logpdf_grad(self, theta):
        theta = _dev(theta, "theta")
        lp = torch.empty(theta.shape[0], dtype=torch.float64, device=theta.device)
        g = torch.empty_like(theta)
        check(lib().sharpy_prior_logpdf_grad(self._h, theta.shape[0], _ptr(theta), _ptr(lp), _ptr(g),
                                             _stream()), "sharpy_prior_logpdf_grad")
        return lp, g

    # ------------------------------------------------------------- sampler
    def nuts_mutate(self, beta, theta, lnl, grad, inv_mass, step, max_depth, n_steps, key, ctr,
                    precision="mixed", stats=True):
        """In-place NUTS transitions; returns the per-particle stats as a uint8 device buffer."""
        n = theta.shape[0]
        st = torch.empty(n * STATS_DTYPE.itemsize, dtype=torch.uint8, device=theta.device) if stats else None
        check(lib().sharpy_nuts_mutate(self._h, n, beta, _ptr(_dev(theta, "theta")), _ptr(_dev(lnl, "lnl")),
                                       _ptr(_dev(grad, "grad")), _ptr(inv_mass), step, max_depth, n_steps,
                                       key, ctr, _prec(precision), _ptr(st), _stream()),
              "sharpy_nuts_mutate")
        return st

    def nuts_mutate_local(self, beta, theta, lnl, grad, inv_mass, chol, step, max_depth, n_steps, key, ctr,
                          precision="mixed", stats=True):
        """nuts_mutate with one metric per particle (inv_mass, chol: [N][D][D] device)."""
        n = theta.shape[0]
        st = torch.empty(n * STATS_DTYPE.itemsize, dtype=torch.uint8, device=theta.device) if stats else None
        check(lib().sharpy_nuts_mutate_local(self._h, n, beta, _ptr(_dev(theta, "theta")), _ptr(_dev(lnl, "lnl")),
                                             _ptr(_dev(grad, "grad")), _ptr(_dev(inv_mass, "inv_mass")),
                                             _ptr(_dev(chol, "chol")), step, max_depth, n_steps, key, ctr,
                                             _prec(precision), _ptr(st), _stream()), "sharpy_nuts_mutate_local")
        return st

    def nuts_mutate_cov_step(self, beta, theta, lnl, grad, cov, eps_scale, max_depth, n_steps, key, ctr,
                             precision="mixed", stats=True):
        """nuts_mutate with the identity metric and step = eps_scale * min_j sqrt(cov[j][j]), the step
        taken on the device from the weighted covariance cov [D][D] (device)."""
        n = theta.shape[0]
        st = torch.empty(n * STATS_DTYPE.itemsize, dtype=torch.uint8, device=theta.device) if stats else None
        check(lib().sharpy_nuts_mutate_cov_step(self._h, n, beta, _ptr(_dev(theta, "theta")), _ptr(_dev(lnl, "lnl")),
                                                _ptr(_dev(grad, "grad")), _ptr(_dev(cov, "cov")), eps_scale,
                                                max_depth, n_steps, key, ctr, _prec(precision), _ptr(st),
                                                _stream()), "sharpy_nuts_mutate_cov_step")
        return st

    def set_shard(self, first_id):
        """Later prior draws and NUTS calls act on rows first_id.. of a larger ensemble (sharpy_set_shard)."""
        check(lib().sharpy_set_shard(self._h, int(first_id)), "sharpy_set_shard")

    def set_nuts_tick_limit(self, max_ticks):
        """Lower the NUTS kernel's tick bound (failure-detection tests); 0 restores the default."""
        check(lib().sharpy_set_nuts_tick_limit(self._h, int(max_ticks)), "sharpy_set_nuts_tick_limit")

    @staticmethod
    def stats_to_numpy(st):
        return np.frombuffer(st.cpu().numpy().tobytes(), dtype=STATS_DTYPE)

    def reweight_resample(self, theta, lnl, grad, beta_prev, alpha, u, want_cov=True):
        n, d = theta.shape
        dev = theta.device
        sc = torch.zeros(3, dtype=torch.float64, device=dev)
        anc = torch.empty(n, dtype=torch.int32, device=dev)
        cov = torch.empty((d, d), dtype=torch.float64, device=dev) if want_cov else None
        check(lib().sharpy_smc_reweight_resample(
            self._h, n, _ptr(theta), _ptr(lnl), _ptr(grad), beta_prev, alpha, u,
            C.c_void_p(sc.data_ptr()), C.c_void_p(sc.data_ptr() + 8), C.c_void_p(sc.data_ptr() + 16),
            _ptr(anc), _ptr(cov), _stream()), "sharpy_smc_reweight_resample")
        return {"beta_next": sc[0], "dlnz": sc[1], "ess": sc[2], "ancestors": anc, "cov": cov}

    def reset_evidence(self):
        check(lib().sharpy_reset_evidence(self._h, _stream()), "sharpy_reset_evidence")

    def set_evidence(self, lnz, n_stages):
        check(lib().sharpy_set_evidence(self._h, float(lnz), int(n_stages), _stream()), "sharpy_set_evidence")

    def log_evidence(self):
        lnz = C.c_double()
        ns = C.c_int()
        check(lib().sharpy_log_evidence(self._h, C.byref(lnz), C.byref(ns)), "sharpy_log_evidence")
        return lnz.value, ns.value

    def smc_run(self, n_particles, alpha, n_mut, max_depth, metric, eps_scale, key,
                precision="mixed", max_stages=500, timing=False, pool_stages=0):
        """Full SMC run. pool_stages > 0 also returns the sample-recycling pool:
        (lnz, theta, lnl, records, pool_theta, pool_lnl) with the particles after
        each of the first pool_stages stages."""
        o = SmcOptions(n_particles, alpha, n_mut, max_depth, metric, eps_scale, _prec(precision), max_stages,
                       1 if timing else 0, 0)
        dev = f"cuda:{self.device}"
        th = torch.empty((n_particles, self.n_dim), dtype=torch.float64, device=dev)
        ll = torch.empty(n_particles, dtype=torch.float64, device=dev)
        if pool_stages > 0:
            cap = pool_stages * n_particles
            pth = torch.empty((cap, self.n_dim), dtype=torch.float64, device=dev)
            pll = torch.empty(cap, dtype=torch.float64, device=dev)
            o.pool_theta, o.pool_lnl, o.pool_cap = pth.data_ptr(), pll.data_ptr(), cap
        stages = (Stage * max_stages)()
        lnz = C.c_double()
        ns = C.c_int()
        check(lib().sharpy_smc_run(self._h, C.byref(o), key, C.byref(lnz), C.byref(ns), _ptr(th), _ptr(ll),
                                   stages, _stream()), "sharpy_smc_run")
        rec = [dict((f, getattr(stages[i], f)) for f, _ in Stage._fields_ if f != "pad")
               for i in range(ns.value)]
        if pool_stages > 0:
            rows = min(len(rec), pool_stages) * n_particles
            return lnz.value, th, ll, rec, pth[:rows], pll[:rows]
        return lnz.value, th, ll, rec

    def local_metric(self, theta, beta, want=("mass", "inv_mass", "chol")):
        """Per-particle mass matrices (sharpy_local_metric): dict of [N][D][D] tensors."""
        theta = _dev(theta, "theta")
        n, d = theta.shape
        out = {k: torch.empty((n, d, d), dtype=torch.float64, device=theta.device) for k in want}
        check(lib().sharpy_local_metric(self._h, n, _ptr(theta), beta, _ptr(out.get("mass")),
                                        _ptr(out.get("inv_mass")), _ptr(out.get("chol")), _stream()),
              "sharpy_local_metric")
        return out

    def status(self):
        return lib().sharpy_get_status(self._h)

    def clear_status(self):
        check(lib().sharpy_clear_status(self._h), "sharpy_clear_status")


def uniform2(key, c0, c1, c2, c3):
    """The kernels' Philox4x32-10 uniforms at one counter (sharpy_uniform2)."""
    u = (C.c_double * 2)()
    lib().sharpy_uniform2(key, c0, c1, c2, c3, u)
    return u[0], u[1]


class SMCRunner:
    """The SMC loop of sharpy_smc_run driven stage by stage from the host through
    the public calls (reweight/resample, local metric, NUTS), with checkpoints
    at stage boundaries. It draws the same random numbers as sharpy_smc_run, so
    a run matches sharpy_smc_run with the same key bit for bit, and a run
    restored from a checkpoint continues exactly as the uninterrupted one."""

    RESAMPLE = 6        # Philox purpose of the resampling uniform
    STAGE_COUNTER = 256  # NUTS step counters of stage t start at t * 256

    def __init__(self, ctx, n_particles, alpha, n_mut, max_depth, metric, eps_scale, key, precision="mixed",
                 max_stages=500):
        self.ctx = ctx
        self.opts = dict(n_particles=int(n_particles), alpha=float(alpha), n_mut=int(n_mut),
                         max_depth=int(max_depth), metric=int(metric), eps_scale=float(eps_scale), key=int(key),
                         precision=precision, max_stages=int(max_stages))
        self.theta = self.lnl = self.grad = None
        self.beta, self.lnz, self.stage = 0.0, 0.0, 0
        self.records = []

    def start(self):
        o = self.opts
        self.theta = self.ctx.prior_sample(o["n_particles"], o["key"], 0)
        self.lnl, self.grad = self.ctx.loglike_grad(self.theta, o["precision"])
        self.ctx.reset_evidence()
        self.beta, self.lnz, self.stage, self.records = 0.0, 0.0, 0, []
        return self

    @property
    def done(self):
        return self.beta >= 1.0 or self.stage >= self.opts["max_stages"]

    def step(self):
        """One stage: reweight, resample, metric, n_mut NUTS transitions."""
        o = self.opts
        self.stage += 1
        t = self.stage
        u = uniform2(o["key"], 0, t, self.RESAMPLE, 0)[0]
        r = self.ctx.reweight_resample(self.theta, self.lnl, self.grad, self.beta, o["alpha"], u)
        beta_next, dlnz = float(r["beta_next"]), float(r["dlnz"])
        args = (o["max_depth"], o["n_mut"], o["key"], t * self.STAGE_COUNTER)
        if o["metric"] == 2:
            met = self.ctx.local_metric(self.theta, beta_next, want=("inv_mass", "chol"))
            st = self.ctx.nuts_mutate_local(beta_next, self.theta, self.lnl, self.grad, met["inv_mass"], met["chol"],
                                            o["eps_scale"], *args, precision=o["precision"])
        elif o["metric"] == 1:
            st = self.ctx.nuts_mutate(beta_next, self.theta, self.lnl, self.grad, r["cov"], o["eps_scale"], *args,
                                      precision=o["precision"])
        else:
            st = self.ctx.nuts_mutate_cov_step(beta_next, self.theta, self.lnl, self.grad, r["cov"], o["eps_scale"],
                                               *args, precision=o["precision"])
        s = Context.stats_to_numpy(st)
        # ln Z: the context's device accumulator of the stage increments (Eq. 8)
        lnz, _ = self.ctx.log_evidence()
        self.records.append({"beta": beta_next, "dlnz": dlnz, "ess": float(r["ess"]),
                             "n_leapfrog": int(s["n_leapfrog"].sum()), "lnz": lnz})
        self.beta = beta_next
        self.lnz = lnz
        return self

    def run(self):
        if self.theta is None:
            self.start()
        while not self.done:
            self.step()
        return self.lnz

    def save(self, path):
        """Checkpoint at a stage boundary (.npz)."""
        np.savez(path, theta=self.theta.cpu().numpy(), lnl=self.lnl.cpu().numpy(), grad=self.grad.cpu().numpy(),
                 scalars=np.array([self.beta, self.lnz, self.stage], dtype=np.float64),
                 opts=np.array(repr(self.opts)), records=np.array(repr(self.records)))

    @classmethod
    def load(cls, ctx, path):
        import ast
        z = np.load(path, allow_pickle=False)
        r = cls(ctx, **ast.literal_eval(str(z["opts"])))
        dev = f"cuda:{ctx.device}"
        r.theta = torch.tensor(z["theta"], dtype=torch.float64, device=dev)
        r.lnl = torch.tensor(z["lnl"], dtype=torch.float64, device=dev)
        r.grad = torch.tensor(z["grad"], dtype=torch.float64, device=dev)
        beta, lnz, stage = (float(x) for x in z["scalars"])
        r.beta, r.lnz, r.stage = beta, lnz, int(stage)
        ctx.set_evidence(lnz, int(stage))
        r.records = ast.literal_eval(str(z["records"]))
        return r


class Batch:
    """Many events sampled together (sharpy_batch_*): one persistent NUTS launch
    and one reweight launch per stage round cover every event still tempering;
    the rounds replay a captured CUDA graph. Keeps references to the contexts."""

    def __init__(self, contexts, n_particles, alpha, n_mut, max_depth, metric, eps_scale, precision="mixed",
                 max_stages=500):
        self.contexts = list(contexts)
        self.n_particles = [int(n) for n in n_particles]
        if len(self.n_particles) != len(self.contexts):
            raise ValueError("one particle count per context")
        self.max_stages = max_stages
        o = SmcOptions(0, alpha, n_mut, max_depth, metric, eps_scale, _prec(precision), max_stages, 0, 0)
        ne = len(self.contexts)
        hs = (C.c_void_p * ne)(*[c._h.value for c in self.contexts])
        ns = (C.c_int64 * ne)(*self.n_particles)
        h = C.c_void_p()
        check(lib().sharpy_batch_create(C.byref(h), hs, ne, ns, C.byref(o)), "sharpy_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().sharpy_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, keys):
        """Run every event to beta = 1. Returns (list of result dicts, rounds)."""
        ne = len(self.contexts)
        if len(keys) != ne:
            raise ValueError("one key per event")
        k = (C.c_uint64 * ne)(*[int(x) for x in keys])
        res = (BatchResult * ne)()
        rounds = C.c_int()
        check(lib().sharpy_batch_run(self._h, k, res, C.byref(rounds), _stream()), "sharpy_batch_run")
        out = [dict((f, getattr(res[e], f)) for f, _ in BatchResult._fields_ if f != "pad") for e in range(ne)]
        return out, rounds.value

    def particles(self, e):
        c = self.contexts[e]
        th = torch.empty((self.n_particles[e], c.n_dim), dtype=torch.float64, device=f"cuda:{c.device}")
        ll = torch.empty(self.n_particles[e], dtype=torch.float64, device=th.device)
        check(lib().sharpy_batch_particles(self._h, e, _ptr(th), _ptr(ll), _stream()), "sharpy_batch_particles")
        return th, ll

    def stages(self, e):
        st = (Stage * self.max_stages)()
        n = C.c_int()
        check(lib().sharpy_batch_stages(self._h, e, st, self.max_stages, C.byref(n)), "sharpy_batch_stages")
        return [dict((f, getattr(st[i], f)) for f, _ in Stage._fields_ if f != "pad") for i in range(n.value)]

    @property
    def slots(self):
        return lib().sharpy_batch_slots(self._h)

    @slots.setter
    def slots(self, value):
        check(lib().sharpy_batch_set_slots(self._h, int(value)), "sharpy_batch_set_slots")

    @property
    def launches(self):
        """Kernels the last run launched (sharpy_batch_launches)."""
        return int(lib().sharpy_batch_launches(self._h))


def recycle(theta, lnl, betas, lnz_t, key):
    """Sample recycling (sharpy_recycle): importance weights of a pool drawn from
    the stages' mixture, and the i.i.d. draws the rejection step keeps.
    theta [m][d], lnl [m] device; betas, lnz_t: one entry per pooled stage.
    Returns (log_w [m], kept theta [n_kept][d])."""
    theta = _dev(theta, "theta")
    lnl = _dev(lnl, "lnl")
    m, d = theta.shape
    t = len(betas)
    b = (C.c_double * t)(*[float(x) for x in betas])
    z = (C.c_double * t)(*[float(x) for x in lnz_t])
    lw = torch.empty(m, dtype=torch.float64, device=theta.device)
    out = torch.empty_like(theta)
    n = C.c_int64()
    check(lib().sharpy_recycle(m, d, t, _ptr(theta), _ptr(lnl), b, z, key, _ptr(lw), _ptr(out), C.byref(n),
                               _stream()), "sharpy_recycle")
    return lw, out[:n.value]


def recycle_run(pool_theta, pool_lnl, records, n_particles, key):
    """Recycle the pool of an smc_run(..., pool_stages=T): its stages' beta and running ln Z (the stage
    records' device-accumulated ln Z)."""
    t = pool_theta.shape[0] // n_particles
    betas = [r["beta"] for r in records[:t]]
    lnz_t = [r["lnz"] for r in records[:t]]
    return recycle(pool_theta, pool_lnl, betas, lnz_t, key)


def systematic_resample(w, u):
    """Bit-exact systematic resampling of device weights w (float64, in [0,1])."""
    w = _dev(w, "w")
    anc = torch.empty(w.shape[0], dtype=torch.int32, device=w.device)
    check(lib().sharpy_systematic_resample(w.shape[0], _ptr(w), u, _ptr(anc), _stream()),
          "sharpy_systematic_resample")
    return anc


class LogLikelihood(torch.autograd.Function):
    """ln L(theta) with the hand-written adjoint as its backward pass.

    forward: the forward-only sweep (no basis moments); backward: the gradient
    sweep, which recomputes the waveform in registers instead of storing the
    particles x bins complex strain.
    """

    @staticmethod
    def forward(ctx, theta, sctx, precision):
        lnl, _ = sctx.loglike_grad(theta.detach().contiguous(), precision, grad=False)
        ctx.save_for_backward(theta)
        ctx.sctx = sctx
        ctx.precision = precision
        return lnl

    @staticmethod
    def backward(ctx, gout):
        (theta,) = ctx.saved_tensors
        _, g = ctx.sctx.loglike_grad(theta.detach().contiguous(), ctx.precision, grad=True)
        return gout[:, None] * g, None, None


def loglike(theta, sctx, precision="mixed"):
    return LogLikelihood.apply(theta, sctx, precision)


# --------------------------------------------------------------- injections
def make_event(w: inputs.Workload, seed=0, device=0, with_noise=True):
    """Synthetic event through the library: h(theta_inj) from sharpy_waveform,
    distance rescaled to the target SNR using SNR^2 = -2 ln L with zero data,
    plus seeded Gaussian noise. Returns (Context, theta_inj, data)."""
    ctx = Context.from_workload(w, device)
    psd = inputs.psd_array(w)
    dets = inputs.detectors(w)
    zeros = np.zeros((w.n_det, w.n_bins, 2))
    ctx.set_data(zeros, psd, w.f_min, w.df, dets)
    th = inputs.injection(w, seed).copy()
    k = inputs.distance_index(w)
    dev = f"cuda:{device}"
    if w.snr_target is not None and k is not None:
        t = torch.tensor(th[None, :], dtype=torch.float64, device=dev)
        lnl, _ = ctx.loglike_grad(t, "fp64", grad=False)
        rho = math.sqrt(-2.0 * float(lnl[0]))
        th[k] = min(max(th[k] * rho / w.snr_target, w.lo[k]), w.hi[k])
    h = ctx.waveform(torch.tensor(th[None, :], dtype=torch.float64, device=dev))[0].cpu().numpy()
    data = h + (inputs.noise(w, seed) if with_noise else 0.0)
    ctx.set_data(data, psd, w.f_min, w.df, dets)
    return ctx, th, data
