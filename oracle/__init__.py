"""Oracle: plain FP64 CPU implementation of the sampler's hot path.

TEST INFRASTRUCTURE ONLY. The test suite, the smoke check and the
benchmark's CPU-baseline leg load it; the product library never does.
It shares no code with the CUDA library (see oracle.h for what each part
follows in the paper).

`build()` compiles model.cpp + sampler.cpp into _build/liboracle.so;
`lib()` loads it. The wrappers below only marshal numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_SRC = ["model.cpp", "sampler.cpp"]
_lock = threading.Lock()
_lib = None

MC, Q, CHI1, CHI2, DL, COSI, PHIC, PSI, RA, SINDEC, TC = range(11)
KIND_GW, KIND_GAUSSMIX = 0, 1
PRIOR_UNIFORM, PRIOR_POWER2 = 0, 1
BOUND_REFLECT, BOUND_PERIODIC = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, FP64, no FMA contraction)."""
    os.makedirs(os.path.join(_HERE, "_build"), exist_ok=True)
    srcs = [os.path.join(_HERE, s) for s in _SRC]
    deps = srcs + [os.path.join(_HERE, h) for h in ("oracle.h", "dual.h")]
    if not force and os.path.exists(_SO):
        t = os.path.getmtime(_SO)
        if all(os.path.getmtime(s) <= t for s in deps):
            return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp] + srcs
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Model(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_dim", C.c_int), ("phys", C.c_int * 11),
                ("lo", C.c_double * 11), ("hi", C.c_double * 11),
                ("prior", C.c_int * 11), ("boundary", C.c_int * 11),
                ("fixed", C.c_double * 11), ("n_comp", C.c_int),
                ("mix_logw", C.c_double * 4), ("mix_mu", (C.c_double * 11) * 4),
                ("mix_sigma", (C.c_double * 11) * 4)]


class Detector(C.Structure):
    _fields_ = [("lat", C.c_double), ("lon", C.c_double), ("azimuth", C.c_double),
                ("fixed_response", C.c_int), ("fplus", C.c_double), ("fcross", C.c_double),
                ("delay", C.c_double)]


class Event(C.Structure):
    _fields_ = [("n_det", C.c_int), ("n_bins", C.c_int64), ("f_min", C.c_double),
                ("df", C.c_double), ("data", C.POINTER(C.c_double)),
                ("psd", C.POINTER(C.c_double)), ("det", Detector * 4)]


class NutsStats(C.Structure):
    _fields_ = [("accept_sum", C.c_double), ("depth_sum", C.c_int), ("n_leapfrog", C.c_int),
                ("n_divergent", C.c_int)]


class SmcOpts(C.Structure):
    _fields_ = [("n_particles", C.c_int64), ("alpha", C.c_double), ("n_mut", C.c_int),
                ("max_depth", C.c_int), ("metric", C.c_int), ("eps_scale", C.c_double),
                ("max_stages", C.c_int)]


class Stage(C.Structure):
    _fields_ = [("beta", C.c_double), ("dbeta", C.c_double), ("ess", C.c_double),
                ("dlnz", C.c_double), ("eps", C.c_double), ("accept_mean", C.c_double),
                ("depth_mean", C.c_double), ("n_leapfrog", C.c_int64), ("n_divergent", C.c_int)]


_P = C.POINTER
_D = _P(C.c_double)
_SIGS = {
    "ref_philox4x32_10": (None, [_P(C.c_uint32), _P(C.c_uint32), _P(C.c_uint32)]),
    "ref_uniform2": (None, [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, _D]),
    "ref_normal2": (None, [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, _D]),
    "ref_antenna": (None, [_P(Detector), C.c_double, C.c_double, C.c_double, _D, _D, _D]),
    "ref_pn_phase": (C.c_double, [C.c_double] * 5),
    "ref_pn_phase_dmc": (C.c_double, [C.c_double] * 5),
    "ref_pn_beta": (C.c_double, [C.c_double] * 3),
    "ref_amplitude": (C.c_double, [C.c_double] * 3),
    "ref_f_isco": (C.c_double, [C.c_double] * 2),
    "ref_waveform": (C.c_int, [_P(Model), _P(Event), _D, _D]),
    "ref_loglike": (C.c_int, [_P(Model), _P(Event), C.c_int64, _D, _D, _D]),
    "ref_set_threads": (C.c_int, [C.c_int]),
    "ref_nuts_mutate_local": (C.c_int, [_P(Model), _P(Event), C.c_int64, C.c_double, _D, _D, _D, _D,
                                        C.c_double, C.c_int, C.c_int, C.c_uint64, C.c_uint32,
                                        _P(NutsStats)]),
    "ref_fisher": (C.c_int, [_P(Model), _P(Event), C.c_int64, _D, _D]),
    "ref_local_metric": (C.c_int, [_P(Model), _P(Event), C.c_int64, _D, C.c_double, _D]),
    "ref_local_inv_mass": (C.c_int, [_P(Model), _P(Event), C.c_int64, _D, C.c_double, _D]),
    "ref_nuts_mutate_local_ids": (C.c_int, [_P(Model), _P(Event), C.c_int64, _P(C.c_int64), C.c_double, _D, _D,
                                            _D, _D, C.c_double, C.c_int, C.c_int, C.c_uint64, C.c_uint32,
                                            _P(NutsStats)]),
    "ref_recycle_weights": (C.c_int, [C.c_int64, C.c_int, _D, _D, _D, _D]),
    "ref_rejection_sample": (C.c_int, [C.c_int64, _D, C.c_uint64, _P(C.c_int32)]),
    "ref_prior_sample": (C.c_int, [_P(Model), C.c_int64, _D, C.c_uint64, C.c_uint32]),
    "ref_prior_logpdf_grad": (C.c_int, [_P(Model), C.c_int64, _D, _D, _D]),
    "ref_nuts_mutate": (C.c_int, [_P(Model), _P(Event), C.c_int64, C.c_double, _D, _D, _D, _D,
                                  C.c_double, C.c_int, C.c_int, C.c_uint64, C.c_uint32,
                                  _P(NutsStats)]),
    "ref_nuts_mutate_ids": (C.c_int, [_P(Model), _P(Event), C.c_int64, _P(C.c_int64), C.c_double, _D, _D, _D,
                                      _D, C.c_double, C.c_int, C.c_int, C.c_uint64, C.c_uint32,
                                      _P(NutsStats)]),
    "ref_smc_reweight": (C.c_int, [C.c_int64, _D, C.c_double, C.c_double, _D, _D, _D, _D]),
    "ref_systematic_resample": (C.c_int, [C.c_int64, _D, C.c_double, _P(C.c_int32)]),
    "ref_weighted_cov": (C.c_int, [C.c_int, C.c_int64, _D, _D, _D]),
    "ref_smc_run": (C.c_int, [_P(Model), _P(Event), _P(SmcOpts), C.c_uint64, _D, _P(C.c_int),
                              _D, _D, _P(Stage)]),
}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            h = C.CDLL(_SO)
            for name, (res, args) in _SIGS.items():
                f = getattr(h, name)
                f.restype = res
                f.argtypes = args
            _lib = h
    return _lib


def _dp(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, name):
    if rc != 0:
        raise RuntimeError(f"oracle {name} returned {rc}")


# ------------------------------------------------------------- structures
def make_model(kind=KIND_GW, phys=(), lo=(), hi=(), prior=(), boundary=(), fixed=None,
               mix_logw=(), mix_mu=(), mix_sigma=()):
    m = Model()
    m.kind = kind
    m.n_dim = len(lo)
    for i in range(len(lo)):
        m.phys[i] = phys[i] if kind == KIND_GW else i
        m.lo[i] = lo[i]
        m.hi[i] = hi[i]
        m.prior[i] = prior[i] if prior else PRIOR_UNIFORM
        m.boundary[i] = boundary[i] if boundary else BOUND_REFLECT
    if fixed is not None:
        for i in range(11):
            m.fixed[i] = fixed[i]
    m.n_comp = len(mix_logw)
    for c in range(len(mix_logw)):
        m.mix_logw[c] = mix_logw[c]
        for i in range(m.n_dim):
            m.mix_mu[c][i] = mix_mu[c][i]
            m.mix_sigma[c][i] = mix_sigma[c][i]
    return m


class EventHolder:
    """Keeps the numpy buffers an Event points to alive."""

    def __init__(self, data, psd, f_min, df, detectors):
        self.data = _f64(data)
        self.psd = _f64(psd)
        n_det, n_bins = self.psd.shape
        assert self.data.shape == (n_det, n_bins, 2)
        ev = Event()
        ev.n_det = n_det
        ev.n_bins = n_bins
        ev.f_min = f_min
        ev.df = df
        ev.data = self.data.ctypes.data_as(_D)
        ev.psd = self.psd.ctypes.data_as(_D)
        for a, d in enumerate(detectors):
            ev.det[a] = make_detector(**d)
        self.ev = ev


def make_detector(lat=0.0, lon=0.0, azimuth=0.0, fixed_response=0, fplus=0.0, fcross=0.0, delay=0.0):
    return Detector(lat, lon, azimuth, fixed_response, fplus, fcross, delay)


# ------------------------------------------------------------------- calls
def philox(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().ref_philox4x32_10(c, k, o)
    return list(o)


def uniform2(key, c0, c1, c2, c3):
    u = np.zeros(2)
    lib().ref_uniform2(key, c0, c1, c2, c3, _dp(u))
    return u


def normal2(key, c0, c1, c2, c3):
    z = np.zeros(2)
    lib().ref_normal2(key, c0, c1, c2, c3, _dp(z))
    return z


def antenna(det: dict, ra, sin_dec, psi):
    d = make_detector(**det)
    fp, fc, dt = C.c_double(), C.c_double(), C.c_double()
    lib().ref_antenna(C.byref(d), ra, sin_dec, psi, C.byref(fp), C.byref(fc), C.byref(dt))
    return fp.value, fc.value, dt.value


def pn_phase(mc, q, chi1, chi2, f):
    return lib().ref_pn_phase(mc, q, chi1, chi2, f)


def pn_phase_dmc(mc, q, chi1, chi2, f):
    """d pn_phase / d mc at fixed q, spins and f (forward-mode dual numbers, no step size)."""
    return lib().ref_pn_phase_dmc(mc, q, chi1, chi2, f)


def pn_beta(q, chi1, chi2):
    return lib().ref_pn_beta(q, chi1, chi2)


def amplitude(mc, dl, f):
    return lib().ref_amplitude(mc, dl, f)


def f_isco(mc, q):
    return lib().ref_f_isco(mc, q)


def waveform(model, event: EventHolder, theta):
    theta = _f64(theta)
    h = np.zeros((event.ev.n_det, event.ev.n_bins, 2))
    _check(lib().ref_waveform(C.byref(model), C.byref(event.ev), _dp(theta), _dp(h)), "waveform")
    return h


def set_threads(n):
    """OpenMP threads of the particle loops (results do not depend on it); returns the previous value."""
    return lib().ref_set_threads(int(n))


def loglike(model, event, theta, grad=True):
    theta = _f64(np.atleast_2d(theta))
    n = theta.shape[0]
    lnl = np.zeros(n)
    g = np.zeros_like(theta) if grad else None
    evp = C.byref(event.ev) if event is not None else None
    _check(lib().ref_loglike(C.byref(model), evp, n, _dp(theta), _dp(lnl), _dp(g)), "loglike")
    return (lnl, g) if grad else lnl


def prior_sample(model, n, key, ctr=0):
    th = np.zeros((n, model.n_dim))
    _check(lib().ref_prior_sample(C.byref(model), n, _dp(th), key, ctr), "prior_sample")
    return th


def prior_logpdf_grad(model, theta):
    theta = _f64(np.atleast_2d(theta))
    lp = np.zeros(theta.shape[0])
    g = np.zeros_like(theta)
    _check(lib().ref_prior_logpdf_grad(C.byref(model), theta.shape[0], _dp(theta), _dp(lp), _dp(g)),
           "prior_logpdf_grad")
    return lp, g


def nuts_mutate(model, event, beta, theta, lnl, grad, inv_mass, step, max_depth, n_steps, key, ctr, ids=None):
    """ids: the rows' indices in the ensemble (they name each particle's random numbers); default 0..N-1."""
    theta = _f64(theta).copy()
    lnl = _f64(lnl).copy()
    grad = _f64(grad).copy()
    n = theta.shape[0]
    st = (NutsStats * n)()
    im = _f64(inv_mass) if inv_mass is not None else None
    evp = C.byref(event.ev) if event is not None else None
    if ids is None:
        _check(lib().ref_nuts_mutate(C.byref(model), evp, n, beta, _dp(theta), _dp(lnl), _dp(grad),
                                     _dp(im), step, max_depth, n_steps, key, ctr, st), "nuts_mutate")
    else:
        idv = np.ascontiguousarray(ids, dtype=np.int64)
        assert idv.shape == (n,)
        _check(lib().ref_nuts_mutate_ids(C.byref(model), evp, n, idv.ctypes.data_as(C.POINTER(C.c_int64)), beta,
                                         _dp(theta), _dp(lnl), _dp(grad), _dp(im), step, max_depth, n_steps, key,
                                         ctr, st), "nuts_mutate")
    stats = {
        "accept_sum": np.array([s.accept_sum for s in st]),
        "depth_sum": np.array([s.depth_sum for s in st]),
        "n_leapfrog": np.array([s.n_leapfrog for s in st]),
        "n_divergent": np.array([s.n_divergent for s in st]),
    }
    return theta, lnl, grad, stats


def nuts_mutate_local(model, event, beta, theta, lnl, grad, inv_mass, step, max_depth, n_steps, key, ctr,
                      ids=None):
    """nuts_mutate with one inverse mass matrix per particle (inv_mass [N][D][D]); ids as in nuts_mutate."""
    theta = _f64(theta).copy()
    lnl = _f64(lnl).copy()
    grad = _f64(grad).copy()
    n = theta.shape[0]
    st = (NutsStats * n)()
    im = _f64(inv_mass)
    evp = C.byref(event.ev) if event is not None else None
    if ids is None:
        _check(lib().ref_nuts_mutate_local(C.byref(model), evp, n, beta, _dp(theta), _dp(lnl), _dp(grad),
                                           _dp(im), step, max_depth, n_steps, key, ctr, st), "nuts_mutate_local")
    else:
        idv = np.ascontiguousarray(ids, dtype=np.int64)
        assert idv.shape == (n,)
        _check(lib().ref_nuts_mutate_local_ids(C.byref(model), evp, n, idv.ctypes.data_as(C.POINTER(C.c_int64)),
                                               beta, _dp(theta), _dp(lnl), _dp(grad), _dp(im), step, max_depth,
                                               n_steps, key, ctr, st), "nuts_mutate_local")
    stats = {
        "accept_sum": np.array([s.accept_sum for s in st]),
        "depth_sum": np.array([s.depth_sum for s in st]),
        "n_leapfrog": np.array([s.n_leapfrog for s in st]),
        "n_divergent": np.array([s.n_divergent for s in st]),
    }
    return theta, lnl, grad, stats


def smc_reweight(lnl, beta_prev, alpha):
    lnl = _f64(lnl)
    n = lnl.shape[0]
    w = np.zeros(n)
    bn, dl, ess = C.c_double(), C.c_double(), C.c_double()
    _check(lib().ref_smc_reweight(n, _dp(lnl), beta_prev, alpha, C.byref(bn), C.byref(dl),
                                  C.byref(ess), _dp(w)), "smc_reweight")
    return bn.value, dl.value, ess.value, w


def systematic_resample(w, u):
    w = _f64(w)
    anc = np.zeros(w.shape[0], dtype=np.int32)
    _check(lib().ref_systematic_resample(w.shape[0], _dp(w), u,
                                         anc.ctypes.data_as(_P(C.c_int32))), "systematic_resample")
    return anc


def weighted_cov(theta, w):
    theta = _f64(theta)
    n, d = theta.shape
    cov = np.zeros((d, d))
    _check(lib().ref_weighted_cov(d, n, _dp(theta), _dp(_f64(w)), _dp(cov)), "weighted_cov")
    return cov


def smc_run(model, event, n_particles, alpha, n_mut, max_depth, metric, eps_scale, key,
            max_stages=500):
    o = SmcOpts(n_particles, alpha, n_mut, max_depth, metric, eps_scale, max_stages)
    lnz = C.c_double()
    ns = C.c_int()
    th = np.zeros((n_particles, model.n_dim))
    lnl = np.zeros(n_particles)
    stages = (Stage * max_stages)()
    evp = C.byref(event.ev) if event is not None else None
    rc = lib().ref_smc_run(C.byref(model), evp, C.byref(o), key, C.byref(lnz), C.byref(ns),
                           _dp(th), _dp(lnl), stages)
    if rc not in (0,):
        raise RuntimeError(f"oracle smc_run did not reach beta = 1 (rc={rc})")
    rec = [dict((f, getattr(stages[i], f)) for f, _ in Stage._fields_) for i in range(ns.value)]
    return lnz.value, th, lnl, rec


def recycle_weights(lnl, beta, lnz_t):
    """ln w of pooled particles for the final target (Sec. 5, sample recycling)."""
    lnl = _f64(lnl)
    beta = _f64(beta)
    lnz_t = _f64(lnz_t)
    out = np.zeros(lnl.shape[0])
    _check(lib().ref_recycle_weights(lnl.shape[0], beta.shape[0], _dp(lnl), _dp(beta), _dp(lnz_t), _dp(out)),
           "recycle_weights")
    return out


def rejection_sample(log_w, key):
    """0/1 keep flags of the rejection step of sample recycling."""
    log_w = _f64(log_w)
    keep = np.zeros(log_w.shape[0], dtype=np.int32)
    _check(lib().ref_rejection_sample(log_w.shape[0], _dp(log_w), key,
                                      keep.ctypes.data_as(C.POINTER(C.c_int32))), "rejection_sample")
    return keep


def fisher(model, event, theta):
    """Fisher information <d_j h | d_k h> at each parameter vector: [N][D][D]."""
    theta = _f64(np.atleast_2d(theta))
    n, d = theta.shape
    out = np.zeros((n, d, d))
    _check(lib().ref_fisher(C.byref(model), C.byref(event.ev), n, _dp(theta), _dp(out)), "fisher")
    return out


def local_inv_mass(model, event, theta, beta):
    """The inverse mass matrices [N][D][D] smc_run's metric 2 mutates with at beta."""
    theta = _f64(np.atleast_2d(theta))
    n, d = theta.shape
    out = np.zeros((n, d, d))
    evp = C.byref(event.ev) if event is not None else None
    _check(lib().ref_local_inv_mass(C.byref(model), evp, n, _dp(theta), beta, _dp(out)), "local_inv_mass")
    return out


def local_metric(model, event, theta, beta):
    """Per-particle mass matrix beta F + prior Hessian + box precision: [N][D][D]."""
    theta = _f64(np.atleast_2d(theta))
    n, d = theta.shape
    out = np.zeros((n, d, d))
    evp = C.byref(event.ev) if event is not None else None
    _check(lib().ref_local_metric(C.byref(model), evp, n, _dp(theta), beta, _dp(out)), "local_metric")
    return out
