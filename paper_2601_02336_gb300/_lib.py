"""ctypes binding of libsharpy (include/sharpy.h): argument marshalling only.

Every computation runs in the CUDA library; there is no CPU fallback. If the
library is missing or no GPU is visible, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

OK, EINVAL, ECUDA, ENOMEM, ENONFINITE, ETIMEOUT, EBOUNDS, ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
FP64, MIXED, MIXED_SPLIT = 0, 1, 2
MODEL_TAYLORF2, MODEL_GAUSSMIX = 0, 1


class Config(C.Structure):
    _fields_ = [("model", C.c_int), ("n_dim", C.c_int), ("phys", C.c_int * 11),
                ("lo", C.c_double * 11), ("hi", C.c_double * 11), ("prior", C.c_int * 11),
                ("boundary", C.c_int * 11), ("fixed", C.c_double * 11), ("n_comp", C.c_int),
                ("mix_logw", C.c_double * 4), ("mix_mu", (C.c_double * 11) * 4),
                ("mix_sigma", (C.c_double * 11) * 4)]


class Detector(C.Structure):
    _fields_ = [("lat", C.c_double), ("lon", C.c_double), ("azimuth", C.c_double),
                ("fixed_response", C.c_int), ("fplus", C.c_double), ("fcross", C.c_double),
                ("delay", C.c_double)]


class NutsStats(C.Structure):
    _fields_ = [("accept_sum", C.c_double), ("active_bins", C.c_double), ("depth_sum", C.c_int),
                ("n_leapfrog", C.c_int), ("n_divergent", C.c_int), ("pad", C.c_int)]


class SmcOptions(C.Structure):
    _fields_ = [("n_particles", C.c_int64), ("alpha", C.c_double), ("n_mut", C.c_int),
                ("max_depth", C.c_int), ("metric", C.c_int), ("eps_scale", C.c_double),
                ("precision", C.c_int), ("max_stages", C.c_int), ("timing", C.c_int),
                ("pad", C.c_int), ("pool_theta", C.c_void_p), ("pool_lnl", C.c_void_p),
                ("pool_cap", C.c_int64)]


class Stage(C.Structure):
    _fields_ = [("beta", C.c_double), ("dbeta", C.c_double), ("ess", C.c_double),
                ("dlnz", C.c_double), ("eps", C.c_double), ("accept_mean", C.c_double),
                ("depth_mean", C.c_double), ("n_leapfrog", C.c_int64), ("n_divergent", C.c_int),
                ("pad", C.c_int), ("active_bins", C.c_double), ("nuts_ms", C.c_double),
                ("reweight_ms", C.c_double), ("lnz", C.c_double)]


class BatchResult(C.Structure):
    _fields_ = [("lnz", C.c_double), ("beta", C.c_double), ("n_leapfrog", C.c_double),
                ("active_bins", C.c_double), ("n_stages", C.c_int), ("pad", C.c_int)]


_VP = C.c_void_p
_CTX = C.c_void_p
_SIGS = {
    "sharpy_create": (C.c_int, [C.POINTER(_CTX), C.POINTER(Config), C.c_int]),
    "sharpy_destroy": (None, [_CTX]),
    "sharpy_set_data": (C.c_int, [_CTX, C.c_int, C.c_int64, C.c_double, C.c_double, _VP, _VP,
                                  C.POINTER(Detector)]),
    "sharpy_prior_sample": (C.c_int, [_CTX, C.c_int64, _VP, C.c_uint64, C.c_uint64, _VP]),
    "sharpy_prior_logpdf_grad": (C.c_int, [_CTX, C.c_int64, _VP, _VP, _VP, _VP]),
    "sharpy_loglike_grad": (C.c_int, [_CTX, C.c_int64, _VP, _VP, _VP, C.c_int, _VP]),
    "sharpy_loglike_split": (C.c_int, [_CTX, C.c_int64, C.c_int, C.c_int]),
    "sharpy_set_loglike_split": (C.c_int, [_CTX, C.c_int]),
    "sharpy_waveform": (C.c_int, [_CTX, C.c_int64, _VP, _VP, _VP]),
    "sharpy_nuts_mutate": (C.c_int, [_CTX, C.c_int64, C.c_double, _VP, _VP, _VP, _VP, C.c_double,
                                     C.c_int, C.c_int, C.c_uint64, C.c_uint64, C.c_int, _VP, _VP]),
    "sharpy_smc_reweight_resample": (C.c_int, [_CTX, C.c_int64, _VP, _VP, _VP, C.c_double,
                                               C.c_double, C.c_double, _VP, _VP, _VP, _VP, _VP,
                                               _VP]),
    "sharpy_systematic_resample": (C.c_int, [C.c_int64, _VP, C.c_double, _VP, _VP]),
    "sharpy_systematic_resample_static": (C.c_int, [C.c_int64, _VP, C.c_double, _VP, _VP]),
    "sharpy_reset_evidence": (C.c_int, [_CTX, _VP]),
    "sharpy_set_evidence": (C.c_int, [_CTX, C.c_double, C.c_int, _VP]),
    "sharpy_log_evidence": (C.c_int, [_CTX, C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    "sharpy_smc_run": (C.c_int, [_CTX, C.POINTER(SmcOptions), C.c_uint64, C.POINTER(C.c_double),
                                 C.POINTER(C.c_int), _VP, _VP, C.POINTER(Stage), _VP]),
    "sharpy_batch_create": (C.c_int, [C.POINTER(_VP), C.POINTER(_CTX), C.c_int, C.POINTER(C.c_int64),
                                      C.POINTER(SmcOptions)]),
    "sharpy_batch_destroy": (None, [_VP]),
    "sharpy_batch_run": (C.c_int, [_VP, C.POINTER(C.c_uint64), C.POINTER(BatchResult),
                                   C.POINTER(C.c_int), _VP]),
    "sharpy_batch_particles": (C.c_int, [_VP, C.c_int, _VP, _VP, _VP]),
    "sharpy_batch_stages": (C.c_int, [_VP, C.c_int, C.POINTER(Stage), C.c_int, C.POINTER(C.c_int)]),
    "sharpy_batch_slots": (C.c_int, [_VP]),
    "sharpy_batch_set_slots": (C.c_int, [_VP, C.c_int]),
    "sharpy_batch_launches": (C.c_int64, [_VP]),
    "sharpy_nuts_mutate_cov_step": (C.c_int, [_CTX, C.c_int64, C.c_double, _VP, _VP, _VP, _VP, C.c_double,
                                              C.c_int, C.c_int, C.c_uint64, C.c_uint64, C.c_int, _VP, _VP]),
    "sharpy_set_nuts_tick_limit": (C.c_int, [_CTX, C.c_int64]),
    "sharpy_set_stage_test_hooks": (C.c_int, [_CTX, C.c_int, C.c_int]),
    "sharpy_set_nuts_slots": (C.c_int, [_CTX, C.c_int]),
    "sharpy_set_shard": (C.c_int, [_CTX, C.c_int64]),
    "sharpy_nuts_mutate_local": (C.c_int, [_CTX, C.c_int64, C.c_double, _VP, _VP, _VP, _VP, _VP, C.c_double,
                                           C.c_int, C.c_int, C.c_uint64, C.c_uint64, C.c_int, _VP, _VP]),
    "sharpy_local_metric": (C.c_int, [_CTX, C.c_int64, _VP, C.c_double, _VP, _VP, _VP, _VP]),
    "sharpy_recycle": (C.c_int, [C.c_int64, C.c_int, C.c_int, _VP, _VP, C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), C.c_uint64, _VP, _VP, C.POINTER(C.c_int64), _VP]),
    "sharpy_uniform2": (None, [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                C.POINTER(C.c_double)]),
    "sharpy_get_status": (C.c_int, [_CTX]),
    "sharpy_clear_status": (C.c_int, [_CTX]),
    "sharpy_error_string": (C.c_char_p, [C.c_int]),
    "sharpy_probe_peaks": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
}


class SharpyError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = lib().sharpy_error_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} ({code})")


def lib(build_if_missing: bool = True):
    """Load libsharpy (building it first if it is stale or missing)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing and not _build.up_to_date():
                _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libsharpy not built ({path}); run __graft_entry__.build()")
            h = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(h, name)
                f.restype = res
                f.argtypes = args
            _lib = h
    return _lib


def check(rc, where):
    if rc != OK:
        raise SharpyError(rc, where)
    return rc
