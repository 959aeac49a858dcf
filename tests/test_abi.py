"""The C-ABI library builds, loads and exports every entry point include/sharpy.h declares.
No compute calls: these run without a GPU."""
import ctypes as C
import os
import re

import pytest

from paper_2601_02336_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "sharpy.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sharpy_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ["sharpy_loglike_grad", "sharpy_nuts_mutate", "sharpy_smc_reweight_resample",
                     "sharpy_log_evidence", "sharpy_create", "sharpy_set_data", "sharpy_prior_sample",
                     "sharpy_systematic_resample", "sharpy_smc_run", "sharpy_get_status"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = _lib.lib()
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert getattr(lib, name) is not None


def test_error_strings():
    lib = _lib.lib()
    for code in range(-7, 1):
        assert len(lib.sharpy_error_string(code)) > 0
    assert lib.sharpy_error_string(-4) == b"non-finite value"


def test_argument_validation_without_device():
    lib = _lib.lib()
    # invalid sizes / uniforms are rejected before any device work
    assert lib.sharpy_systematic_resample(0, None, 0.5, None, None) == _lib.EINVAL
    assert lib.sharpy_systematic_resample(4, C.c_void_p(16), 1.0, C.c_void_p(16), None) == _lib.EINVAL
    out = C.c_void_p()
    cfg = _lib.Config()
    cfg.n_dim = 0
    assert lib.sharpy_create(C.byref(out), C.byref(cfg), 0) == _lib.EINVAL
    cfg.n_dim = 2
    cfg.lo[0], cfg.hi[0] = 1.0, 0.0  # empty box
    assert lib.sharpy_create(C.byref(out), C.byref(cfg), 0) == _lib.EINVAL
    assert lib.sharpy_loglike_grad(None, 1, None, None, None, 1, None) == _lib.EINVAL
    assert lib.sharpy_nuts_mutate(None, 1, 1.0, None, None, None, None, 0.1, 3, 1, 0, 0, 1, None,
                                  None) == _lib.EINVAL
