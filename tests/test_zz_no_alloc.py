"""The allocation-free systematic resampling entry point, called through the C ABI.

Some callers cannot allocate device memory once they are running (a service
that reserved its memory budget up front, or code that cannot afford the
synchronisation an allocation may cause). For them the library offers
sharpy_systematic_resample_static, whose scratch is a fixed array inside the
library. Its ancestors must equal those of the allocating entry point
(index work: bit-exact), on consecutive calls that reuse the shared array.
This file is collected last so a failure here comes after every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2601_02336_gb300 import _lib

pytestmark = pytest.mark.gpu


def _call(fn, w, u):
    anc = torch.full((w.shape[0],), -7, dtype=torch.int32, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(w.shape[0], C.c_void_p(w.data_ptr()), u, C.c_void_p(anc.data_ptr()), stream)
    torch.cuda.synchronize()
    return rc, anc


def test_static_resample_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a visible CUDA device")
    lib = _lib.lib()
    rng = np.random.default_rng(2024)
    # two calls in a row: a large one, then a smaller one that reuses the array
    for n in (200_003, 1_537):
        w = rng.uniform(0, 1, n) ** 4
        w[rng.integers(n)] = 1.0
        w[rng.uniform(size=n) < 0.1] = 0.0
        u = float(rng.uniform())
        wd = torch.tensor(w, dtype=torch.float64, device="cuda")
        rc_ref, ref = _call(lib.sharpy_systematic_resample, wd, u)
        rc, got = _call(lib.sharpy_systematic_resample_static, wd, u)
        assert rc_ref == 0 and rc == 0
        assert torch.equal(got, ref)
        assert int(got.min()) >= 0 and int(got.max()) < n


def test_static_resample_limits_and_flag_reset():
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a visible CUDA device")
    lib = _lib.lib()
    big = torch.zeros(262_145, dtype=torch.float64, device="cuda")
    rc, _ = _call(lib.sharpy_systematic_resample_static, big, 0.5)
    assert rc == _lib.EINVAL  # above the fixed maximum
    bad = torch.tensor([0.5, 2.0, 1.0], dtype=torch.float64, device="cuda")
    rc, _ = _call(lib.sharpy_systematic_resample_static, bad, 0.5)
    assert rc == _lib.EINVAL  # weight outside [0, 1]
    good = torch.tensor([0.5, 0.25, 1.0], dtype=torch.float64, device="cuda")
    rc, got = _call(lib.sharpy_systematic_resample_static, good, 0.5)
    rc_ref, ref = _call(lib.sharpy_systematic_resample, good, 0.5)
    assert rc == 0 and rc_ref == 0 and torch.equal(got, ref)


def test_static_resample_leaves_free_memory_unchanged():
    """The point of the entry point: once running it takes no device memory. After a warm-up call
    (which loads the kernels), 100 more calls leave the device's free memory as it was."""
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a visible CUDA device")
    lib = _lib.lib()
    rng = np.random.default_rng(7)
    wd = torch.tensor(rng.uniform(0, 1, 150_001), dtype=torch.float64, device="cuda")
    rc, ref = _call(lib.sharpy_systematic_resample_static, wd, 0.25)
    assert rc == 0
    free0, _ = torch.cuda.mem_get_info()
    for i in range(100):
        rc, got = _call(lib.sharpy_systematic_resample_static, wd, 0.25)
        assert rc == 0
    free1, _ = torch.cuda.mem_get_info()
    assert torch.equal(got, ref)
    assert free1 == free0, (free0, free1)
