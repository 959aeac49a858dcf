"""Shared pieces of the GPU parity tests: the same seeded event handed to both
the oracle and the CUDA library."""
import numpy as np
import pytest
import torch

from paper_2601_02336_gb300 import api, inputs
from tests import helpers


def require_gpu():
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a visible CUDA device")


def width(w):
    return np.array(w.hi) - np.array(w.lo)


def event_pair(w, seed=0, with_noise=True):
    """(oracle EventHolder, GPU Context, theta_inj, data) on identical arrays."""
    ev, th, data = helpers.make_event(w, seed, with_noise)
    ctx = api.Context.from_workload(w)
    ctx.set_data(data, inputs.psd_array(w), w.f_min, w.df, inputs.detectors(w))
    return ev, ctx, th, data


def to_dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def grad_rel_err(g, gref, wid):
    """Per-particle ||(g - g_ref) * width|| / ||g_ref * width||."""
    num = np.linalg.norm((g - gref) * wid[None, :], axis=1)
    den = np.linalg.norm(gref * wid[None, :], axis=1)
    return num / np.maximum(den, 1e-300)
