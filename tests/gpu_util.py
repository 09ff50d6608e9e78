"""Helpers of the GPU parity tests: error measures and a shared oracle setup."""
from __future__ import annotations

import os

import numpy as np
import pytest

from oracle import oracle as OR


def oracle():
    O = OR.default()
    O.set_threads(os.cpu_count() or 1)
    return O


def max_rel_err(got, ref, floor_rel=1e-14):
    """Per-cell relative error with a floor of floor_rel * max|ref| (needed
    where the reference is exactly zero); returns the maximum."""
    ref = np.asarray(ref)
    floor = floor_rel * max(float(np.abs(ref).max()), 1e-300)
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), floor)))


def rel_l1(got, ref):
    return float(np.abs(got - ref).sum() / max(np.abs(ref).sum(), 1e-300))


def require_gpu():
    try:
        import torch
        ok = torch.cuda.is_available()
    except Exception:
        ok = False
    if not ok:
        pytest.skip("no CUDA device")
