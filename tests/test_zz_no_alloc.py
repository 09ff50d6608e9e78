"""Totals through the allocation-free entry point, shasta_totals_noalloc.

That call exists for callers that cannot allocate device memory where they
need the totals (code running under another framework's memory pool, or code
that must not allocate after start-up); it keeps its partial sums in a fixed
array inside the library instead.  These tests check, through the C ABI, that
two calls in a row give the same sums as the ordinary shasta_totals, within
the totals tolerance of the other parity tests (1e-13 of the sum of absolute
values, since the two reduce in different orders), and that the size limit
is enforced before any GPU work.

The file is named to be collected last: a run that stops at its first failure
has run every other test by the time it gets here.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1206_0919_gb300 import shasta as S
from paper_1206_0919_gb300 import workloads as W
from gpu_util import require_gpu


def _close(got, ref, fields):
    scale = np.array([float(np.abs(f).sum()) for f in fields])
    return np.all(np.abs(got - ref) <= 1e-13 * scale + 1e-300), (got, ref)


def test_size_limit_rejected_before_any_gpu_work():
    """More cells than the fixed scratch holds: EINVAL, checked on the host
    before the pointers are touched (runs without a GPU)."""
    from paper_1206_0919_gb300 import build as B
    B.build()
    L = S.lib()
    fake = C.c_void_p(256)  # never dereferenced: the size check comes first
    st = L.shasta_totals_noalloc(fake, fake, fake, fake, fake,
                                 S.TOTALS_NOALLOC_MAX_CELLS + 1, fake, None)
    assert st == S.EINVAL
    st = L.shasta_totals_noalloc(fake, fake, fake, fake, fake, 16, None, None)
    assert st == S.EINVAL


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_totals_match_shasta_totals_twice(precision):
    """First call on a 64x60x56 grid (27 blocks of partials, the last one
    ragged), second call on a 40x36x32 grid (6 blocks, the last one ragged):
    the first call leaves partials of other data in every slot the second
    reads, so a second call that read a wrong block count or stride, or a
    slot it did not write, would pick them up and fail."""
    require_gpu()
    import torch
    dev = torch.device("cuda:0")
    out = torch.full((5,), float("nan"), dtype=torch.float64, device=dev)
    for shape, seed, steps in (((64, 60, 56), 11, 3), ((40, 36, 32), 12, 2)):
        prims = W.hot_spots(seed=seed, n_spots=6, radial_flow=0.3, shape=shape)
        with S.Solver(shape, precision=precision) as s:
            s.set_primitives(*prims.as_list())
            s.step(steps)
            ref = s.totals()
            fields = [torch.empty(s.grid_shape, dtype=torch.float64, device=dev)
                      for _ in range(5)]
            s.get_conserved(fields)
            torch.cuda.synchronize()
            out.fill_(float("nan"))
            S.totals_noalloc(*fields, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            host = [f.cpu().numpy() for f in fields]
        ok, info = _close(got, ref, host)
        assert ok, info
        # the sums are those of the fields themselves
        direct = np.array([math_fsum(h) for h in host])
        ok, info = _close(got, direct, host)
        assert ok, info


def math_fsum(a):
    import math
    return math.fsum(np.asarray(a, dtype=np.float64).ravel().tolist())
