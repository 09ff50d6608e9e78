"""The C ABI library loads and exports every function include/*.h declares
(no compute calls: this runs without a GPU)."""
import glob
import os
import re

import pytest

from paper_1206_0919_gb300 import shasta as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(shasta_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1206_0919_gb300 import build as B
    B.build()
    return S.lib()


def test_header_declares_functions():
    assert len(declared_functions()) >= 15


@pytest.mark.parametrize("name", declared_functions())
def test_symbol_exported(lib, name):
    assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_binding_covers_header():
    missing = [n for n in declared_functions() if n not in S.SIGNATURES]
    assert not missing, missing


def test_create_without_gpu_fails_cleanly(lib):
    """On a machine without a CUDA device create returns an error code (no
    crash, no CPU fallback)."""
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(S.ShastaError) as ei:
        S.Solver((4, 4, 4))
    assert ei.value.status in (S.ECUDA, S.EINVAL)
    assert lib.shasta_status_string(S.EUNPHYSICAL) == b"SHASTA_EUNPHYSICAL"
    assert lib.shasta_version().startswith(b"shasta-gb300")


def test_bad_scheme_is_rejected_before_any_device_call(lib):
    """Unknown schemes and the split scheme outside FP32 are option errors
    (EINVAL), found before the library looks for a device."""
    for kw in ({"scheme": 7}, {"scheme": "split", "precision": "fp64"},
               {"scheme": "split", "precision": "mixed"},
               {"scheme": "split", "precision": "mixed_fp64"}, {"precision": 4},
               {"scheme": "two_sweeps", "precision": "fp64"},
               {"scheme": "two_sweeps", "precision": "mixed"},
               {"scheme": "two_sweeps", "bc": "frozen"}):
        with pytest.raises(S.ShastaError) as ei:
            S.Solver((4, 4, 4), **kw)
        assert ei.value.status == S.EINVAL, kw


@pytest.mark.parametrize("shape,kw,needle", [
    ((0, 4, 4), {}, "grid sizes"),
    ((4, -1, 4), {}, "grid sizes"),
    ((1 << 16, 1 << 16, 1), {"precision": "fp64"}, "plane too large"),
    ((1, 1 << 16, 1 << 16), {"precision": "fp64"}, "plane too large"),
    ((2048, 2048, 1024), {}, "2^32 cells"),
    ((2048, 2048, 1024), {"precision": "mixed"}, "2^32 cells"),
    ((4, 4, 4), {"lam": 0.0}, "lambda"),
    ((4, 4, 4), {"lam": 0.51}, "lambda"),
    ((4, 4, 4), {"lam": float("nan")}, "lambda"),
    ((4, 4, 4), {"dx": 0.0}, "dx"),
    ((4, 4, 4), {"dx": float("inf")}, "dx"),
    ((4, 4, 4), {"eta": -0.1}, "eta"),
    ((4, 4, 4), {"eta": 0.6}, "eta"),
    ((4, 4, 4), {"delta": 0.5}, "delta"),
    ((4, 4, 4), {"delta": -1e-3}, "delta"),
    ((4, 4, 4), {"bc": 9}, "boundary"),
    ((4, 4, 4), {"eos": 7}, "EoS"),
    ((4, 4, 4), {"eos": "bag", "bag_B": 0.2, "bag_ec": 0.5}, "4B <= e_c"),
    ((4, 4, 4), {"eos": "bag", "bag_B": -0.1}, "4B <= e_c"),
])
def test_bad_grids_and_options_are_rejected_before_any_device_call(lib, shape, kw, needle):
    """Grid sizes (each >= 1; every plane < 2^31 lines; FP32 / MIXED grids
    under 2^32 cells, the kernels' 32-bit cell offsets), the time-step ratio
    (0 < lambda <= 0.5), dx, eta, the clamp margin, the boundary rule and
    the EoS parameters are checked on the host first: EINVAL with the
    reason, on any machine, before the library looks for a device."""
    with pytest.raises(S.ShastaError) as ei:
        S.Solver(shape, **kw)
    assert ei.value.status == S.EINVAL, (shape, kw)
    assert needle in str(ei.value), str(ei.value)


def test_bad_eos_tables_are_rejected(lib):
    """A tabulated EoS must be finite, p >= 0, monotone and causal
    (0 <= dp/de < 1), with at least two values and table_de > 0; MIXED has
    no tabulated path.  All are option errors found before any device call."""
    import numpy as np
    good = np.arange(10) * 0.1 / 3.0
    bad = [dict(table=good[:1], table_de=0.1), dict(table=good, table_de=0.0),
           dict(table=-good - 1.0, table_de=0.1), dict(table=good[::-1].copy(), table_de=0.1),
           dict(table=np.arange(10) * 0.1 * 1.5, table_de=0.1),
           dict(table=np.where(np.arange(10) == 4, np.nan, good), table_de=0.1),
           dict(table=good, table_de=0.1, precision="mixed"),
           dict(table=good, table_de=0.1, precision="mixed_fp64"),
           dict(table=good, table_de=0.1, scheme="no_antiflux"),
           dict(table=good, table_de=0.1, scheme="two_sweeps")]
    for kw in bad:
        with pytest.raises(S.ShastaError) as ei:
            S.Solver((4, 4, 4), eos="table", **kw)
        assert ei.value.status == S.EINVAL, kw


def test_batch_and_server_without_gpu_fail_cleanly(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(S.ShastaError) as ei:
        S.Batch(1 << 20)
    assert ei.value.status == S.ECUDA
    with pytest.raises(S.ShastaError) as ei:
        S.Server(1 << 30)
    assert ei.value.status == S.ECUDA
    # option errors are reported before any device call
    with pytest.raises(S.ShastaError) as ei:
        S.Server(1 << 30, staging_bytes=1 << 31)
    assert ei.value.status == S.EINVAL
    for precision in ("fp64", "mixed_fp64"):  # batches run FP32 or MIXED
        with pytest.raises(S.ShastaError) as ei:
            S.Batch(1 << 20, precision=precision)
        assert ei.value.status == S.EINVAL


def test_null_handles_are_rejected(lib):
    """Every entry point given a NULL handle or NULL output returns an error
    status (or its documented sentinel) without touching the device."""
    import ctypes as C
    null = None
    i64 = (C.c_int64 * 16)()
    dbl = (C.c_double * 16)()
    ints = (C.c_int * 8)()
    ptrs5 = (C.c_void_p * 5)()
    ptrs6 = (C.c_void_p * 6)()
    # single event
    assert lib.shasta_destroy(null) == S.OK
    assert lib.shasta_set_conserved(null, None, None, None, None, None, 0) == S.EINVAL
    assert lib.shasta_set_primitives(null, None, None, None, None, None, 0) == S.EINVAL
    assert lib.shasta_step(null, 1) == S.EINVAL
    assert lib.shasta_sweep(null, 0) == S.EINVAL
    assert lib.shasta_sync(null) == S.EINVAL
    assert lib.shasta_autotune(null) == S.EINVAL
    assert lib.shasta_get_tuning(null, ints) == S.EINVAL
    assert lib.shasta_get_conserved(null, None, None, None, None, None, 0) == S.EINVAL
    assert lib.shasta_get_primitives(null, None, None, None, None, None, None, 0) == S.EINVAL
    assert lib.shasta_totals(null, dbl) == S.EINVAL
    assert lib.shasta_steps_done(null) == -1
    assert lib.shasta_set_step_counter(null, 0) == S.EINVAL
    assert lib.shasta_counters(null, i64) == S.EINVAL
    u64 = (C.c_ulonglong * 3)()
    assert lib.shasta_checked_report(null, u64) == S.EINVAL
    assert lib.shasta_stream(null) is None
    assert lib.shasta_create(None, 1.0, 0.4, None, None, None) == S.EINVAL
    # batches
    assert lib.shasta_batch_destroy(null) == S.OK
    assert lib.shasta_batch_create(None, None) == S.EINVAL
    assert lib.shasta_batch_add(null, None, 1.0, 0.4, None, ptrs5, 0, 0, None) == S.EINVAL
    assert lib.shasta_batch_remove(null, 0) == S.EINVAL
    assert lib.shasta_batch_step(null, 1) == S.EINVAL
    assert lib.shasta_batch_sync(null) == S.EINVAL
    assert lib.shasta_batch_autotune(null) == S.EINVAL
    assert lib.shasta_batch_get_conserved(null, 0, ptrs5, 0) == S.EINVAL
    assert lib.shasta_batch_get_primitives(null, 0, ptrs6, 0) == S.EINVAL
    assert lib.shasta_batch_totals(null, 0, dbl) == S.EINVAL
    assert lib.shasta_batch_steps_done(null, 0) == -1
    assert lib.shasta_batch_counters(null, 0, i64) == S.EINVAL
    assert lib.shasta_batch_checked_report(null, u64) == S.EINVAL
    assert lib.shasta_batch_info(null, i64) == S.EINVAL
    assert lib.shasta_batch_stream(null) is None
    assert lib.shasta_batch_last_error(null) is not None
    # serving
    assert lib.shasta_server_destroy(null) == S.OK
    assert lib.shasta_server_create(None, None) == S.EINVAL
    assert lib.shasta_submit(null, None, None) == S.EINVAL
    assert lib.shasta_poll(null, 1, None) == S.EINVAL
    assert lib.shasta_server_drain(null, 0.0) == S.EINVAL
    assert lib.shasta_server_stats(null, dbl) == S.EINVAL
    assert lib.shasta_server_clock(null) == 0.0
    assert lib.shasta_server_last_error(null) is not None
    assert lib.shasta_last_error(null) is not None
