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
    with pytest.raises(S.ShastaError) as ei:
        S.Batch(1 << 20, precision="fp64")
    assert ei.value.status == S.EINVAL
