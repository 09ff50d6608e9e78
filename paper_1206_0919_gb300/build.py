"""Builds the in-tree CUDA library ``libshasta.so`` for sm_103a with nvcc.

Translation units are compiled in parallel.  The FP64 units (the fused FP64
sweep and the auxiliary maps) are built with ``-fmad=false`` and IEEE
division / square root so that they evaluate each expression in plain double
precision in source order; the FP32 / mixed sweeps use flush-to-zero and
fast division / square root; their fused multiply-adds
are explicit (also built with ``-fmad=false``, so that every instantiation of
the streaming step rounds alike).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libshasta.so")
# checked build: the same library with every global access of the sweeps and
# every shared-memory access of the FP32 / MIXED ones bounds-tested (refused
# accesses are counted and skipped; shasta_checked_report reads the record);
# for tests, not for speed
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libshasta_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
          "--expt-relaxed-constexpr", "-I", CSRC, "-I", INCLUDE]
EXACT = ["-fmad=false", "-prec-div=true", "-prec-sqrt=true", "-ftz=false"]
FAST = ["-fmad=false", "-prec-div=false", "-prec-sqrt=false", "-ftz=true"]

UNITS = [
    ("api.cu", EXACT),
    ("aux.cu", EXACT),
    ("noalloc.cu", EXACT),
    ("batch.cu", EXACT),
    ("server.cu", EXACT),
    ("sweep_f64.cu", EXACT),
    ("sweep_f32.cu", FAST),
    ("sweep_f32_noaf.cu", FAST),
    ("sweep_split.cu", FAST),
    ("sweep_fuse2.cu", FAST),
    ("sweep_mixed.cu", FAST),
    ("sweep_mixed64.cu", FAST),
    ("batch_f32.cu", FAST),
    ("batch_mixed.cu", FAST),
    ("alu_peak.cu", FAST),
]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libshasta")
    return p


def _deps_mtime() -> float:
    m = 0.0
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            m = max(m, os.path.getmtime(os.path.join(d, f)))
    return max(m, os.path.getmtime(__file__))


def _compile(unit, flags, verbose, build_dir=BUILD, extra=()):
    src = os.path.join(CSRC, unit)
    obj = os.path.join(build_dir, unit.replace(".cu", ".o"))
    cmd = [nvcc()] + ARCH + COMMON + flags + list(extra) + ["-c", src, "-o", obj]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {unit}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(force: bool = False, verbose: bool = False, jobs: int | None = None,
          checked: bool = False) -> str:
    """Compile every unit and link libshasta.so (checked: libshasta_checked.so,
    built with -DSHASTA_CHECKED); returns its path."""
    lib, build_dir = (LIB_CHECKED, BUILD_CHECKED) if checked else (LIB, BUILD)
    extra = ("-DSHASTA_CHECKED",) if checked else ()
    if not force and not verbose and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    os.makedirs(build_dir, exist_ok=True)
    jobs = jobs or min(len(UNITS), os.cpu_count() or 1)
    objs, logs = [], []
    with cf.ThreadPoolExecutor(jobs) as ex:
        for obj, log in ex.map(lambda u: _compile(u[0], u[1], verbose, build_dir, extra), UNITS):
            objs.append(obj)
            logs.append(log)
    tmp = lib + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    if verbose:
        sys.stderr.write("".join(logs))
    return lib


if __name__ == "__main__":
    build(force=True, verbose="-v" in sys.argv)
    print(LIB)
