"""ctypes front end of the plain FP64 SHASTA oracle (``shasta_oracle.c``).

TEST INFRASTRUCTURE: only the test suite, the package's smoke check and the
benchmark's CPU-baseline leg may import this module.  It shares no code with
the CUDA library of the package and is never reached from its product path.

Arrays are float64 numpy arrays of shape (nz, ny, nx) (x fastest), matching
the C storage ``i + nx*(j + ny*k)``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "shasta_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

BC_REFLECT, BC_PERIODIC, BC_FROZEN = 0, 1, 2
EOS_IDEAL, EOS_BAG, EOS_TABLE = 0, 1, 2

_lock = threading.Lock()


def build(force: bool = False, src: str = SRC, out: str = LIB) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, OpenMP if present)."""
    hdr = os.path.join(HERE, "shasta_oracle.h")
    if not force and os.path.exists(out) and os.path.getmtime(out) >= max(
        os.path.getmtime(src), os.path.getmtime(hdr)
    ):
        return out
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            "-std=c11", "-I", HERE, "-o", out, src, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    return out


class Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("bc", C.c_int), ("eos", C.c_int),
        ("lam", C.c_double), ("eta", C.c_double),
        ("bag_B", C.c_double), ("bag_ec", C.c_double), ("delta", C.c_double),
        ("table", C.POINTER(C.c_double)), ("table_n", C.c_int), ("table_de", C.c_double),
    ]


def params(shape, lam=0.4, eta=0.125, bc=BC_REFLECT, eos=EOS_IDEAL, bag_B=0.1,
           bag_ec=0.5, delta=1e-10, table=None, table_de=0.0) -> Params:
    """shape = (nx, ny, nz).  table: p at e = k * table_de (EOS_TABLE)."""
    nx, ny, nz = shape
    P = Params(nx, ny, nz, bc, eos, lam, eta, bag_B, bag_ec, delta)
    if table is not None:
        t = np.ascontiguousarray(table, dtype=np.float64)
        P._table = t  # keeps the array alive as long as the parameters
        P.table = t.ctypes.data_as(C.POINTER(C.c_double))
        P.table_n = t.size
        P.table_de = table_de
    return P


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """One loaded build of the oracle (the default one, or a test variant)."""

    def __init__(self, path: str):
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        pp = C.POINTER(Params)
        L.or_eos_p.argtypes = [pp, C.c_double]
        L.or_eos_p.restype = C.c_double
        L.or_fixed_point.argtypes = [pp, C.c_double, C.c_double, dp, dp]
        L.or_fixed_point.restype = C.c_int
        L.or_prim2cons.argtypes = [pp, C.c_size_t] + [dp] * 10
        L.or_recover.argtypes = [pp, C.c_size_t] + [dp] * 11
        L.or_line.argtypes = [C.c_int, dp, dp, dp, C.c_double, C.c_double, dp]
        L.or_sweep.argtypes = [pp, C.c_int] + [dp] * 5 + [dp]
        L.or_step.argtypes = [pp] + [dp] * 5 + [dp, C.c_long, C.c_long]
        L.or_step.restype = C.c_int
        L.or_frozen_size.argtypes = [pp]
        L.or_frozen_size.restype = C.c_size_t
        L.or_frozen_capture.argtypes = [pp] + [dp] * 6
        L.or_totals.argtypes = [C.c_size_t] + [dp] * 5 + [dp]
        L.or_axis.argtypes = [C.c_long, C.c_int]
        L.or_axis.restype = C.c_int
        L.or_set_threads.argtypes = [C.c_int]
        L.or_get_threads.restype = C.c_int
        self.L = L
        self.path = path

    def set_threads(self, n: int) -> None:
        self.L.or_set_threads(int(n))

    def get_threads(self) -> int:
        return self.L.or_get_threads()

    def axis(self, step: int, sub: int) -> int:
        return self.L.or_axis(step, sub)

    def eos_p(self, P: Params, e: float) -> float:
        return self.L.or_eos_p(C.byref(P), e)

    def fixed_point(self, P: Params, E: float, M: float):
        """(e, p, iterations) of the tabulated recovery of one cell."""
        e, p = C.c_double(), C.c_double()
        it = self.L.or_fixed_point(C.byref(P), E, M, C.byref(e), C.byref(p))
        return e.value, p.value, it

    def prim2cons(self, P: Params, e, vx, vy, vz, nb):
        e, vx, vy, vz, nb = map(_f64, (e, vx, vy, vz, nb))
        out = [np.empty_like(e) for _ in range(5)]
        self.L.or_prim2cons(C.byref(P), e.size, _p(e), _p(vx), _p(vy), _p(vz), _p(nb),
                            *[_p(o) for o in out])
        return out

    def recover(self, P: Params, U):
        U = [_f64(u) for u in U]
        out = [np.empty_like(U[0]) for _ in range(6)]
        self.L.or_recover(C.byref(P), U[0].size, *[_p(u) for u in U], *[_p(o) for o in out])
        return dict(zip(("e", "vx", "vy", "vz", "n", "p"), out))

    def line(self, u, w, f, tau, eta):
        """One SHASTA pass of one field on a padded line (3 ghosts per side)."""
        u, w = _f64(u), _f64(w)
        f = None if f is None else _f64(f)
        n = u.size - 6
        out = np.empty(n)
        self.L.or_line(n, _p(u), _p(w), _p(f), tau, eta, _p(out))
        return out

    def frozen_capture(self, P: Params, U):
        U = [_f64(u) for u in U]
        fr = np.empty(self.L.or_frozen_size(C.byref(P)))
        self.L.or_frozen_capture(C.byref(P), *[_p(u) for u in U], _p(fr))
        return fr

    def sweep(self, P: Params, U, ax: int, frozen=None):
        """One sweep along axis ax (returns new arrays)."""
        U = [_f64(u).copy() for u in U]
        self.L.or_sweep(C.byref(P), ax, *[_p(u) for u in U], _p(frozen))
        return U

    def step(self, P: Params, U, nsteps: int, step0: int = 0, frozen=None):
        """State after nsteps full split steps (the input is copied)."""
        U = [_f64(u).copy() for u in U]
        if P.bc == BC_FROZEN and frozen is None:
            frozen = self.frozen_capture(P, U)
        rc = self.L.or_step(C.byref(P), *[_p(u) for u in U], _p(frozen), step0, nsteps)
        if rc != 0:
            raise ValueError(f"or_step failed with code {rc}")
        return U

    def totals(self, U):
        U = [_f64(u) for u in U]
        out = np.empty(5)
        self.L.or_totals(U[0].size, *[_p(u) for u in U], _p(out))
        return out


_default = None


def default() -> Oracle:
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
    return _default


def __getattr__(name):
    # module-level shortcuts: oracle.step(...), oracle.recover(...), ...
    if name in ("set_threads", "get_threads", "axis", "eos_p", "fixed_point", "prim2cons",
                "recover", "line",
                "frozen_capture", "sweep", "step", "totals"):
        return getattr(default(), name)
    raise AttributeError(name)
