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
# the same source evaluated in single precision (see shasta_oracle_f32.c)
SRC32 = os.path.join(HERE, "shasta_oracle_f32.c")
LIB32 = os.path.join(HERE, "liboracle_f32.so")

BC_REFLECT, BC_PERIODIC, BC_FROZEN = 0, 1, 2
EOS_IDEAL, EOS_BAG, EOS_TABLE = 0, 1, 2

_lock = threading.Lock()


def build(force: bool = False, src: str = SRC, out: str = LIB, extra=()) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, OpenMP if present)."""
    deps = [src, os.path.join(os.path.dirname(src), "shasta_oracle.h"), SRC]
    if not force and os.path.exists(out) and os.path.getmtime(out) >= max(
        os.path.getmtime(d) for d in deps if os.path.exists(d)
    ):
        return out
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", *extra, "-fPIC", "-shared",
            "-std=c11", "-I", os.path.dirname(src), "-o", out, src, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    return out


def build_single(force: bool = False) -> str:
    """Compile the single-precision build of the oracle (shasta_oracle_f32.c)."""
    return build(force, SRC32, LIB32, extra=("-fsingle-precision-constant",))


def _params_fields(real):
    return [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("bc", C.c_int), ("eos", C.c_int),
        ("lam", real), ("eta", real),
        ("bag_B", real), ("bag_ec", real), ("delta", real),
        ("table", C.POINTER(real)), ("table_n", C.c_int), ("table_de", real),
    ]


class Params(C.Structure):
    _fields_ = _params_fields(C.c_double)


class Params32(C.Structure):
    """or_params of the single-precision build (every double a float)."""
    _fields_ = _params_fields(C.c_float)


def _single_params(P: Params) -> Params32:
    Q = Params32(P.nx, P.ny, P.nz, P.bc, P.eos, P.lam, P.eta, P.bag_B, P.bag_ec, P.delta)
    if getattr(P, "_table", None) is not None:
        t = np.ascontiguousarray(P._table, dtype=np.float32)
        Q._table = t
        Q.table = t.ctypes.data_as(C.POINTER(C.c_float))
        Q.table_n = t.size
        Q.table_de = P.table_de
    return Q


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


class Oracle:
    """One loaded build of the oracle (the default one, a test variant, or
    the single-precision build with single=True: its arrays are float32)."""

    def __init__(self, path: str, single: bool = False):
        L = C.CDLL(path)
        real = C.c_float if single else C.c_double
        self.single = single
        self.dtype = np.float32 if single else np.float64
        self._real = real
        dp = C.POINTER(real)
        pp = C.POINTER(Params32 if single else Params)
        L.or_eos_p.argtypes = [pp, real]
        L.or_eos_p.restype = real
        L.or_fixed_point.argtypes = [pp, real, real, dp, dp]
        L.or_fixed_point.restype = C.c_int
        L.or_prim2cons.argtypes = [pp, C.c_size_t] + [dp] * 10
        L.or_recover.argtypes = [pp, C.c_size_t] + [dp] * 11
        L.or_line.argtypes = [C.c_int, dp, dp, dp, real, real, dp]
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

    def _P(self, P):
        return C.byref(_single_params(P) if self.single else P)

    def _arr(self, a):
        """The build's own floating type (float64, or float32 when single)."""
        return np.ascontiguousarray(a, dtype=self.dtype)

    def _p(self, a):
        if a is None:
            return None
        assert a.dtype == self.dtype and a.flags.c_contiguous
        return a.ctypes.data_as(C.POINTER(self._real))

    def set_threads(self, n: int) -> None:
        self.L.or_set_threads(int(n))

    def get_threads(self) -> int:
        return self.L.or_get_threads()

    def axis(self, step: int, sub: int) -> int:
        return self.L.or_axis(step, sub)

    def eos_p(self, P: Params, e: float) -> float:
        return self.L.or_eos_p(self._P(P), e)

    def fixed_point(self, P: Params, E: float, M: float):
        """(e, p, iterations) of the tabulated recovery of one cell."""
        e, p = self._real(), self._real()
        it = self.L.or_fixed_point(self._P(P), E, M, C.byref(e), C.byref(p))
        return e.value, p.value, it

    def prim2cons(self, P: Params, e, vx, vy, vz, nb):
        e, vx, vy, vz, nb = map(self._arr, (e, vx, vy, vz, nb))
        out = [np.empty_like(e) for _ in range(5)]
        self.L.or_prim2cons(self._P(P), e.size, *[self._p(a) for a in (e, vx, vy, vz, nb)],
                            *[self._p(o) for o in out])
        return out

    def recover(self, P: Params, U):
        U = [self._arr(u) for u in U]
        out = [np.empty_like(U[0]) for _ in range(6)]
        self.L.or_recover(self._P(P), U[0].size, *[self._p(u) for u in U],
                          *[self._p(o) for o in out])
        return dict(zip(("e", "vx", "vy", "vz", "n", "p"), out))

    def line(self, u, w, f, tau, eta):
        """One SHASTA pass of one field on a padded line (3 ghosts per side)."""
        u, w = self._arr(u), self._arr(w)
        f = None if f is None else self._arr(f)
        n = u.size - 6
        out = np.empty(n, dtype=self.dtype)
        self.L.or_line(n, self._p(u), self._p(w), self._p(f), tau, eta, self._p(out))
        return out

    def frozen_capture(self, P: Params, U):
        U = [self._arr(u) for u in U]
        fr = np.empty(self.L.or_frozen_size(self._P(P)), dtype=self.dtype)
        self.L.or_frozen_capture(self._P(P), *[self._p(u) for u in U], self._p(fr))
        return fr

    def sweep(self, P: Params, U, ax: int, frozen=None):
        """One sweep along axis ax (returns new arrays)."""
        U = [self._arr(u).copy() for u in U]
        self.L.or_sweep(self._P(P), ax, *[self._p(u) for u in U], self._p(frozen))
        return U

    def step(self, P: Params, U, nsteps: int, step0: int = 0, frozen=None):
        """State after nsteps full split steps (the input is copied)."""
        U = [self._arr(u).copy() for u in U]
        if P.bc == BC_FROZEN and frozen is None:
            frozen = self.frozen_capture(P, U)
        rc = self.L.or_step(self._P(P), *[self._p(u) for u in U], self._p(frozen), step0, nsteps)
        if rc != 0:
            raise ValueError(f"or_step failed with code {rc}")
        return U

    def totals(self, U):
        U = [self._arr(u) for u in U]
        out = np.empty(5, dtype=self.dtype)
        self.L.or_totals(U[0].size, *[self._p(u) for u in U], self._p(out))
        return out


_default = None
_single = None


def default() -> Oracle:
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
    return _default


def single() -> Oracle:
    """The oracle's algorithm evaluated in single precision (float32 arrays
    in and out); a yardstick of single-precision rounding, not a reference."""
    global _single
    with _lock:
        if _single is None:
            _single = Oracle(build_single(), single=True)
    return _single


def __getattr__(name):
    # module-level shortcuts: oracle.step(...), oracle.recover(...), ...
    if name in ("set_threads", "get_threads", "axis", "eos_p", "fixed_point", "prim2cons",
                "recover", "line",
                "frozen_capture", "sweep", "step", "totals"):
        return getattr(default(), name)
    raise AttributeError(name)
