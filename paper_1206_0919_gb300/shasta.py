"""Thin ctypes binding of ``libshasta.so`` (the C ABI in include/shasta.h).

Argument marshalling only: every numerical step runs in the library's CUDA
kernels.  The binding has no fallback: if the library is missing or cannot
be loaded, importing a solver raises.

Functions with the ABI's names (``shasta_create`` ...) are exported as-is;
``Solver`` wraps one context for numpy / torch callers.  Arrays are float64,
shape (nz, ny, nx) (x fastest).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# SHASTA_LIBRARY may name another build of the library, e.g. the checked one
# (build.build(checked=True)); there is no fallback if it is missing
LIB_PATH = os.environ.get("SHASTA_LIBRARY") or os.path.join(HERE, "libshasta.so")

OK, EINVAL, ENOMEM, EAGAIN, EUNPHYSICAL, ETIMEOUT, ECUDA, ENOTFOUND = range(8)
BC_REFLECT, BC_PERIODIC, BC_FROZEN = 0, 1, 2
EOS_IDEAL, EOS_BAG, EOS_TABLE = 0, 1, 2
FP64, FP32, MIXED, MIXED_FP64 = 0, 1, 2, 3
MEM_HOST, MEM_DEVICE = 0, 1

PRECISIONS = {"fp64": FP64, "fp32": FP32, "mixed": MIXED, "mixed_fp64": MIXED_FP64}
BCS = {"reflect": BC_REFLECT, "periodic": BC_PERIODIC, "frozen": BC_FROZEN}


class ShastaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_name(status)}: {msg}")
        self.status = status


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("bc", C.c_int)]


class Eos(C.Structure):
    _fields_ = [("kind", C.c_int), ("B", C.c_double), ("e_c", C.c_double),
                ("table", C.POINTER(C.c_double)), ("table_n", C.c_int), ("table_de", C.c_double)]


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("eta", C.c_double), ("delta", C.c_double),
                ("stream", C.c_void_p), ("device", C.c_int), ("check_input", C.c_int),
                ("autotune", C.c_int), ("use_graphs", C.c_int), ("scheme", C.c_int)]


SCHEMES = {"fused": 0, "no_antiflux": 1, "split": 2, "two_sweeps": 3}


class BatchOpts(C.Structure):
    _fields_ = [("precision", C.c_int), ("eta", C.c_double), ("delta", C.c_double),
                ("stream", C.c_void_p), ("device", C.c_int), ("check_input", C.c_int),
                ("autotune", C.c_int), ("use_graphs", C.c_int), ("max_events", C.c_int),
                ("capacity_cells", C.c_int64)]


STATE_CONSERVED, STATE_PRIMITIVE = 0, 1


class ServerOpts(C.Structure):
    _fields_ = [("precision", C.c_int), ("eta", C.c_double), ("delta", C.c_double),
                ("device", C.c_int), ("hbm_budget_bytes", C.c_int64),
                ("staging_bytes", C.c_int64), ("max_resident", C.c_int),
                ("max_queue", C.c_int), ("steps_per_round", C.c_int)]


class Event(C.Structure):
    _fields_ = [("grid", Grid), ("dx", C.c_double), ("lam", C.c_double), ("eos", Eos),
                ("fields", C.c_void_p * 5), ("kind", C.c_int), ("nsteps", C.c_int),
                ("out_prims", C.c_void_p * 6), ("out_cons", C.c_void_p * 5)]


class Result(C.Structure):
    _fields_ = [("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("steps", C.c_int64), ("clamp_count", C.c_int64)]

_lock = threading.Lock()
_lib = None

_dp = C.POINTER(C.c_double)
_vp = C.c_void_p

# name -> (restype, argtypes); the single source of the Python-side ABI.
SIGNATURES = {
    "shasta_default_opts": (None, [C.POINTER(Opts)]),
    "shasta_create": (C.c_int, [C.POINTER(Grid), C.c_double, C.c_double, C.POINTER(Eos),
                                C.POINTER(Opts), C.POINTER(_vp)]),
    "shasta_destroy": (C.c_int, [_vp]),
    "shasta_set_conserved": (C.c_int, [_vp] + [_vp] * 5 + [C.c_int]),
    "shasta_set_primitives": (C.c_int, [_vp] + [_vp] * 5 + [C.c_int]),
    "shasta_step": (C.c_int, [_vp, C.c_int]),
    "shasta_sweep": (C.c_int, [_vp, C.c_int]),
    "shasta_sync": (C.c_int, [_vp]),
    "shasta_autotune": (C.c_int, [_vp]),
    "shasta_get_tuning": (C.c_int, [_vp, C.POINTER(C.c_int)]),
    "shasta_get_conserved": (C.c_int, [_vp] + [_vp] * 5 + [C.c_int]),
    "shasta_get_primitives": (C.c_int, [_vp] + [_vp] * 6 + [C.c_int]),
    "shasta_totals": (C.c_int, [_vp, _dp]),
    "shasta_totals_noalloc": (C.c_int, [_vp] * 5 + [C.c_size_t, _vp, _vp]),
    "shasta_alu_peak": (C.c_int, [C.c_int, C.c_int, _vp, C.POINTER(C.c_double),
                                  C.POINTER(C.c_double)]),
    "shasta_steps_done": (C.c_int64, [_vp]),
    "shasta_set_step_counter": (C.c_int, [_vp, C.c_int64]),
    "shasta_counters": (C.c_int, [_vp, C.POINTER(C.c_int64)]),
    "shasta_checked_report": (C.c_int, [_vp, C.POINTER(C.c_ulonglong)]),
    "shasta_stream": (_vp, [_vp]),
    "shasta_last_error": (C.c_char_p, [_vp]),
    "shasta_status_string": (C.c_char_p, [C.c_int]),
    "shasta_version": (C.c_char_p, []),
    # include/shasta_batch.h
    "shasta_batch_default_opts": (None, [C.POINTER(BatchOpts)]),
    "shasta_batch_create": (C.c_int, [C.POINTER(BatchOpts), C.POINTER(_vp)]),
    "shasta_batch_destroy": (C.c_int, [_vp]),
    "shasta_batch_add": (C.c_int, [_vp, C.POINTER(Grid), C.c_double, C.c_double, C.POINTER(Eos),
                                   C.POINTER(_vp), C.c_int, C.c_int, C.POINTER(C.c_int)]),
    "shasta_batch_remove": (C.c_int, [_vp, C.c_int]),
    "shasta_batch_step": (C.c_int, [_vp, C.c_int]),
    "shasta_batch_sync": (C.c_int, [_vp]),
    "shasta_batch_autotune": (C.c_int, [_vp]),
    "shasta_batch_get_conserved": (C.c_int, [_vp, C.c_int, C.POINTER(_vp), C.c_int]),
    "shasta_batch_get_primitives": (C.c_int, [_vp, C.c_int, C.POINTER(_vp), C.c_int]),
    "shasta_batch_totals": (C.c_int, [_vp, C.c_int, _dp]),
    "shasta_batch_steps_done": (C.c_int64, [_vp, C.c_int]),
    "shasta_batch_set_step_counter": (C.c_int, [_vp, C.c_int, C.c_int64]),
    "shasta_batch_counters": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_int64)]),
    "shasta_batch_checked_report": (C.c_int, [_vp, C.POINTER(C.c_ulonglong)]),
    "shasta_batch_info": (C.c_int, [_vp, C.POINTER(C.c_int64)]),
    "shasta_batch_stream": (_vp, [_vp]),
    "shasta_batch_last_error": (C.c_char_p, [_vp]),
    # include/shasta_serve.h
    "shasta_server_default_opts": (None, [C.POINTER(ServerOpts)]),
    "shasta_server_create": (C.c_int, [C.POINTER(ServerOpts), C.POINTER(_vp)]),
    "shasta_server_destroy": (C.c_int, [_vp]),
    "shasta_submit": (C.c_int, [_vp, C.POINTER(Event), C.POINTER(C.c_uint64)]),
    "shasta_poll": (C.c_int, [_vp, C.c_uint64, C.POINTER(Result)]),
    "shasta_server_drain": (C.c_int, [_vp, C.c_double]),
    "shasta_server_stats": (C.c_int, [_vp, C.POINTER(C.c_double)]),
    "shasta_server_clock": (C.c_double, [_vp]),
    "shasta_server_last_error": (C.c_char_p, [_vp]),
}


def lib():
    """The loaded library; raises if it is not built (no fallback exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(
                    f"{LIB_PATH} is missing: build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def status_name(s: int) -> str:
    try:
        return lib().shasta_status_string(s).decode()
    except Exception:  # library not loadable
        return f"status {s}"


def _check(status, ctx=None):
    if status != OK:
        msg = lib().shasta_last_error(ctx).decode()
        raise ShastaError(status, msg)


def __getattr__(name):
    if name in SIGNATURES:
        return getattr(lib(), name)
    raise AttributeError(name)


# ------------------------------------------------------------- helpers ----

def _host_ptr(a):
    assert isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptrs(arrays):
    """(pointers, mem, keepalive) for a list of numpy or torch float64 arrays."""
    if all(a is None for a in arrays):
        return [None] * len(arrays), MEM_HOST, []
    first = next(a for a in arrays if a is not None)
    if _is_torch(first):
        import torch
        if first.is_cuda:
            for a in arrays:
                if a is not None:
                    assert a.dtype == torch.float64 and a.is_contiguous() and a.is_cuda
            return [None if a is None else a.data_ptr() for a in arrays], MEM_DEVICE, arrays
        keep = [None if a is None else a.contiguous().numpy() for a in arrays]
        return [None if a is None else _host_ptr(a) for a in keep], MEM_HOST, keep
    keep = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in arrays]
    return [None if a is None else _host_ptr(a) for a in keep], MEM_HOST, keep


TOTALS_NOALLOC_MAX_CELLS = 1 << 26


def totals_noalloc(E, Mx, My, Mz, R, out, stream=None):
    """Sums of five caller-owned device fields into the caller's device
    tensor ``out`` (5 float64) without any device allocation, for callers
    that cannot allocate (see ``shasta_totals_noalloc``).  The fields are
    contiguous float64 CUDA tensors of one size on the current device;
    ``stream`` is a torch.cuda.Stream or raw cudaStream_t (default: torch's
    current stream).  Enqueues and returns without waiting."""
    import torch
    fields = (E, Mx, My, Mz, R)
    n = E.numel()
    for a in fields + (out,):
        if not (a.is_cuda and a.dtype == torch.float64 and a.is_contiguous()):
            raise ValueError("fields and out must be contiguous float64 CUDA tensors")
    if any(a.numel() != n for a in fields) or out.numel() < 5:
        raise ValueError("fields must have one size and out at least 5 elements")
    if n > TOTALS_NOALLOC_MAX_CELLS:
        raise ShastaError(EINVAL, f"{n} cells exceed the fixed scratch limit of "
                                  f"{TOTALS_NOALLOC_MAX_CELLS} cells of shasta_totals_noalloc")
    if stream is None:
        stream = torch.cuda.current_stream(E.device).cuda_stream
    elif not isinstance(stream, int):
        stream = stream.cuda_stream
    with torch.cuda.device(E.device):  # the call works on the current device
        st = lib().shasta_totals_noalloc(*[a.data_ptr() for a in fields], n, out.data_ptr(),
                                         stream)
    if st != OK:
        raise ShastaError(st, "shasta_totals_noalloc failed"
                          + (" (more cells than its fixed scratch holds, or a NULL pointer)"
                             if st == EINVAL else ""))


def alu_peak(kind="fp32", device=0, stream=None):
    """Measured CUDA-core rate of `device` (shasta_alu_peak): (floating-point
    operations per second, seconds per timed launch); kind "fp32" or "fp64"."""
    flops, secs = C.c_double(), C.c_double()
    _check(lib().shasta_alu_peak({"fp32": 0, "fp64": 1}[kind], device, stream, C.byref(flops),
                                 C.byref(secs)))
    return flops.value, secs.value


class Solver:
    """One solver context (one event) of the C ABI."""

    def __init__(self, shape, lam=0.4, dx=1.0, precision="fp32", bc="reflect", eos="ideal",
                 bag_B=0.1, bag_ec=0.5, eta=0.125, delta=0.0, stream=None, device=0,
                 check_input=True, autotune=True, use_graphs=True, scheme="fused", table=None,
                 table_de=0.0):
        L = lib()
        nx, ny, nz = shape
        self.shape = (nx, ny, nz)
        g = Grid(nx, ny, nz, BCS[bc] if isinstance(bc, str) else bc)
        kind = {"ideal": EOS_IDEAL, "bag": EOS_BAG, "table": EOS_TABLE}[eos] \
            if isinstance(eos, str) else eos
        e = Eos(kind, bag_B, bag_ec)
        if table is not None:
            t = np.ascontiguousarray(table, dtype=np.float64)  # copied by shasta_create
            e.table = t.ctypes.data_as(C.POINTER(C.c_double))
            e.table_n = t.size
            e.table_de = table_de
        o = Opts()
        L.shasta_default_opts(C.byref(o))
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else precision
        o.eta = eta
        o.delta = delta
        o.stream = stream
        o.device = device
        o.check_input = 1 if check_input else 0
        o.autotune = 1 if autotune else 0
        o.use_graphs = 1 if use_graphs else 0
        o.scheme = SCHEMES[scheme] if isinstance(scheme, str) else scheme
        h = _vp()
        _check(L.shasta_create(C.byref(g), dx, lam, C.byref(e), C.byref(o), C.byref(h)))
        self._h = h
        self.precision = precision

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().shasta_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def grid_shape(self):
        nx, ny, nz = self.shape
        return (nz, ny, nx)

    def set_conserved(self, U):
        p, mem, keep = _ptrs(list(U))
        _check(lib().shasta_set_conserved(self._h, *p, mem), self._h)

    def set_primitives(self, e, vx, vy, vz, n):
        p, mem, keep = _ptrs([e, vx, vy, vz, n])
        _check(lib().shasta_set_primitives(self._h, *p, mem), self._h)

    def step(self, nsteps=1):
        _check(lib().shasta_step(self._h, int(nsteps)), self._h)

    def sweep(self, axis):
        _check(lib().shasta_sweep(self._h, int(axis)), self._h)

    def autotune(self):
        _check(lib().shasta_autotune(self._h), self._h)

    def tuning(self):
        out = (C.c_int * 6)()
        _check(lib().shasta_get_tuning(self._h, out), self._h)
        return [(out[2 * a], out[2 * a + 1]) for a in range(3)]

    def sync(self):
        _check(lib().shasta_sync(self._h), self._h)

    def get_conserved(self, out=None):
        if out is None:
            out = [np.empty(self.grid_shape) for _ in range(5)]
        p, mem, keep = _ptrs(list(out))
        _check(lib().shasta_get_conserved(self._h, *p, mem), self._h)
        return out

    def get_primitives(self, out=None):
        if out is None:
            out = [np.empty(self.grid_shape) for _ in range(6)]
        p, mem, keep = _ptrs(list(out))
        _check(lib().shasta_get_primitives(self._h, *p, mem), self._h)
        return dict(zip(("e", "vx", "vy", "vz", "n", "p"), out))

    def totals(self):
        out = (C.c_double * 5)()
        _check(lib().shasta_totals(self._h, out), self._h)
        return np.array(out[:])

    @property
    def steps_done(self):
        return int(lib().shasta_steps_done(self._h))

    def set_step_counter(self, n):
        _check(lib().shasta_set_step_counter(self._h, int(n)), self._h)

    def counters(self):
        out = (C.c_int64 * 1)()
        _check(lib().shasta_counters(self._h, out), self._h)
        return int(out[0])

    def checked_report(self):
        """Checked builds: (refused accesses, first code, first index); clears."""
        out = (C.c_ulonglong * 3)()
        _check(lib().shasta_checked_report(self._h, out), self._h)
        return tuple(int(x) for x in out)

    @property
    def stream(self):
        return lib().shasta_stream(self._h)


def _bcheck(status, b=None):
    if status != OK:
        raise ShastaError(status, lib().shasta_batch_last_error(b).decode())


def _eos_struct(eos, bag_B, bag_ec):
    kind = {"ideal": EOS_IDEAL, "bag": EOS_BAG}[eos] if isinstance(eos, str) else eos
    return Eos(kind, bag_B, bag_ec)


class Batch:
    """Many events in one device pool, advanced together (include/shasta_batch.h)."""

    def __init__(self, capacity_cells, precision="fp32", max_events=1024, eta=0.125, delta=0.0,
                 stream=None, device=0, check_input=True, autotune=True, use_graphs=True):
        L = lib()
        o = BatchOpts()
        L.shasta_batch_default_opts(C.byref(o))
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else precision
        o.eta = eta
        o.delta = delta
        o.stream = stream
        o.device = device
        o.check_input = 1 if check_input else 0
        o.autotune = 1 if autotune else 0
        o.use_graphs = 1 if use_graphs else 0
        o.max_events = max_events
        o.capacity_cells = int(capacity_cells)
        h = _vp()
        _bcheck(L.shasta_batch_create(C.byref(o), C.byref(h)))
        self._h = h
        self.shapes = {}

    def close(self):
        if getattr(self, "_h", None):
            lib().shasta_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _add(self, shape, arrays, kind, lam, dx, bc, eos, bag_B, bag_ec):
        nx, ny, nz = shape
        g = Grid(nx, ny, nz, BCS[bc] if isinstance(bc, str) else bc)
        e = _eos_struct(eos, bag_B, bag_ec)
        p, mem, keep = _ptrs(list(arrays))
        arr = (_vp * 5)(*p)
        out = C.c_int(-1)
        _bcheck(lib().shasta_batch_add(self._h, C.byref(g), dx, lam, C.byref(e), arr, kind, mem,
                                       C.byref(out)), self._h)
        self.shapes[out.value] = (nz, ny, nx)
        return out.value

    def add_conserved(self, shape, U, lam=0.4, dx=1.0, bc="reflect", eos="ideal", bag_B=0.1,
                      bag_ec=0.5):
        return self._add(shape, U, STATE_CONSERVED, lam, dx, bc, eos, bag_B, bag_ec)

    def add_primitives(self, shape, prims, lam=0.4, dx=1.0, bc="reflect", eos="ideal",
                       bag_B=0.1, bag_ec=0.5):
        return self._add(shape, prims, STATE_PRIMITIVE, lam, dx, bc, eos, bag_B, bag_ec)

    def remove(self, eid):
        _bcheck(lib().shasta_batch_remove(self._h, eid), self._h)
        self.shapes.pop(eid, None)

    def step(self, nsteps=1):
        _bcheck(lib().shasta_batch_step(self._h, int(nsteps)), self._h)

    def sync(self):
        _bcheck(lib().shasta_batch_sync(self._h), self._h)

    def autotune(self):
        _bcheck(lib().shasta_batch_autotune(self._h), self._h)

    def get_conserved(self, eid, out=None):
        if out is None:
            shape = self.shapes.get(eid)  # unknown ids reach the library (ENOTFOUND)
            out = [None if shape is None else np.empty(shape) for _ in range(5)]
        p, mem, keep = _ptrs(list(out))
        _bcheck(lib().shasta_batch_get_conserved(self._h, eid, (_vp * 5)(*p), mem), self._h)
        return out

    def get_primitives(self, eid, out=None):
        if out is None:
            shape = self.shapes.get(eid)  # unknown ids reach the library (ENOTFOUND)
            out = [None if shape is None else np.empty(shape) for _ in range(6)]
        p, mem, keep = _ptrs(list(out))
        _bcheck(lib().shasta_batch_get_primitives(self._h, eid, (_vp * 6)(*p), mem), self._h)
        return dict(zip(("e", "vx", "vy", "vz", "n", "p"), out))

    def totals(self, eid):
        out = (C.c_double * 5)()
        _bcheck(lib().shasta_batch_totals(self._h, eid, out), self._h)
        return np.array(out[:])

    def steps_done(self, eid):
        return int(lib().shasta_batch_steps_done(self._h, eid))

    def set_step_counter(self, eid, steps):
        _bcheck(lib().shasta_batch_set_step_counter(self._h, eid, int(steps)), self._h)

    def counters(self, eid):
        out = (C.c_int64 * 1)()
        _bcheck(lib().shasta_batch_counters(self._h, eid, out), self._h)
        return int(out[0])

    def checked_report(self):
        """Checked builds: (refused accesses, first code, first index); clears."""
        out = (C.c_ulonglong * 3)()
        _bcheck(lib().shasta_batch_checked_report(self._h, out), self._h)
        return tuple(int(x) for x in out)

    def info(self):
        out = (C.c_int64 * 7)()
        _bcheck(lib().shasta_batch_info(self._h, out), self._h)
        keys = ("events", "cells_used", "capacity", "largest_free", "launches_per_step",
                "items_per_step", "launches")
        return dict(zip(keys, (int(v) for v in out)))

    @property
    def stream(self):
        return lib().shasta_batch_stream(self._h)


def _scheck(status, srv=None):
    if status != OK:
        raise ShastaError(status, lib().shasta_server_last_error(srv).decode())


class Server:
    """Serving loop (include/shasta_serve.h): submit events as they arrive,
    poll for their results."""

    def __init__(self, hbm_budget_bytes, precision="fp32", staging_bytes=0, max_resident=256,
                 max_queue=4096, steps_per_round=6, eta=0.125, delta=0.0, device=0):
        L = lib()
        o = ServerOpts()
        L.shasta_server_default_opts(C.byref(o))
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else precision
        o.eta = eta
        o.delta = delta
        o.device = device
        o.hbm_budget_bytes = int(hbm_budget_bytes)
        o.staging_bytes = int(staging_bytes)
        o.max_resident = max_resident
        o.max_queue = max_queue
        o.steps_per_round = steps_per_round
        h = _vp()
        _scheck(L.shasta_server_create(C.byref(o), C.byref(h)))
        self._h = h
        self._pending = {}

    def close(self):
        if getattr(self, "_h", None):
            lib().shasta_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, shape, arrays, nsteps, kind="primitive", lam=0.4, dx=1.0, bc="reflect",
               eos="ideal", bag_B=0.1, bag_ec=0.5, prims_out=True, cons_out=False):
        """Queues one event (five host arrays, copied); returns its ticket.
        Raises ShastaError with status EAGAIN when the queue is full."""
        nx, ny, nz = shape
        ev = Event()
        ev.grid = Grid(nx, ny, nz, BCS[bc] if isinstance(bc, str) else bc)
        ev.dx = dx
        ev.lam = lam
        ev.eos = _eos_struct(eos, bag_B, bag_ec)
        keep = [np.ascontiguousarray(a, dtype=np.float64) for a in arrays]
        for k in range(5):
            assert keep[k].size == nx * ny * nz
            ev.fields[k] = keep[k].ctypes.data
        ev.kind = STATE_PRIMITIVE if kind == "primitive" else STATE_CONSERVED
        ev.nsteps = int(nsteps)
        outs = {"prims": [np.empty((nz, ny, nx)) for _ in range(6)] if prims_out else None,
                "cons": [np.empty((nz, ny, nx)) for _ in range(5)] if cons_out else None}
        if outs["prims"]:
            for k in range(6):
                ev.out_prims[k] = outs["prims"][k].ctypes.data
        if outs["cons"]:
            for k in range(5):
                ev.out_cons[k] = outs["cons"][k].ctypes.data
        t = C.c_uint64(0)
        _scheck(lib().shasta_submit(self._h, C.byref(ev), C.byref(t)), self._h)
        self._pending[t.value] = outs
        return t.value

    def poll(self, ticket):
        """None while pending; a dict of timings and result arrays once the
        event has finished; raises ShastaError if it failed."""
        r = Result()
        st = lib().shasta_poll(self._h, ticket, C.byref(r))
        if st == EAGAIN:
            return None
        outs = self._pending.pop(ticket, None)
        if st != OK:
            raise ShastaError(st, lib().shasta_server_last_error(self._h).decode())
        d = {"t_submit": r.t_submit, "t_admit": r.t_admit, "t_done": r.t_done,
             "steps": int(r.steps), "clamp_count": int(r.clamp_count)}
        if outs and outs["prims"]:
            d["prims"] = dict(zip(("e", "vx", "vy", "vz", "n", "p"), outs["prims"]))
        if outs and outs["cons"]:
            d["cons"] = outs["cons"]
        return d

    def drain(self, timeout_s=60.0):
        _scheck(lib().shasta_server_drain(self._h, float(timeout_s)), self._h)

    def stats(self):
        out = (C.c_double * 16)()
        _scheck(lib().shasta_server_stats(self._h, out), self._h)
        keys = ("submitted", "finished", "failed", "queued", "in_flight", "peak_resident",
                "batch_steps", "pool_cells", "sweep_launches", "t_copy_in", "t_admit",
                "t_harvest", "t_step_enqueue", "t_copy_out", "t_wait_steps", "t_idle")
        return dict(zip(keys, out[:]))

    def clock(self):
        return float(lib().shasta_server_clock(self._h))
