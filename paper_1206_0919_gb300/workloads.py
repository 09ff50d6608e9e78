"""Seeded synthetic initial data for the relativistic SHASTA solver.

This module only draws initial PRIMITIVE fields (rest-frame energy density e,
velocity v, baryon density n) on a Cartesian grid.  It holds none of the
solver's arithmetic, imports neither the CUDA binding nor the oracle, and is
the one module both sides of every parity check take their inputs from.

The paper's own workloads (UrQMD initial states of Au+Au collisions, an
expanding ball, Sec. 4) are not available, so these recipes stand in:

* ``shock_tube``   -- planar Riemann problem along x (classic test problem).
* ``hot_spots``    -- sum of Gaussian hot spots on a small background, the
                      stand-in for a fluctuating collision initial state.
* ``blast``        -- a steep spherical blast (high-gamma stress case), also
                      the expanding-ball shape of Sec. 4 at other radii.

Grids are indexed [k, j, i] = [z, y, x] (x fastest); cell i has its centre at
x = i + 1/2 in units of dx.  Random numbers come from numpy's PCG64
(``numpy.random.default_rng(seed)``).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Prims:
    """Primitive fields, each a float64 array of shape (nz, ny, nx)."""

    e: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    n: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def shape_xyz(self):
        nz, ny, nx = self.e.shape
        return (nx, ny, nz)

    def as_list(self):
        return [self.e, self.vx, self.vy, self.vz, self.n]


def _zeros(nx, ny, nz):
    return np.zeros((nz, ny, nx), dtype=np.float64)


def shock_tube(nx=64, ny=64, nz=64, e_l=1.0, e_r=0.01, n_l=1.0, n_r=0.01, axis=0) -> Prims:
    """Planar Riemann problem: left state for cell index < N/2 along ``axis``."""
    shape = (nz, ny, nx)
    n_ax = (nx, ny, nz)[axis]
    idx = np.arange(n_ax)
    left = idx < n_ax // 2
    bshape = [1, 1, 1]
    bshape[2 - axis] = n_ax
    left = left.reshape(bshape)
    e = np.broadcast_to(np.where(left, e_l, e_r), shape).astype(np.float64).copy()
    n = np.broadcast_to(np.where(left, n_l, n_r), shape).astype(np.float64).copy()
    z = _zeros(nx, ny, nz)
    return Prims(e, z, z.copy(), z.copy(), n, dict(kind="shock_tube", axis=axis))


def _centred_coords(nx, ny, nz):
    x = np.arange(nx) + 0.5
    y = np.arange(ny) + 0.5
    z = np.arange(nz) + 0.5
    return x, y, z


def hot_spots(N=200, seed=2, n_spots=30, sigma=(3.0, 8.0), log10_amp=(-1.0, 1.0),
              background=1e-6, radial_flow=0.0, shape=None) -> Prims:
    """Gaussian hot spots: e = bg + sum_k A_k exp(-|x - c_k|^2 / (2 sigma_k^2)).

    Centres uniform in the central half of the box ([N/4, 3N/4) per axis),
    sigma_k uniform in ``sigma``, log10 A_k uniform in ``log10_amp``;
    n = e^(3/4).  With ``radial_flow`` = a, the initial velocity is radial,
    v = a * r / R_box with R_box = N/2 measured from the box centre.
    """
    nx, ny, nz = shape if shape is not None else (N, N, N)
    rng = np.random.default_rng(seed)
    x, y, z = _centred_coords(nx, ny, nz)
    e = np.full((nz, ny, nx), background, dtype=np.float64)
    lo = np.array([nx, ny, nz]) / 4.0
    hi = 3.0 * np.array([nx, ny, nz]) / 4.0
    for _ in range(n_spots):
        c = rng.uniform(lo, hi)
        s = rng.uniform(*sigma)
        a = 10.0 ** rng.uniform(*log10_amp)
        gx = np.exp(-((x - c[0]) ** 2) / (2 * s * s))
        gy = np.exp(-((y - c[1]) ** 2) / (2 * s * s))
        gz = np.exp(-((z - c[2]) ** 2) / (2 * s * s))
        e += a * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    n = e ** 0.75
    vx, vy, vz = _zeros(nx, ny, nz), _zeros(nx, ny, nz), _zeros(nx, ny, nz)
    if radial_flow:
        Rb = min(nx, ny, nz) / 2.0
        dx = (x - nx / 2.0)[None, None, :]
        dy = (y - ny / 2.0)[None, :, None]
        dz = (z - nz / 2.0)[:, None, None]
        vx = np.broadcast_to(radial_flow * dx / Rb, e.shape).copy()
        vy = np.broadcast_to(radial_flow * dy / Rb, e.shape).copy()
        vz = np.broadcast_to(radial_flow * dz / Rb, e.shape).copy()
    return Prims(e, vx, vy, vz, n, dict(kind="hot_spots", seed=seed, n_spots=n_spots))


def blast(N=512, radius=40.0, e_in=1e3, e_out=0.1, shape=None) -> Prims:
    """Spherical blast: e = e_in inside ``radius`` cells of the centre, else e_out."""
    nx, ny, nz = shape if shape is not None else (N, N, N)
    x, y, z = _centred_coords(nx, ny, nz)
    r2 = ((x - nx / 2.0) ** 2)[None, None, :] + ((y - ny / 2.0) ** 2)[None, :, None] + \
        ((z - nz / 2.0) ** 2)[:, None, None]
    e = np.where(r2 < radius * radius, e_in, e_out).astype(np.float64)
    n = e ** 0.75
    z0 = _zeros(nx, ny, nz)
    return Prims(e, z0, z0.copy(), z0.copy(), n, dict(kind="blast", radius=radius))


def ball(N=200, radius=10.0, e_in=1.0, e_out=1e-6, shape=None) -> Prims:
    """Expanding ball of Sec. 4: a sphere of constant energy density at rest,
    radius 2 fm at dx = 0.2 fm (10 cells), in a near-empty box (e_out, the
    floor of the hot-spot states); n = e^(3/4)."""
    pr = blast(N=N, radius=radius, e_in=e_in, e_out=e_out, shape=shape)
    pr.meta = dict(kind="ball", radius=radius, e_in=e_in, e_out=e_out)
    return pr


def random_state(shape, seed=0, vmax=0.6, e_range=(0.05, 5.0)) -> Prims:
    """Smooth-free random primitives for stress tests: e log-uniform, |v| < vmax."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    e = np.exp(rng.uniform(np.log(e_range[0]), np.log(e_range[1]), (nz, ny, nx)))
    v = rng.normal(size=(3, nz, ny, nx))
    v /= np.sqrt((v * v).sum(0)) + 1e-30
    v *= vmax * rng.uniform(0.0, 1.0, (nz, ny, nx)) ** 0.5
    n = rng.uniform(0.1, 2.0, (nz, ny, nx))
    return Prims(e, v[0].copy(), v[1].copy(), v[2].copy(), n, dict(kind="random", seed=seed))


# ------------------------------------------------------------ event mixes --

BATCH_SIZES = (48, 64, 96, 128, 160)


def batch_events(n_events=64, seed=3, sizes=BATCH_SIZES, radial_flow=0.1):
    """Many independent events of uneven size (hot spots + radial flow).

    Event i draws N uniformly from ``sizes`` and 5-40 hot spots with the
    per-event seed 1000*seed + i.
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_events):
        N = int(rng.choice(sizes))
        k = int(rng.integers(5, 41))
        out.append(dict(N=N, n_spots=k, seed=1000 * seed + i, radial_flow=radial_flow))
    return out


def event_prims(ev: dict) -> Prims:
    return hot_spots(N=ev["N"], seed=ev["seed"], n_spots=ev["n_spots"],
                     radial_flow=ev.get("radial_flow", 0.0))


SERVE_SIZES = (64, 96, 128, 192)
SERVE_PROBS = (0.4, 0.3, 0.2, 0.1)


def serving_stream(n_events=2000, rate_hz=200.0, seed=4, sizes=SERVE_SIZES,
                   probs=SERVE_PROBS, steps=150):
    """Poisson arrival stream: exponential gaps of mean 1/rate; EoS alternates
    between the ideal gas (even index) and the bag model (odd index)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n_events):
        t += rng.exponential(1.0 / rate_hz)
        N = int(rng.choice(sizes, p=probs))
        k = int(rng.integers(5, 41))
        out.append(dict(t_arrival=t, N=N, n_spots=k, seed=1000 * seed + i,
                        eos="ideal" if i % 2 == 0 else "bag", steps=steps))
    return out


# ------------------------------------------------- single-precision inputs ----

def rounded_to_single(fields):
    """Each array rounded to the nearest float32 and widened back to float64:
    the values a single-precision state holds for these inputs."""
    return [np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64) for a in fields]


def ulp_flips(fields, seed):
    """Each array rounded to float32, then every nonzero value moved one
    float32 ulp up or down at random (seeded; zeros stay zero), widened back
    to float64: seeded rounding-size perturbations of a single-precision
    input."""
    rng = np.random.default_rng(seed)
    out = []
    for a in fields:
        f = np.asarray(a, dtype=np.float64).astype(np.float32)
        up = rng.integers(0, 2, size=f.shape).astype(bool)
        g = np.where(up, np.nextafter(f, np.float32(np.inf)), np.nextafter(f, np.float32(-np.inf)))
        out.append(np.where(f == 0, f, g).astype(np.float64))
    return out
