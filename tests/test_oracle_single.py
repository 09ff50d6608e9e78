"""The oracle's source evaluated in single precision (oracle/shasta_oracle_f32.c),
checked on the CPU before the full-length GPU tests use it as a yardstick.

That build is not a second reference: the tests measure with it how far
single-precision rounding alone carries the plain algorithm from the
double-precision oracle.  For that it must be the same algorithm (it agrees
with the double-precision build to single-precision rounding where the flow
does not amplify it, and meets the same exact facts: the Riemann problem, a
uniform state, conservation), and it must really round to single precision
(its results are float32 and differ from the double-precision ones by
about the single-precision unit roundoff, not by zero).
"""
import numpy as np
import pytest

import pins
from oracle import oracle as OR
from paper_1206_0919_gb300 import workloads as W


@pytest.fixture(scope="module")
def O32():
    O = OR.single()
    O.set_threads(2)
    return O


@pytest.fixture(scope="module")
def O64():
    return OR.default()


def test_single_build_keeps_float32_arrays(O32):
    shape = (6, 5, 4)
    P = OR.params(shape)
    U = O32.prim2cons(P, *W.random_state(shape, seed=3).as_list())
    assert all(u.dtype == np.float32 for u in U)
    U2 = O32.step(P, U, 1)
    assert all(u.dtype == np.float32 for u in U2)


def test_single_build_is_the_same_algorithm(O32, O64):
    """Two steps of a random subluminal state: the single-precision build
    stays within a few hundred units of single-precision roundoff of the
    double-precision oracle (relative L1 per field), and is not bitwise
    equal to it."""
    shape = (23, 17, 11)
    P = OR.params(shape, delta=1e-6)
    U0 = W.rounded_to_single(O64.prim2cons(P, *W.random_state(shape, seed=5, vmax=0.5).as_list()))
    a = O64.step(P, U0, 2)
    b = O32.step(P, U0, 2)
    errs = [float(np.abs(np.float64(y) - x).sum() / np.abs(x).sum()) for x, y in zip(a, b)]
    assert max(errs) < 300 * 2.0 ** -24, errs
    assert max(errs) > 0.1 * 2.0 ** -24, errs  # it really rounds to single precision


def test_single_build_uniform_state_bitwise(O32):
    """A uniform fluid at rest stays bitwise uniform in single precision too
    (Q+- = 1/2 exactly, every difference zero), for every boundary rule."""
    for bc in (OR.BC_REFLECT, OR.BC_PERIODIC, OR.BC_FROZEN):
        for shape in ((7, 5, 3), (1, 9, 2)):
            P = OR.params(shape, bc=bc)
            U = [np.float32(v) * np.ones(shape[::-1], dtype=np.float32)
                 for v in (2.0, 0.0, 0.0, 0.0, 0.7)]
            U2 = O32.step(P, U, 3)
            for a, b in zip(U, U2):
                assert np.array_equal(a, b), (bc, shape)


def test_single_build_riemann(O32):
    """Exact relativistic Riemann problem for p = e/3 at N = 64 and 128:
    the same L1 bound and first-order convergence as the double build."""
    r64 = pins.riemann_error(O32, 64)
    r128 = pins.riemann_error(O32, 128)
    assert r64["err"] < 0.04, r64["err"]
    assert r64["err"] / r128["err"] > 1.7


def test_single_build_conserves_in_a_closed_box(O32):
    """E and R in a reflecting box: conserved to single-precision round-off
    (the sums taken in double)."""
    shape = (19, 14, 11)
    P = OR.params(shape)
    pr = W.hot_spots(shape=shape, seed=17, n_spots=4, sigma=(1.5, 3.0), radial_flow=0.1)
    U = O32.prim2cons(P, *pr.as_list())
    U2 = O32.step(P, U, 5)
    for k in (0, 4):
        t0 = float(np.sum(U[k], dtype=np.float64))
        t1 = float(np.sum(U2[k], dtype=np.float64))
        assert abs(t1 - t0) <= 1e-5 * abs(t0), (k, t0, t1)
