"""The sweep schemes of include/shasta.h and the expanding ball, against the
oracle (GPU).

SPLIT is the alternative decomposition of Sec. 3.1 (separate recovery,
transport and antidiffusion kernels, intermediates in device memory), FP32:
the same method as the fused sweep, checked against the oracle with the
FP32 bar and against the fused FP32 sweep.

NO_ANTIFLUX leaves antidiffusion and flux limiter out of every pass: A = 0
in the update of Sec. 3 (Eq. shasta-n), which is what the oracle computes
with eta = 0 (A^ph = 0, so the limited flux is 0).  FP32 runs dedicated
kernels without that stage; FP64 and MIXED run the fused kernels with
eta = 0.

The expanding ball of Sec. 4 (radius 2 fm at dx = 0.2 fm, i.e. 10 cells, of
constant energy density) runs with both schemes: FP64 equals the oracle,
FP32 meets the 1e-4 bar in e.
"""
import numpy as np
import pytest

from gpu_util import max_rel_err, oracle, rel_l1, require_gpu
from oracle import oracle as OR
from paper_1206_0919_gb300 import shasta as S
from paper_1206_0919_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BC_NAMES = {OR.BC_REFLECT: "reflect", OR.BC_PERIODIC: "periodic", OR.BC_FROZEN: "frozen"}
EOS_NAMES = {OR.EOS_IDEAL: "ideal", OR.EOS_BAG: "bag"}


def run(shape, U0, nsteps, precision, scheme, bc=OR.BC_REFLECT, eos=OR.EOS_IDEAL, eta=0.125,
        delta=0.0):
    with S.Solver(shape, precision=precision, bc=BC_NAMES[bc], eos=EOS_NAMES[eos], eta=eta,
                  delta=delta, scheme=scheme) as s:
        s.set_conserved(U0)
        s.step(nsteps)
        return s.get_conserved(), s.get_primitives(), s.counters()


def state(shape, bc, eos, seed):
    pr = W.random_state(shape, seed=seed, vmax=0.6,
                        e_range=(0.3, 3.0) if eos == OR.EOS_BAG else (0.05, 5.0))
    P = OR.params(shape, bc=bc, eos=eos)
    return P, oracle().prim2cons(P, *pr.as_list())


@pytest.mark.parametrize("bc", [OR.BC_REFLECT, OR.BC_PERIODIC, OR.BC_FROZEN])
@pytest.mark.parametrize("eos", [OR.EOS_IDEAL, OR.EOS_BAG])
@pytest.mark.parametrize("shape", [(37, 21, 13), (40, 3, 2), (5, 33, 9)])
def test_no_antiflux_fp32_is_fused_with_eta_zero(shape, bc, eos):
    """The FP32 kernels without the stage give the fused kernels' result at
    eta = 0 (A = 0 exactly there), value for value; 7 steps cover the axis
    table."""
    require_gpu()
    _, U0 = state(shape, bc, eos, seed=3 * sum(shape) + bc + 7 * eos)
    a, _, _ = run(shape, U0, 7, "fp32", "no_antiflux", bc=bc, eos=eos)
    b, _, _ = run(shape, U0, 7, "fp32", "fused", bc=bc, eos=eos, eta=0.0)
    for f in range(5):
        assert np.array_equal(a[f], b[f]), f


@pytest.mark.parametrize("bc", [OR.BC_REFLECT, OR.BC_PERIODIC])
@pytest.mark.parametrize("eos", [OR.EOS_IDEAL, OR.EOS_BAG])
def test_no_antiflux_against_oracle(bc, eos):
    """FP64: the oracle with eta = 0 to 1e-12 per cell.  FP32 and MIXED:
    1e-4 relative L1 in e, totals to 1e-5."""
    require_gpu()
    shape = (29, 17, 23)
    P, U0 = state(shape, bc, eos, seed=11 + bc + 5 * eos)
    P0 = OR.params(shape, bc=bc, eos=eos, eta=0.0)
    O = oracle()
    ref = O.step(P0, U0, 9)
    rp = O.recover(P0, ref)
    got, _, _ = run(shape, U0, 9, "fp64", "no_antiflux", bc=bc, eos=eos)
    assert max(max_rel_err(g, r) for g, r in zip(got, ref)) <= 1e-12
    for prec in ("fp32", "mixed"):
        got, prim, _ = run(shape, U0, 9, prec, "no_antiflux", bc=bc, eos=eos)
        assert rel_l1(prim["e"], rp["e"]) <= 1e-4, prec
        for g, r in zip(got, ref):
            assert abs(g.sum() - r.sum()) <= 1e-5 * np.abs(r).sum() + 1e-12, prec


def test_no_antiflux_differs_from_fused():
    """The stage left out is not a no-op: on a hot-spot state the two
    schemes part (the transport alone is more diffusive: lower peak)."""
    require_gpu()
    shape = (32, 32, 32)
    pr = W.hot_spots(shape=shape, seed=4, n_spots=4, sigma=(1.5, 3.0))
    U0 = oracle().prim2cons(OR.params(shape), *pr.as_list())
    a, pa, _ = run(shape, U0, 10, "fp32", "no_antiflux")
    b, pb, _ = run(shape, U0, 10, "fp32", "fused")
    assert rel_l1(pa["e"], pb["e"]) > 1e-3
    assert pa["e"].max() < pb["e"].max()


@pytest.mark.parametrize("scheme", ["fused", "no_antiflux"])
def test_ball_against_oracle(scheme):
    """64^3 expanding ball (radius 10 cells, e = 1 in a box at 1e-6):
    FP64 to 1e-12 per cell after 20 steps; FP32 (clamp margin 1e-6 on both
    sides) within 1e-4 relative L1 in e, totals within 1e-5."""
    require_gpu()
    N = 64
    shape = (N, N, N)
    eta = 0.125 if scheme == "fused" else 0.0
    O = oracle()
    P = OR.params(shape, eta=eta)
    U0 = O.prim2cons(P, *W.ball(N=N).as_list())
    ref = O.step(P, U0, 20)
    got, _, _ = run(shape, U0, 20, "fp64", scheme)
    assert max(max_rel_err(g, r) for g, r in zip(got, ref)) <= 1e-12
    P6 = OR.params(shape, eta=eta, delta=1e-6)
    ref6 = O.step(P6, U0, 20)
    rp6 = O.recover(P6, ref6)
    got, prim, _ = run(shape, U0, 20, "fp32", scheme, delta=1e-6)
    assert rel_l1(prim["e"], rp6["e"]) <= 1e-4
    for g, r in zip(got, ref6):
        assert abs(g.sum() - r.sum()) <= 1e-5 * np.abs(r).sum() + 1e-12


@pytest.mark.parametrize("bc", [OR.BC_REFLECT, OR.BC_PERIODIC, OR.BC_FROZEN])
@pytest.mark.parametrize("eos", [OR.EOS_IDEAL, OR.EOS_BAG])
@pytest.mark.parametrize("shape", [(37, 21, 13), (40, 3, 2), (5, 33, 9), (1, 1, 1)])
def test_split_against_oracle(shape, bc, eos):
    """Ragged shapes, every boundary rule and both EoS, 7 steps: relative
    L1 of e <= 1e-4 and totals within 1e-5 of the oracle; the first sweep's
    clamp count equals the fused sweep's (same level-n state, same
    recovery)."""
    require_gpu()
    P, U0 = state(shape, bc, eos, seed=5 * sum(shape) + bc + 3 * eos)
    O = oracle()
    ref = O.step(OR.params(shape, bc=bc, eos=eos, delta=1e-6), U0, 7)
    rp = O.recover(OR.params(shape, bc=bc, eos=eos, delta=1e-6), ref)
    got, prim, _ = run(shape, U0, 7, "fp32", "split", bc=bc, eos=eos)
    assert rel_l1(prim["e"], rp["e"]) <= 1e-4
    for g, r in zip(got, ref):
        assert abs(g.sum() - r.sum()) <= 1e-5 * np.abs(r).sum() + 1e-12
    counts = []
    for scheme in ("split", "fused"):
        with S.Solver(shape, precision="fp32", bc=BC_NAMES[bc], eos=EOS_NAMES[eos],
                      scheme=scheme) as s:
            s.set_conserved(U0)
            s.sweep(0)
            s.sync()
            counts.append(s.counters())
    assert counts[0] == counts[1]


def test_split_close_to_fused_on_hot_spots():
    """The two FP32 decompositions of the same method agree to rounding on
    a hot-spot state (20 steps; they differ only in the order of a few
    differences)."""
    require_gpu()
    shape = (48, 40, 36)
    pr = W.hot_spots(shape=shape, seed=8, n_spots=6, sigma=(2.0, 4.0), radial_flow=0.1)
    U0 = oracle().prim2cons(OR.params(shape), *pr.as_list())
    _, pa, _ = run(shape, U0, 20, "fp32", "split")
    _, pb, _ = run(shape, U0, 20, "fp32", "fused")
    assert rel_l1(pa["e"], pb["e"]) <= 2e-5


def test_ball_split_against_oracle():
    """The 64^3 ball with the split scheme: FP32 bar against the oracle at
    the FP32 clamp margin after 20 steps."""
    require_gpu()
    N = 64
    shape = (N, N, N)
    O = oracle()
    P6 = OR.params(shape, delta=1e-6)
    U0 = O.prim2cons(P6, *W.ball(N=N).as_list())
    ref = O.step(P6, U0, 20)
    rp = O.recover(P6, ref)
    got, prim, _ = run(shape, U0, 20, "fp32", "split", delta=1e-6)
    assert rel_l1(prim["e"], rp["e"]) <= 1e-4
    for g, r in zip(got, ref):
        assert abs(g.sum() - r.sum()) <= 1e-5 * np.abs(r).sum() + 1e-12
