"""Tabulated EoS with the fixed-point recovery of Sec. 3, CUDA path against
the oracle (GPU).

The table holds p at e = k de (linear in between).  FP64 follows the
oracle's lookup and iteration operation for operation (<= 1e-12 per cell);
FP32 iterates in float to a 1e-7 change of |v| and meets the FP32 bar.
"""
import numpy as np
import pytest

from gpu_util import max_rel_err, oracle, rel_l1, require_gpu
from oracle import oracle as OR
from paper_1206_0919_gb300 import shasta as S
from paper_1206_0919_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BC_NAMES = {OR.BC_REFLECT: "reflect", OR.BC_PERIODIC: "periodic", OR.BC_FROZEN: "frozen"}
DE = 0.005
SOFT = np.arange(20001) * DE / 3.0 * (1.0 - np.exp(-np.arange(20001) * DE / 0.3))
IDEAL = np.arange(20001) * DE / 3.0


def run(shape, U0, nsteps, precision, table, bc=OR.BC_REFLECT, scheme="fused", delta=0.0):
    with S.Solver(shape, precision=precision, bc=BC_NAMES[bc], eos="table", table=table,
                  table_de=DE, scheme=scheme, delta=delta) as s:
        s.set_conserved(U0)
        s.step(nsteps)
        return s.get_conserved(), s.get_primitives(), s.totals()


def oracle_run(shape, U0, nsteps, table, bc=OR.BC_REFLECT, delta=1e-10):
    O = oracle()
    P = OR.params(shape, bc=bc, eos=OR.EOS_TABLE, table=table, table_de=DE, delta=delta)
    ref = O.step(P, U0, nsteps)
    return ref, O.recover(P, ref)


def state(shape, table, seed, vmax=0.6):
    pr = W.random_state(shape, seed=seed, vmax=vmax)
    P = OR.params(shape, eos=OR.EOS_TABLE, table=table, table_de=DE)
    return oracle().prim2cons(P, *pr.as_list())


@pytest.mark.parametrize("bc", [OR.BC_REFLECT, OR.BC_PERIODIC, OR.BC_FROZEN])
@pytest.mark.parametrize("shape", [(13, 9, 7), (37, 21, 5), (40, 1, 1), (1, 1, 1)])
@pytest.mark.parametrize("name", ["soft", "ideal"])
def test_fp64_table_against_oracle(shape, bc, name):
    """Ragged shapes, every boundary rule, 7 steps (the whole axis table):
    <= 1e-12 per cell, primitives included."""
    require_gpu()
    table = SOFT if name == "soft" else IDEAL
    U0 = state(shape, table, seed=sum(shape) + 7 * bc)
    ref, rp = oracle_run(shape, U0, 7, table, bc=bc)
    got, prim, tot = run(shape, U0, 7, "fp64", table, bc=bc)
    assert max(max_rel_err(g, r) for g, r in zip(got, ref)) <= 1e-12
    for k in ("e", "vx", "vy", "vz", "n", "p"):
        assert max_rel_err(prim[k], rp[k]) <= 1e-11, k


@pytest.mark.parametrize("scheme", ["fused", "split"])
@pytest.mark.parametrize("bc", [OR.BC_REFLECT, OR.BC_PERIODIC, OR.BC_FROZEN])
def test_fp32_table_against_oracle(bc, scheme):
    """FP32 (fused and split sweeps): relative L1 of e <= 1e-4 and totals
    within 1e-5 after 7 steps, at the FP32 clamp margin."""
    require_gpu()
    shape = (37, 21, 13)
    U0 = state(shape, SOFT, seed=31 + bc)
    ref, rp = oracle_run(shape, U0, 7, SOFT, bc=bc, delta=1e-6)
    got, prim, _ = run(shape, U0, 7, "fp32", SOFT, bc=bc, scheme=scheme)
    assert rel_l1(prim["e"], rp["e"]) <= 1e-4
    for g, r in zip(got, ref):
        assert abs(g.sum() - r.sum()) <= 1e-5 * np.abs(r).sum() + 1e-12


def test_fp32_ideal_table_follows_closed_form():
    """An FP32 run with the p = e/3 table stays within the FP32 bar of the
    closed-form ideal-gas run on hot spots (20 steps)."""
    require_gpu()
    shape = (48, 40, 36)
    pr = W.hot_spots(shape=shape, seed=9, n_spots=6, sigma=(2.0, 4.0), radial_flow=0.1)
    U0 = oracle().prim2cons(OR.params(shape), *pr.as_list())
    with S.Solver(shape, precision="fp32") as s:
        s.set_conserved(U0)
        s.step(20)
        ideal = s.get_primitives()
    _, prim, _ = run(shape, U0, 20, "fp32", IDEAL)
    assert rel_l1(prim["e"], ideal["e"]) <= 1e-4


def test_batches_and_servers_refuse_a_table():
    """Batches and the serving loop take closed-form EoS only: an event with
    a tabulated EoS is refused with EINVAL."""
    require_gpu()
    shape = (8, 8, 8)
    pr = W.hot_spots(shape=shape, seed=1, n_spots=2).as_list()
    with S.Batch(4096, max_events=4) as b:
        with pytest.raises(S.ShastaError) as ei:
            b.add_primitives(shape, pr, eos=S.EOS_TABLE)
        assert ei.value.status == S.EINVAL
    with S.Server(1 << 28) as srv:
        with pytest.raises(S.ShastaError) as ei:
            srv.submit(shape, pr, 2, eos=S.EOS_TABLE)
        assert ei.value.status == S.EINVAL
