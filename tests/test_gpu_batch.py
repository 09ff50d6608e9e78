"""Batched sweeps (include/shasta_batch.h) on the GPU.

Every event of a batch must advance exactly as a single context with the
same grid, boundary rule, EoS and lambda: the batched launch runs the same
arithmetic, so the comparison is bit for bit.  Events join at different
times (so they run different phases of the axis permutation of Sec. 3.1.4
in the same launches), are removed, and their pool room is reused.
"""
import numpy as np
import pytest

from paper_1206_0919_gb300 import shasta as S
from paper_1206_0919_gb300 import workloads as W
from oracle import oracle as OR
from gpu_util import oracle, rel_l1, require_gpu

pytestmark = pytest.mark.gpu

# (shape, bc, eos, seed, radial flow)
EVENTS = [
    ((40, 36, 28), "reflect", "ideal", 1, 0.1),
    ((33, 20, 48), "periodic", "bag", 2, 0.0),
    ((24, 40, 16), "frozen", "ideal", 3, 0.2),
    ((48, 48, 48), "reflect", "ideal", 4, 0.1),
    ((17, 9, 30), "reflect", "bag", 5, 0.0),
]


def prims_of(shape, seed, flow, eos):
    nx, ny, nz = shape
    p = W.hot_spots(seed=seed, n_spots=5, radial_flow=flow, shape=shape,
                    log10_amp=(-1.0, 0.3) if eos == "bag" else (-1.0, 1.0))
    return p.as_list()


def single(shape, bc, eos, prims, nsteps, precision):
    with S.Solver(shape, precision=precision, bc=bc, eos=eos) as s:
        s.set_primitives(*prims)
        s.step(nsteps)
        return s.get_conserved(), s.totals(), s.counters()


def capacity(events, extra=0):
    return sum(int(np.prod(e[0])) for e in events) + 64 * len(events) + extra


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
@pytest.mark.parametrize("graphs,tune,rng", [(True, True, None), (False, False, None),
                                             (True, False, "0"), (False, False, "19")])
def test_batch_matches_single_bitwise(monkeypatch, precision, graphs, tune, rng):
    """rng forces the work decomposition: "0" whole line groups, "19"
    ranges of 19 positions (lines cut at arbitrary and chunk-rounded
    places, across event boundaries)."""
    require_gpu()
    if rng is not None:
        monkeypatch.setenv("SHASTA_BATCH_RANGE", rng)
    with S.Batch(capacity(EVENTS), precision=precision, use_graphs=graphs,
                 autotune=tune) as b:
        ids, prims = [], []
        for shape, bc, eos, seed, flow in EVENTS[:2]:
            pr = prims_of(shape, seed, flow, eos)
            ids.append(b.add_primitives(shape, pr, bc=bc, eos=eos))
            prims.append(pr)
        b.step(2)
        for shape, bc, eos, seed, flow in EVENTS[2:]:
            pr = prims_of(shape, seed, flow, eos)
            ids.append(b.add_primitives(shape, pr, bc=bc, eos=eos))
            prims.append(pr)
        b.step(7)  # six as one graph (when enabled), one more directly
        info = b.info()
        assert info["events"] == len(EVENTS)
        assert 1 <= info["launches_per_step"] <= 3 * 3 * 2
        for eid, (shape, bc, eos, seed, flow), pr in zip(ids, EVENTS, prims):
            k = b.steps_done(eid)
            assert k == (9 if eid in ids[:2] else 7)
            ref, rtot, rcnt = single(shape, bc, eos, pr, k, precision)
            got = b.get_conserved(eid)
            for f, (g, r) in enumerate(zip(got, ref)):
                assert np.array_equal(g, r), (shape, bc, eos, f, float(np.abs(g - r).max()))
            assert np.array_equal(b.totals(eid), rtot)
            assert b.counters(eid) == rcnt


def test_batch_event_vs_oracle():
    """One hot-spot event inside a batch of three against the FP64 oracle
    (FP32 bar: relative L1 error of e <= 1e-4, totals within 1e-5 of the
    oracle's)."""
    require_gpu()
    shape = (32, 28, 24)
    P = OR.params(shape)
    O = oracle()
    pr = prims_of(shape, 9, 0.1, "ideal")
    U0 = O.prim2cons(P, *pr)
    ref = O.step(P, U0, 12)
    with S.Batch(3 * 32 * 28 * 24 + 1024) as b:
        other = [b.add_primitives(shape, prims_of(shape, s, 0.0, "ideal")) for s in (10, 11)]
        eid = b.add_conserved(shape, U0)
        b.step(12)
        prim = b.get_primitives(eid)
        got = b.get_conserved(eid)
        assert len(other) == 2
    rp = O.recover(P, ref)
    assert rel_l1(prim["e"], rp["e"]) <= 1e-4
    # totals against the oracle's after the same steps (momentum is not
    # conserved against reflecting walls; E and R are)
    t_ref, t1 = O.totals(ref), np.array([float(np.sum(u)) for u in got])
    scale = np.array([np.abs(u).sum() for u in ref])
    assert np.all(np.abs(t1 - t_ref) <= 1e-5 * scale), (t1, t_ref)
    t0 = O.totals(U0)
    assert abs(t1[0] - t0[0]) <= 1e-5 * scale[0] and abs(t1[4] - t0[4]) <= 1e-5 * scale[4]


def test_batch_remove_and_reuse():
    """Removing an event frees its room; a new event fills the hole and the
    remaining events are unaffected."""
    require_gpu()
    shapes = [(32, 32, 32), (24, 24, 24), (32, 32, 32)]
    cap = sum(int(np.prod(s)) for s in shapes) + 3 * 64
    with S.Batch(cap, autotune=False) as b:
        prims = [prims_of(s, 20 + i, 0.1, "ideal") for i, s in enumerate(shapes)]
        ids = [b.add_primitives(s, p) for s, p in zip(shapes, prims)]
        b.step(3)
        with pytest.raises(S.ShastaError) as ei:
            b.add_primitives((40, 40, 40), prims_of((40, 40, 40), 30, 0.0, "ideal"))
        assert ei.value.status == S.EAGAIN
        b.remove(ids[1])
        assert b.steps_done(ids[1]) == -1
        with pytest.raises(S.ShastaError) as ei:
            b.get_conserved(ids[1])
        assert ei.value.status == S.ENOTFOUND
        new_shape = (20, 24, 24)
        pn = prims_of(new_shape, 31, 0.0, "ideal")
        nid = b.add_primitives(new_shape, pn)
        b.step(4)
        for eid, s, p in ((ids[0], shapes[0], prims[0]), (ids[2], shapes[2], prims[2]),
                          (nid, new_shape, pn)):
            ref, _, _ = single(s, "reflect", "ideal", p, b.steps_done(eid), "fp32")
            got = b.get_conserved(eid)
            assert all(np.array_equal(g, r) for g, r in zip(got, ref)), s


def test_batch_errors():
    require_gpu()
    with pytest.raises(S.ShastaError) as ei:
        S.Batch(1000, precision="fp64")
    assert ei.value.status == S.EINVAL
    with pytest.raises(S.ShastaError) as ei:
        S.Batch(0)
    assert ei.value.status == S.EINVAL
    with S.Batch(4096, max_events=2) as b:
        pr = prims_of((8, 8, 8), 1, 0.0, "ideal")
        b.add_primitives((8, 8, 8), pr)
        b.add_primitives((8, 8, 8), pr)
        with pytest.raises(S.ShastaError) as ei:
            b.add_primitives((8, 8, 8), pr)
        assert ei.value.status == S.EAGAIN
        with pytest.raises(S.ShastaError) as ei:
            b.add_primitives((20, 20, 20), prims_of((20, 20, 20), 1, 0.0, "ideal"))
        assert ei.value.status == S.EINVAL  # larger than the whole pool
        bad = [a.copy() for a in pr]
        bad[1][0, 0, 0] = 1.5  # |v| >= 1
        b.remove(0)
        with pytest.raises(S.ShastaError) as ei:
            b.add_primitives((8, 8, 8), bad)
        assert ei.value.status == S.EUNPHYSICAL
        with pytest.raises(S.ShastaError) as ei:
            b.add_primitives((8, 8, 8), pr, lam=0.7)
        assert ei.value.status == S.EINVAL


def test_batch_device_arrays_and_empty_step():
    """Device (torch) input and output arrays; stepping an empty batch is a
    no-op."""
    require_gpu()
    import torch
    shape = (24, 20, 16)
    pr = prims_of(shape, 7, 0.1, "ideal")
    with S.Batch(8192) as b:
        b.step(3)
        dev = [torch.from_numpy(a).cuda() for a in pr]
        eid = b.add_primitives(shape, dev)
        b.step(5)
        out = [torch.empty(b.shapes[eid], dtype=torch.float64, device="cuda") for _ in range(5)]
        b.get_conserved(eid, out)
        got = [o.cpu().numpy() for o in out]
    ref, _, _ = single(shape, "reflect", "ideal", pr, 5, "fp32")
    assert all(np.array_equal(g, r) for g, r in zip(got, ref))


def test_batch_checkpoint_resume_bitwise():
    """An event saved after 5 steps (conserved state + step counter) and
    added again with its counter restored continues exactly as if it had
    never left the batch, while another event keeps running."""
    require_gpu()
    shape, other = (32, 24, 20), (24, 24, 24)
    pa, pb = prims_of(shape, 41, 0.1, "ideal"), prims_of(other, 42, 0.0, "ideal")
    cap = 4 * (32 * 24 * 20 + 24 ** 3)
    with S.Batch(cap, check_input=False) as b:  # a saved state is taken as it is
        ia, ib = b.add_primitives(shape, pa), b.add_primitives(other, pb)
        b.step(5)
        saved, k = b.get_conserved(ia), b.steps_done(ia)
        b.remove(ia)
        b.step(2)  # the other event runs on meanwhile
        ia2 = b.add_conserved(shape, saved)
        b.set_step_counter(ia2, k)
        b.step(9)
        got = b.get_conserved(ia2)
        assert b.steps_done(ia2) == 14
    ref, _, _ = single(shape, "reflect", "ideal", pa, 14, "fp32")
    assert all(np.array_equal(g, r) for g, r in zip(got, ref))
