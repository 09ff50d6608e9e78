"""Serving loop (include/shasta_serve.h) on the GPU.

The central property: an event's result does not depend on what else the
server is running.  Each event is run alone (a server with nothing else to
do) and in a mix (submitted together with the others, so that they are
admitted while others are resident and advance in shared launches); the
two results must agree bit for bit, and agree with a single context.
"""
import time

import numpy as np
import pytest

from paper_1206_0919_gb300 import shasta as S
from paper_1206_0919_gb300 import workloads as W
from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

# (shape, eos, nsteps, seed)
MIX = [
    ((32, 32, 32), "ideal", 9, 1),
    ((48, 40, 24), "bag", 4, 2),
    ((24, 24, 24), "ideal", 13, 3),
    ((40, 40, 40), "bag", 7, 4),
    ((16, 48, 32), "ideal", 0, 5),
    ((36, 28, 44), "ideal", 6, 6),
]


def prims_of(shape, seed, eos):
    return W.hot_spots(seed=seed, n_spots=6, radial_flow=0.1, shape=shape,
                       log10_amp=(-1.0, 0.3) if eos == "bag" else (-1.0, 1.0)).as_list()


def wait(srv, ticket, timeout=120.0):
    t_end = time.time() + timeout
    while time.time() < t_end:
        r = srv.poll(ticket)
        if r is not None:
            return r
        time.sleep(0.002)
    raise AssertionError("event did not finish")


def run_alone(shape, eos, nsteps, seed, precision):
    with S.Server(1 << 30, precision=precision) as srv:
        t = srv.submit(shape, prims_of(shape, seed, eos), nsteps, eos=eos, cons_out=True)
        return wait(srv, t)


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_results_same_alone_and_in_the_mix(precision):
    require_gpu()
    alone = [run_alone(sh, eos, k, seed, precision) for sh, eos, k, seed in MIX]
    # the mix: at most three resident at once, so that later events join a
    # batch that is already running (inputs made first: the submissions
    # follow each other closely)
    inputs = [prims_of(sh, seed, eos) for sh, eos, k, seed in MIX]
    with S.Server(1 << 30, precision=precision, max_resident=3, steps_per_round=1) as srv:
        tickets = [srv.submit(sh, pr, k, eos=eos, cons_out=True)
                   for (sh, eos, k, seed), pr in zip(MIX, inputs)]
        srv.drain(120.0)
        mixed = [srv.poll(t) for t in tickets]
        st = srv.stats()
    assert st["finished"] == len(MIX) and st["failed"] == 0
    assert st["peak_resident"] >= 2, st  # events really shared the batch
    # resident events stay at one phase of the axis table: every sweep slot
    # sweeps one axis, at most one launch per EoS (2 EoS x 3 slots a step)
    assert st["sweep_launches"] <= 6 * st["batch_steps"], st
    for (sh, eos, k, seed), a, m in zip(MIX, alone, mixed):
        assert a["steps"] == m["steps"] == k
        for key in ("e", "vx", "vy", "vz", "n", "p"):
            assert np.array_equal(a["prims"][key], m["prims"][key]), (sh, eos, key)
        for f in range(5):
            assert np.array_equal(a["cons"][f], m["cons"][f]), (sh, eos, f)
        assert a["clamp_count"] == m["clamp_count"]
        assert m["t_submit"] <= m["t_admit"] <= m["t_done"]
    # and the same as a single context
    sh, eos, k, seed = MIX[3]
    with S.Solver(sh, precision=precision, eos=eos) as s:
        s.set_primitives(*prims_of(sh, seed, eos))
        s.step(k)
        ref = s.get_conserved()
    assert all(np.array_equal(r, g) for r, g in zip(ref, mixed[3]["cons"]))


def test_admission_by_footprint():
    """A pool with room for one 32^3 event: three of them run one after the
    other, each admitted only after the previous one left."""
    require_gpu()
    shape = (32, 32, 32)
    cells = 32 ** 3
    staging = 4 * 11 * 8 * cells
    budget = staging + 40 * (cells + 16)
    with S.Server(budget, staging_bytes=staging) as srv:
        assert srv.stats()["pool_cells"] < 2 * cells
        ts = [srv.submit(shape, prims_of(shape, 10 + i, "ideal"), 5) for i in range(3)]
        srv.drain(120.0)
        res = [srv.poll(t) for t in ts]
        st = srv.stats()
    assert st["peak_resident"] == 1
    for a, b in zip(res, res[1:]):
        assert b["t_admit"] >= a["t_admit"]
    assert all(r["steps"] == 5 for r in res)


def test_queue_full_and_bad_events():
    require_gpu()
    shape = (32, 32, 32)
    cells = 32 ** 3
    staging = 4 * 11 * 8 * cells
    budget = staging + 40 * (cells + 16)
    with S.Server(budget, staging_bytes=staging, max_queue=2) as srv:
        long_t = srv.submit(shape, prims_of(shape, 1, "ideal"), 60)
        accepted, refused = [], 0
        for i in range(4):
            try:
                accepted.append(srv.submit(shape, prims_of(shape, 2 + i, "ideal"), 1))
            except S.ShastaError as e:
                assert e.status == S.EAGAIN
                refused += 1
        assert refused >= 1
        # invalid arguments are refused at once
        with pytest.raises(S.ShastaError) as ei:
            srv.submit(shape, prims_of(shape, 1, "ideal"), 3, lam=0.9)
        assert ei.value.status == S.EINVAL
        with pytest.raises(S.ShastaError) as ei:
            srv.submit((64, 64, 64), prims_of((64, 64, 64), 1, "ideal"), 3)
        assert ei.value.status == S.EINVAL  # never fits the pool
        srv.drain(120.0)
        assert srv.poll(long_t)["steps"] == 60
        for t in accepted:
            assert srv.poll(t)["steps"] == 1
        with pytest.raises(S.ShastaError) as ei:
            srv.poll(long_t)
        assert ei.value.status == S.ENOTFOUND
    # an unphysical event fails on its own; the others finish
    with S.Server(1 << 28) as srv:
        bad = prims_of(shape, 3, "ideal")
        bad[1] = bad[1].copy()
        bad[1][3, 3, 3] = 1.2
        tb = srv.submit(shape, bad, 4)
        tg = srv.submit(shape, prims_of(shape, 4, "ideal"), 4)
        srv.drain(120.0)
        with pytest.raises(S.ShastaError) as ei:
            srv.poll(tb)
        assert ei.value.status == S.EUNPHYSICAL
        assert srv.poll(tg)["steps"] == 4
        st = srv.stats()
        assert st["failed"] == 1 and st["finished"] == 1


def test_drain_times_out_then_completes():
    """A bounded wait that runs out returns ETIMEOUT and leaves the server
    working: the event still finishes and a later drain succeeds."""
    require_gpu()
    shape = (96, 96, 96)
    with S.Server(1 << 30) as srv:
        t = srv.submit(shape, prims_of(shape, 7, "ideal"), 400)
        with pytest.raises(S.ShastaError) as ei:
            srv.drain(1e-4)
        assert ei.value.status == S.ETIMEOUT
        r = srv.poll(t)  # almost surely still running (about 100 rounds of steps)
        if r is None:
            srv.drain(120.0)
            r = srv.poll(t)
        assert r["steps"] == 400


def test_conserved_inputs_and_their_scan():
    """Events given as conserved fields: a valid one gives the single
    context's result bit for bit and reports the clamp counter; one with a
    cell where |M| >= E is refused (EUNPHYSICAL) by the scan on the copy
    stream while the other events keep running; an event without result
    buffers still finishes."""
    require_gpu()
    from oracle import oracle as OR
    from gpu_util import oracle
    shape = (24, 20, 16)
    P = OR.params(shape)
    U = oracle().prim2cons(P, *prims_of(shape, 12, "ideal"))
    bad = [u.copy() for u in U]
    bad[1][2, 3, 4] = 1.5 * bad[0][2, 3, 4]  # |M| > E
    with S.Server(1 << 30) as srv:
        tg = srv.submit(shape, U, 11, kind="conserved", cons_out=True)
        tb = srv.submit(shape, bad, 11, kind="conserved")
        tn = srv.submit(shape, U, 5, kind="conserved", prims_out=False)
        srv.drain(120.0)
        good = srv.poll(tg)
        with pytest.raises(S.ShastaError) as ei:
            srv.poll(tb)
        assert ei.value.status == S.EUNPHYSICAL
        assert srv.poll(tn)["steps"] == 5
    with S.Solver(shape) as s:
        s.set_conserved(U)
        s.step(11)
        ref = s.get_conserved()
        clamps = s.counters()
    assert all(np.array_equal(r, g) for r, g in zip(ref, good["cons"]))
    assert good["clamp_count"] == clamps
