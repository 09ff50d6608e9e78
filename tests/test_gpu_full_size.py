"""Parity at the full workload sizes, in the launch configuration the
benchmark times (autotuned launch choice, six-step CUDA graphs).

Both long workloads amplify rounding-size perturbations by orders of
magnitude before their stated step counts, so at full length a result kept
in single precision is held to the error that single-precision rounding
alone produces, measured on the oracle's own algorithm: the oracle's source
evaluated in single precision, started from the float32-rounded state and
from three seeded one-ulp perturbations of it, against the double-precision
oracle (tests/golden/sensitivity.json, written from the oracle alone by
tests/golden/make_sensitivity.py; the same comparison of a single-precision
code with a double-precision one as in Sec. 4).  Every comparison starts the
GPU and the double-precision oracle from the same float32 values with the
same clamp margin (delta = 1e-6), so the gap is arithmetic alone.

* 200^3 hot spots (the benchmark's workload), FP32, MIXED and MIXED_FP64: relative L1
  error of e <= 1e-4 (the FP32 bar) at 75 steps; at 100, 150 and 200 steps
  at most twice the largest single-precision distance; conserved totals
  within 1e-5 of the oracle's and of their initial values (E, R).
* 64 uneven events in one batch, 100 steps (MIXED): the smallest events of
  the batch against the oracle, cell by cell (<= 1e-4).
* 512^3 blast, 500 steps: the totals of E and R in the closed box
  (reflecting walls) stay within 1e-5 of their initial values.  The same
  setup at 128^3 (radius 10 cells): <= 1e-4 at 50 steps, at most twice the
  largest single-precision distance at 125.

With SHASTA_REPORT_DIR set, the measured errors (with the yardsticks and
the clamp counts) are written to full_size_report.json there.
"""
import json
import os

import numpy as np
import pytest

from paper_1206_0919_gb300 import shasta as S
from paper_1206_0919_gb300 import workloads as W
from oracle import oracle as OR
from gpu_util import oracle, rel_l1, require_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

REPORT = {}


def report(key, value):
    REPORT[key] = value
    d = os.environ.get("SHASTA_REPORT_DIR")
    if d:
        with open(os.path.join(d, "full_size_report.json"), "w") as fh:
            json.dump(REPORT, fh, indent=1, sort_keys=True)


def totals_gap(got, ref):
    """max over fields of |sum(got) - sum(ref)| / sum|ref|."""
    out = []
    for g, r in zip(got, ref):
        out.append(abs(float(np.sum(g)) - float(np.sum(r))) / max(float(np.abs(r).sum()), 1e-300))
    return out


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "sensitivity.json")


def sensitivity():
    with open(GOLDEN) as fh:
        return json.load(fh)


CHECKPOINTS = (75, 100, 150, 200)


@pytest.fixture(scope="module")
def hot_spots_200():
    require_gpu()
    N = 200
    P = OR.params((N, N, N), delta=1e-6)
    O = oracle()
    U0 = W.rounded_to_single(O.prim2cons(P, *W.hot_spots(N=N, seed=2, n_spots=30).as_list()))
    ref, U, prev = {}, U0, 0
    for m in CHECKPOINTS:
        U = O.step(P, U, m - prev, step0=prev)
        prev = m
        ref[m] = O.recover(P, U)["e"]
    return U0, ref, U


@pytest.mark.parametrize("precision", ["fp32", "mixed", "mixed_fp64"])
def test_hot_spots_200_against_oracle(hot_spots_200, precision):
    U0, ref_e, ref = hot_spots_200
    N = 200
    yard = sensitivity()["hot_spots_200"]["single_precision"]["max"]
    err = {}
    with S.Solver((N, N, N), precision=precision) as s:  # autotune + graphs, as benched
        s.set_conserved(U0)
        prev = 0
        for m in CHECKPOINTS:
            s.step(m - prev)
            prev = m
            err[m] = rel_l1(s.get_primitives()["e"], ref_e[m])
        got = s.get_conserved()
        clamps = s.counters()
    gaps = totals_gap(got, ref)
    drift = [abs(float(np.sum(g)) - float(np.sum(u))) / float(np.abs(u).sum())
             for g, u in zip((got[0], got[4]), (U0[0], U0[4]))]
    report(f"hot_spots_200_{precision}", {
        "rel_l1_e": {str(m): err[m] for m in CHECKPOINTS},
        "single_precision_yardstick": {str(m): yard[str(m)] for m in CHECKPOINTS},
        "ratio_to_yardstick": {str(m): err[m] / yard[str(m)] for m in CHECKPOINTS},
        "clamped_recoveries": clamps,
        "totals_gap_vs_oracle_200": gaps, "drift_E_R_vs_initial_200": drift})
    assert err[75] <= 1e-4, err
    for m in CHECKPOINTS[1:]:
        assert err[m] <= 2 * yard[str(m)], (m, err[m], yard[str(m)])
    assert max(gaps) <= 1e-5, gaps
    assert max(drift) <= 1e-5, drift


def test_batch_64_events_sampled_against_oracle():
    require_gpu()
    evs = W.batch_events(n_events=64, seed=3)
    total = sum(ev["N"] ** 3 for ev in evs)
    smallest = sorted(range(len(evs)), key=lambda i: evs[i]["N"])[:3]
    inputs = {}
    with S.Batch(total + 64 * len(evs), precision="mixed", max_events=len(evs)) as b:
        ids = []
        for i, ev in enumerate(evs):
            pr = W.event_prims(ev).as_list()
            if i in smallest:
                inputs[i] = pr
            ids.append(b.add_primitives((ev["N"],) * 3, pr))
        b.step(100)
        got = {i: (b.get_primitives(ids[i]), b.get_conserved(ids[i])) for i in smallest}
    O = oracle()
    errs = {}
    for i in smallest:
        N = evs[i]["N"]
        P = OR.params((N, N, N))
        ref = O.step(P, O.prim2cons(P, *inputs[i]), 100)
        rp = O.recover(P, ref)
        errs[i] = (rel_l1(got[i][0]["e"], rp["e"]), max(totals_gap(got[i][1], ref)))
    report("batch_64_events_sampled_mixed", {f"event{i}_N{evs[i]['N']}": {"rel_l1_e": e, "totals_gap": t}
                                     for i, (e, t) in errs.items()})
    for i, (e, t) in errs.items():
        assert e <= 1e-4 and t <= 1e-5, (i, e, t)


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_blast_512(precision):
    require_gpu()
    # 512^3, 500 steps: conservation of E and R in the closed box
    N = 512
    pr = W.blast(N=N, radius=40.0)
    with S.Solver((N, N, N), precision=precision) as s:
        s.set_primitives(*pr.as_list())
        t0 = s.totals()
        s.step(500)
        t1 = s.totals()
        clamps = s.counters()
    del pr
    drift = [abs(t1[k] - t0[k]) / abs(t0[k]) for k in (0, 4)]
    # the same setup at 128^3 against the oracle, both from the float32-rounded
    # state at the same clamp margin
    n = 128
    small = W.blast(N=n, radius=10.0)
    O = oracle()
    P = OR.params((n, n, n), delta=1e-6)
    U0 = W.rounded_to_single(O.prim2cons(P, *small.as_list()))
    U50 = O.step(P, U0, 50)
    e50 = O.recover(P, U50)["e"]
    ref = O.step(P, U50, 75, step0=50)
    rp = O.recover(P, ref)
    with S.Solver((n, n, n), precision=precision, delta=1e-6) as s:
        s.set_conserved(U0)
        s.step(50)
        err50 = rel_l1(s.get_primitives()["e"], e50)
        s.step(75)
        prim = s.get_primitives()
        got = s.get_conserved()
        clamps128 = s.counters()
    err125 = rel_l1(prim["e"], rp["e"])
    gaps = totals_gap(got, ref)
    yard = sensitivity()["blast_128"]["single_precision"]["max"]
    report(f"blast_512_{precision}", {"drift_E_R_512": drift, "clamped_recoveries_512": clamps,
                                    "rel_l1_e_128": {"50": err50, "125": err125},
                                    "single_precision_yardstick_128": yard,
                                    "ratio_to_yardstick_128_125": err125 / yard["125"],
                                    "clamped_recoveries_128": clamps128,
                                    "totals_gap_128_125": gaps})
    assert max(drift) <= 1e-5, drift
    assert max(gaps) <= 1e-5, gaps
    assert err50 <= 1e-4, err50
    assert err125 <= 2 * yard["125"], (err125, yard)
