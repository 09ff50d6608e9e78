"""Writes sensitivity.json: how far single-precision rounding alone carries the
plain SHASTA algorithm from the double-precision oracle, on the two
full-length workloads whose FP32 / MIXED GPU results the tests bound with it.

Both flows amplify rounding-size perturbations by orders of magnitude before
the stated step counts, so no single-precision computation can stay within a
fixed tolerance of the double-precision answer there.  The measure of what
single precision costs is the paper's own comparison (Sec. 4: the
single-precision implementation against a double-precision code): here the
oracle's source evaluated in single precision (oracle/shasta_oracle_f32.c)
against the oracle in double precision.

For each workload:

* reference: the double-precision oracle started from the initial conserved
  state rounded to float32 (the values an FP32 state holds), clamp margin
  delta = 1e-6 (the FP32 kernels' margin);
* members: the single-precision oracle started from that rounded state and
  from three seeded one-ulp perturbations of it (workloads.ulp_flips, seeds
  1-3), same delta;
* "single_precision": relative L1 distance of e between each member and the
  reference at the checkpoints, and the largest of them ("max");
* "fp64_input_flips": for comparison, the double-precision oracle from the
  three perturbed inputs against the reference (the spread the input
  perturbation alone causes when the arithmetic stays in double).

Workloads: hot spots 200^3 (30 spots, seed 2) at 75 .. 200 steps; blast
128^3 (e = 1e3 inside radius 10, 0.1 outside) at 50 and 125 steps.

Calls only the oracle (all host cores; about half an hour on eight):

    python tests/golden/make_sensitivity.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as OR  # noqa: E402
from paper_1206_0919_gb300 import workloads as W  # noqa: E402

SEEDS = (1, 2, 3)


def rel_l1(a, ref):
    a = np.asarray(a, dtype=np.float64)
    return float(np.abs(a - ref).sum() / np.abs(ref).sum())


def trajectory(O, P, U, checkpoints):
    """e at each checkpoint of one oracle run."""
    out, prev = {}, 0
    for m in checkpoints:
        U = O.step(P, U, m - prev, step0=prev)
        prev = m
        out[m] = np.asarray(O.recover(P, U)["e"], dtype=np.float64)
    return out


def study(O64, O32, P, U0, checkpoints):
    ref = trajectory(O64, P, W.rounded_to_single(U0), checkpoints)
    starts = {"rounded": W.rounded_to_single(U0)}
    starts.update({f"flips{s}": W.ulp_flips(U0, s) for s in SEEDS})
    single = {}
    for name, U in starts.items():
        tr = trajectory(O32, P, U, checkpoints)
        single[name] = {str(m): rel_l1(tr[m], ref[m]) for m in checkpoints}
    single["max"] = {str(m): max(single[k][str(m)] for k in starts) for m in checkpoints}
    flips64 = {}
    for s in SEEDS:
        tr = trajectory(O64, P, W.ulp_flips(U0, s), checkpoints)
        flips64[f"flips{s}"] = {str(m): rel_l1(tr[m], ref[m]) for m in checkpoints}
    flips64["max"] = {str(m): max(flips64[f"flips{s}"][str(m)] for s in SEEDS)
                      for m in checkpoints}
    return {"single_precision": single, "fp64_input_flips": flips64,
            "reference": "double-precision oracle from the float32-rounded state, delta 1e-6"}


def main():
    O64, O32 = OR.default(), OR.single()
    for O in (O64, O32):
        O.set_threads(os.cpu_count() or 1)
    out = {}
    N = 200
    P = OR.params((N, N, N), delta=1e-6)
    U0 = O64.prim2cons(P, *W.hot_spots(N=N, seed=2, n_spots=30).as_list())
    out["hot_spots_200"] = study(O64, O32, P, U0, (75, 100, 125, 150, 175, 200))
    n = 128
    P = OR.params((n, n, n), delta=1e-6)
    U0 = O64.prim2cons(P, *W.blast(N=n, radius=10.0).as_list())
    out["blast_128"] = study(O64, O32, P, U0, (50, 125))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sensitivity.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
