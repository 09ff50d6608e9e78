"""Writes sensitivity.json: how far the FP64 oracle's own answer moves under
perturbations of the size an FP32 computation makes, on the two full-length
workloads whose FP32 results the GPU tests bound with it.

* hot spots 200^3 (30 spots, seed 2): the oracle from the initial state
  against the oracle from the same state rounded to FP32 (relative L1
  difference of e after 25 .. 200 steps).  The flow amplifies the input
  rounding (about 1e-8) by about 1e5 by step 200.
* blast 128^3 (e = 1e3 inside radius 10, 0.1 outside): the oracle with the
  clamp margin |M| <= (1 - delta) E at delta = 1e-10 against delta = 1e-6
  (the FP32 default; FP32 cannot resolve a smaller margin) after 25, 50
  and 125 steps.  The front keeps producing states with |M| >= E that the
  recovery clamps, so the answer depends on the margin.

Calls only the oracle (all host cores; about ten minutes on eight):

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


def rel_l1(a, b):
    return float(np.abs(a - b).sum() / np.abs(a).sum())


def main():
    O = OR.default()
    O.set_threads(os.cpu_count() or 1)
    out = {}
    N = 200
    P = OR.params((N, N, N))
    U0 = O.prim2cons(P, *W.hot_spots(N=N, seed=2, n_spots=30).as_list())
    U0r = [u.astype(np.float32).astype(np.float64) for u in U0]
    A, B, prev, curve = U0, U0r, 0, {}
    for m in (25, 50, 75, 100, 150, 200):
        A = O.step(P, A, m - prev, step0=prev)
        B = O.step(P, B, m - prev, step0=prev)
        prev = m
        curve[str(m)] = rel_l1(O.recover(P, A)["e"], O.recover(P, B)["e"])
    out["hot_spots_200_input_rounding"] = curve
    n = 128
    prims = W.blast(N=n, radius=10.0).as_list()
    res = {}
    for d in (1e-10, 1e-6):
        P = OR.params((n, n, n), delta=d)
        U, prev = O.prim2cons(P, *prims), 0
        for m in (25, 50, 125):
            U = O.step(P, U, m - prev, step0=prev)
            prev = m
            res[(d, m)] = O.recover(P, U)["e"]
    out["blast_128_delta_1e-6_vs_1e-10"] = {str(m): rel_l1(res[(1e-10, m)], res[(1e-6, m)])
                                            for m in (25, 50, 125)}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sensitivity.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1, sort_keys=True)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
