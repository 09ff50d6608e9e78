"""The sweep kernels stay inside their buffers.

compute-sanitizer is not available to these tests, so the library is built a
second time with SHASTA_CHECKED: every global access of the streaming sweeps
(state loads and stores, frozen-ghost loads, the range table; FP64, FP32 and
MIXED) and every shared-memory ring access of the FP32 / MIXED sweeps at a
computed offset is tested against its buffer's bounds first, and a miss is
counted and skipped.  A child process runs the checked library over ragged
shapes, every boundary rule, both closed-form EoS, single contexts under
every launch choice (autotuned, uniform and
forced work ranges, both register variants, CTA work shares) and batches of
uneven events (work units of whole line groups and of position ranges); it
must report no refused access, and its states must be bitwise those of the
regular library run the same way (the checks change nothing else)."""
import json
import os
import subprocess
import sys

import pytest

from gpu_util import require_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RUNNER = r"""
import hashlib, json, os, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
from paper_1206_0919_gb300 import shasta as S
from paper_1206_0919_gb300 import workloads as W
checked = os.environ.get("SHASTA_LIBRARY", "").endswith("libshasta_checked.so")

def h(arrays):
    d = hashlib.sha256()
    for a in arrays:
        d.update(np.ascontiguousarray(a).tobytes())
    return d.hexdigest()[:16]

SHAPES = [(13, 9, 7), (37, 21, 5), (3, 5, 2), (1, 1, 1), (40, 1, 1), (1, 33, 1), (2, 1, 29),
          (72, 56, 48), (17, 40, 9)]
CHOICES = [dict(autotune=True), dict(autotune=False),
           dict(autotune=False, env={"SHASTA_BALANCE": "0"}),
           dict(autotune=False, env={"SHASTA_RANGE": "5", "SHASTA_VARIANT": "1"}),
           dict(autotune=False, env={"SHASTA_RANGE": "37", "SHASTA_VARIANT": "0"}),
           dict(autotune=False, env={"SHASTA_RANGE": "100000"}),
           dict(autotune=False, env={"SHASTA_RANK_SKEW": "0.45", "SHASTA_EDGE_COST": "40"})]
ENV_KEYS = ("SHASTA_BALANCE", "SHASTA_RANGE", "SHASTA_VARIANT", "SHASTA_RANK_SKEW",
            "SHASTA_EDGE_COST", "SHASTA_BATCH_RANGE")
out = {}

def report(obj):
    return list(obj.checked_report()) if checked else [0, 0, 0]

for prec in ("fp32", "mixed", "fp64"):
    for si, shape in enumerate(SHAPES):
        for bc in ("reflect", "periodic", "frozen"):
            for eos in ("ideal", "bag"):
                pr = W.random_state(shape, seed=100 + si, vmax=0.6,
                                    e_range=(0.3, 3.0) if eos == "bag" else (0.05, 5.0))
                choices = CHOICES if (bc == "reflect" and eos == "ideal") else CHOICES[:2]
                for ci, ch in enumerate(choices):
                    for k in ENV_KEYS:
                        os.environ.pop(k, None)
                    os.environ.update(ch.get("env", {}))
                    with S.Solver(shape, precision=prec, bc=bc, eos=eos,
                                  autotune=ch["autotune"]) as s:
                        s.set_primitives(*pr.as_list())
                        s.step(7)
                        U = s.get_conserved()
                        out[f"{prec}/{shape}/{bc}/{eos}/{ci}"] = [h(U), s.counters(), report(s)]
for k in ENV_KEYS:
    os.environ.pop(k, None)
# batches: uneven events of every boundary rule and both EoS, whole line
# groups and position ranges as work units
for prec in ("fp32", "mixed"):
    for mode, env in (("auto", {}), ("groups", {"SHASTA_BATCH_RANGE": "0"}),
                      ("ranges", {"SHASTA_BATCH_RANGE": "29"})):
        for k in ENV_KEYS:
            os.environ.pop(k, None)
        os.environ.update(env)
        with S.Batch(2_000_000, precision=prec) as b:
            ids = []
            for i, shape in enumerate(SHAPES):
                bc = ("reflect", "periodic", "frozen")[i % 3]
                eos = ("ideal", "bag")[i % 2]
                pr = W.random_state(shape, seed=300 + i, vmax=0.6,
                                    e_range=(0.3, 3.0) if eos == "bag" else (0.05, 5.0))
                ids.append(b.add_primitives(shape, pr.as_list(), bc=bc, eos=eos))
                if i == 4:
                    b.step(3)  # later events join at another phase
            b.step(7)
            states = [h(b.get_conserved(e)) for e in ids]
            out[f"batch/{prec}/{mode}"] = [states, [b.counters(e) for e in ids], report(b)]
print(json.dumps(out))
"""


def run(env_extra):
    env = dict(os.environ)
    env.pop("SHASTA_LIBRARY", None)
    env.update(env_extra)
    r = subprocess.run([sys.executable, "-c", RUNNER, ROOT], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_stays_in_bounds():
    require_gpu()
    sys.path.insert(0, ROOT)
    from paper_1206_0919_gb300 import build as B

    checked_lib = B.build(checked=True)
    regular = run({})
    checked = run({"SHASTA_LIBRARY": checked_lib})
    assert checked.keys() == regular.keys()
    refused = {k: v[-1] for k, v in checked.items() if v[-1][0] != 0}
    assert not refused, f"accesses outside their buffers (count, code, index): {refused}"
    for k in regular:
        assert checked[k][:2] == regular[k][:2], k


PLANTED = r"""
import json, os, sys
sys.path.insert(0, sys.argv[1])
from paper_1206_0919_gb300 import shasta as S
from paper_1206_0919_gb300 import workloads as W
shape = (24, 20, 16)
pr = W.random_state(shape, seed=5)
with S.Solver(shape, precision="fp32", autotune=False, use_graphs=False) as s:
    s.set_primitives(*pr.as_list())
    os.environ["SHASTA_CHECKED_NCAP"] = str(24 * 20 * 16 // 2)
    s.step(1)
    print(json.dumps(list(s.checked_report())))
"""


def test_checked_build_refuses_accesses_past_a_smaller_bound():
    """The checks fire: with the state arrays' bound lowered to half the grid
    (a test aid of checked builds only), the sweeps' loads and stores of the
    upper half are refused and counted, not performed."""
    require_gpu()
    sys.path.insert(0, ROOT)
    from paper_1206_0919_gb300 import build as B

    env = dict(os.environ, SHASTA_LIBRARY=B.build(checked=True))
    r = subprocess.run([sys.executable, "-c", PLANTED, ROOT], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    count, code, index = json.loads(r.stdout.strip().splitlines()[-1])
    assert count > 0 and code in (1, 3) and index >= 24 * 20 * 16 // 2
