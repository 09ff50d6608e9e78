"""The benchmark's headline line on a GPU: one JSON line with the contract's
keys, the roofline of the sweep kernel, the end-to-end figure through the
public API, the clocks, and the batched, serving, precision and ALU-peak
legs, each with plausible values, and the event's error against FP64 (a
short run: one timed event)."""
import json
import os
import subprocess
import sys

import pytest

from gpu_util import require_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_headline_line_keys_and_legs():
    require_gpu()
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "1",
                        "--warmup", "1", "--e2e-events", "2", "--no-cpu-baseline"],
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.strip().splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "roofline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["unit"] == "cell-updates/s" and d["steps"] == 1 and d["n_gpus"] == 1
    assert 1e9 < d["value"] < 2e11
    rf = d["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and 0.05 < rf["frac"] < 1.2
    assert rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"])
    # the instruction-issue roof, when the committed capture matches the sources
    ri = d["roofline_issue"]
    if ri is not None:
        assert ri["bound"] == "issue" and 0.05 < ri["frac"] < 1.05
        assert ri["frac"] == pytest.approx(ri["achieved"] / ri["peak"])
    e2e = d["e2e"]
    assert e2e["h2d_bytes_per_step"] == 40 * 200 ** 3 and e2e["d2h_bytes_per_step"] == 48 * 200 ** 3
    assert 0.2 * d["value"] < e2e["value"] < 1.2 * d["value"]
    assert d["gpu_launches"] == 606
    for k in ("sm_mhz", "sm_max_mhz", "reasons"):
        assert k in d["clocks"], k
    b = d["batch64"]
    assert b["events"] == 64 and b["value"] > 1e9 and 0.05 < b["roofline"]["frac"] < 1.2
    # sampled events against FP64, beside their own one-ulp sensitivity (the
    # single-precision algorithm itself runs 2-30x its one-ulp spread)
    for acc in (b["accuracy"], d["serve"]["200_per_s"]["accuracy"]):
        assert len(acc["events"]) >= 3
        assert all(v["fp64_ulp_flip_spread"] > 0 for v in acc["events"].values())
        assert 0 < acc["max_ratio_to_spread"] < 100 and acc["max_rel_l1_e"] < 0.05
    for rate in ("60_per_s", "200_per_s"):
        s = d["serve"][rate]
        assert s["events"] == 300 and s["value"] > 1.0
        assert 0 < s["latency_s"]["p50"] <= s["latency_s"]["p99"]
    p = d["precisions"]
    assert p["mixed"]["value"] > 1e9 and p["mixed_fp64"]["value"] > 1e8
    a = d["alu_peaks"]
    assert a["fp32"]["tflops"] > 10 * a["fp64"]["tflops"] > 0
    assert d["fp64_path"]["speedup_of_value"] > 10
    # the event's error against FP64 after its 200 steps, within twice the
    # single-precision yardstick, and the drift of the conserved totals
    acc = d["accuracy"]
    assert acc["steps"] == 200 and acc["single_precision_yardstick"] > 0
    assert 0 < acc["rel_l1_e"] <= 2 * acc["single_precision_yardstick"]
    assert acc["totals_drift"]["E"] <= 1e-5 and acc["totals_drift"]["R"] <= 1e-5
