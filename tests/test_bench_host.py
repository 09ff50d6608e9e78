"""Host-side helpers of bench.py that need no GPU: the relative L1 distance,
the accuracy summary of sampled results, the oracle-rate sampling bound and
the workload seeds of replica ranks."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_rel_l1():
    ref = np.array([1.0, -2.0, 3.0, 0.0])
    assert bench.rel_l1(ref, ref) == 0.0
    got = ref + np.array([0.0, 0.6, 0.0, 0.0])
    assert bench.rel_l1(got, ref) == pytest.approx(0.1)
    # symmetric perturbation sizes count alike
    assert bench.rel_l1(ref - np.array([0.6, 0, 0, 0]), ref) == pytest.approx(0.1)


def test_accuracy_summary_takes_the_worst_event():
    errs = {"a": {"rel_l1_e": 1e-6, "fp64_ulp_flip_spread": 1e-7},
            "b": {"rel_l1_e": 4e-4, "fp64_ulp_flip_spread": 2e-5},
            "c": {"rel_l1_e": 2e-4, "fp64_ulp_flip_spread": 1e-6}}
    s = bench.accuracy_summary(errs, 112)
    assert s["max_rel_l1_e"] == 4e-4
    assert s["max_ratio_to_spread"] == pytest.approx(200.0)  # event c
    assert s["steps"] == 112 and s["events"] is errs
    # a zero spread (a flow that does not amplify) gives a huge ratio, not an error
    s0 = bench.accuracy_summary({"z": {"rel_l1_e": 1e-7, "fp64_ulp_flip_spread": 0.0}}, 3)
    assert s0["max_ratio_to_spread"] > 1e100


def test_replica_seeds_differ():
    seeds = {bench.workload_seed(r) for r in range(8)}
    assert len(seeds) == 8 and bench.workload_seed(0) == 2


def test_oracle_rate_sample_is_bounded(monkeypatch):
    """oracle_rate runs whole steps until the time target and never past the
    event's steps (a fake oracle stands in for the C library)."""
    calls = []

    class FakeOracle:
        def set_threads(self, n):
            pass

        def prim2cons(self, P, *prims):
            return prims

        def step(self, P, U, n, step0=0):
            calls.append(step0)
            return U

    import oracle.oracle as OR
    monkeypatch.setattr(OR, "default", lambda: FakeOracle())
    monkeypatch.setattr(OR, "params", lambda shape: None)
    monkeypatch.setattr(bench, "workload_prims", lambda N: type("P", (), {"as_list": lambda self: []})())
    rate, threads, steps, t = bench.oracle_rate(4, target_s=0.0, threads=3)
    assert steps == 1 and threads == 3 and calls == [0]
    calls.clear()
    rate, threads, steps, t = bench.oracle_rate(4, max_steps=5, target_s=1e9, threads=1)
    assert steps == 5 and calls == [0, 1, 2, 3, 4]


def test_committed_figures_only_for_the_current_kernel_sources(tmp_path, monkeypatch):
    """The roofline's traffic and instruction counts come from the committed
    ncu summary only while its kernel-source hash is that of the sources."""
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "sweep_kernel_hot_spots.md").write_text(
        "kernel sources sha256[:16]: 0123456789abcdef\n"
        "traffic_per_launch[fp32,200]: 3.10e8\n"
        "inst_per_cell[fp32,200]: 11.05\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0123456789abcdef")
    assert bench.committed_traffic("fp32", 200) == 3.1e8
    assert bench.committed_figure("inst_per_cell", "fp32", 200) == 11.05
    assert bench.committed_figure("inst_per_cell", "fp32", 256) is None
    assert bench.committed_figure("inst_per_cell", "mixed", 200) is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "fedcba9876543210")
    assert bench.committed_traffic("fp32", 200) is None
    assert bench.committed_figure("inst_per_cell", "fp32", 200) is None
