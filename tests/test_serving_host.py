"""Host logic of the serving driver (paper_1206_0919_gb300/serving.py): no
GPU.  Sharding of an arrival stream over ranks, latency summaries, the
gather over a gloo process group of two ranks, and the client replay loop
against a fake server that refuses submissions when its queue is full."""
import os
import time

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1206_0919_gb300 import serving
from paper_1206_0919_gb300 import workloads as W


def test_shard_partitions_the_stream():
    stream = W.serving_stream(n_events=37, rate_hz=500.0, seed=9)
    parts = [serving.shard(stream, r, 3) for r in range(3)]
    assert sum(len(p) for p in parts) == len(stream)
    merged = sorted((ev for p in parts for ev in p), key=lambda e: e["t_arrival"])
    assert merged == stream
    for p in parts:  # arrival order kept within a shard
        assert all(a["t_arrival"] < b["t_arrival"] for a, b in zip(p, p[1:]))


def test_stream_recipe():
    """Poisson arrivals of mean rate, size mix 40/30/20/10, EoS alternating."""
    s = W.serving_stream(n_events=4000, rate_hz=200.0, seed=4)
    gaps = np.diff([0.0] + [e["t_arrival"] for e in s])
    assert abs(gaps.mean() - 1 / 200.0) < 0.05 / 200.0 * 4
    sizes = np.array([e["N"] for e in s])
    for N, p in zip(W.SERVE_SIZES, W.SERVE_PROBS):
        assert abs((sizes == N).mean() - p) < 0.03
    assert [e["eos"] for e in s[:4]] == ["ideal", "bag", "ideal", "bag"]
    assert all(e["steps"] == 150 for e in s)


def test_summary():
    lat = list(np.linspace(0.0, 1.0, 101))
    s = serving.summary(lat)
    assert s["n"] == 101 and s["p50"] == pytest.approx(0.5) and s["p99"] == pytest.approx(0.99)
    assert s["max"] == 1.0 and s["mean"] == pytest.approx(0.5)
    assert serving.summary([])["p99"] is None


def _gather_worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [rank + 0.1 * k for k in range(3 + rank)]
    allv = serving.gather(local, dist)
    s = serving.summary(allv)
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as fh:
        fh.write(repr((allv, s["p50"], s["p99"])))
    dist.destroy_process_group()


def test_gather_over_two_gloo_ranks(tmp_path):
    port = 29500 + (os.getpid() % 1000)
    mp.start_processes(_gather_worker, args=(2, port, str(tmp_path)), nprocs=2,
                       start_method="spawn")
    got = [eval(open(tmp_path / f"r{r}.txt").read()) for r in range(2)]
    expect = [0.0, 0.1, 0.2] + [1.0, 1.1, 1.2, 1.3]
    for allv, p50, p99 in got:
        assert allv == pytest.approx(expect)
        assert p50 == pytest.approx(float(np.percentile(expect, 50)))
        assert p99 == pytest.approx(float(np.percentile(expect, 99)))
    assert serving.gather([1, 2]) == [1, 2]  # no process group: the list itself


class _Refused(Exception):
    status = 3  # EAGAIN


class FakeServer:
    """Finishes each event `delay` seconds after its submission; refuses
    every submission while `cap` events are unfinished."""

    def __init__(self, delay=0.01, cap=2):
        self.t0 = time.perf_counter()
        self.delay, self.cap = delay, cap
        self.jobs, self.next = {}, 1

    def clock(self):
        return time.perf_counter() - self.t0

    def submit(self, shape, arrays, nsteps, eos="ideal"):
        now = self.clock()
        if sum(1 for j in self.jobs.values() if j[1] > now) >= self.cap:
            raise _Refused()
        t = self.next
        self.next += 1
        self.jobs[t] = (now, now + self.delay, nsteps)
        return t

    def poll(self, t):
        sub, done, k = self.jobs[t]
        if self.clock() < done:
            return None
        del self.jobs[t]
        return {"t_submit": sub, "t_admit": sub, "t_done": done, "steps": k}


def test_replay_against_a_fake_server():
    events = [dict(t_arrival=0.002 * i, N=8, eos="ideal", steps=3 + i) for i in range(12)]
    srv = FakeServer(delay=0.01, cap=2)
    recs = serving.replay(srv, events, lambda ev: None)
    assert [r["i"] for r in recs] == list(range(12))
    assert all(r["steps"] == 3 + r["i"] for r in recs)
    assert sum(r["refusals"] for r in recs) > 0  # the queue filled up
    for r in recs:
        assert r["t_arrival"] <= r["t_submit"] + 1e-3 <= r["t_done"] + 1e-3
