"""The benchmark's replica path on two gloo ranks (CPU, no GPU).

Under torchrun every rank advances its own events (replicas: the events of
this solver are independent, so there is no data-path collective).  The
process group only brackets the timed region with barriers, takes the
maximum of the timings over ranks and gathers summary numbers.  These tests
run that host logic of bench.py (`Ranks`, `job_rate`, `workload_seed`) as
two processes over gloo, with the timings of the two ranks made different
on purpose, and check that the oracle arm does its work on rank 0 only.
"""
import os
import sys
import time

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    ranks = bench.Ranks("gloo")
    res = {"rank": ranks.rank, "world": ranks.world, "local": ranks.local}
    # the timed region as bench.py brackets it: barrier, work, barrier; rank 1
    # is the slow one
    ranks.barrier()
    t0 = time.perf_counter()
    time.sleep(0.05 + 0.25 * rank)
    ranks.barrier()
    mine = time.perf_counter() - t0
    res["elapsed_mine"] = mine
    res["elapsed_max"] = ranks.max(0.05 + 0.25 * rank)
    res["sum"] = ranks.sum(rank + 1)
    res["gather"] = ranks.gather([10 * rank, 10 * rank + 1])
    res["seed"] = bench.workload_seed(rank)
    res["seeds"] = ranks.gather([bench.workload_seed(rank)])
    res["rate"] = bench.job_rate(ranks.world, 1000, res["elapsed_max"])
    # the oracle arm: ranks other than 0 return at once without output
    if rank != 0:
        class A:
            steps, warmup, grid, precision = 1, 0, 200, "fp32"
        t = time.perf_counter()
        res["reference_rc"] = bench.run_reference(A())
        res["reference_s"] = time.perf_counter() - t
    ranks.close()
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as fh:
        fh.write(repr(res))


def test_replica_timing_over_two_gloo_ranks(tmp_path):
    port = 29700 + (os.getpid() % 1000)
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    got = [eval(open(tmp_path / f"r{r}.txt").read()) for r in range(2)]
    for r, res in enumerate(got):
        assert (res["rank"], res["world"], res["local"]) == (r, 2, r)
        # the barrier after the work holds the fast rank until the slow one ends
        assert res["elapsed_mine"] >= 0.3 - 0.02
        # every rank reports the slowest rank's time, and the job rate counts
        # the units of both ranks over it
        assert res["elapsed_max"] == pytest.approx(0.30)
        assert res["rate"] == pytest.approx(2 * 1000 / 0.30)
        assert res["sum"] == 3.0
        assert res["gather"] == [0, 1, 10, 11]
        assert res["seeds"] == [2, 1002]  # each replica its own event
    assert got[1]["reference_rc"] == 0 and got[1]["reference_s"] < 5.0


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench

    saved = {k: os.environ.pop(k, None) for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    try:
        ranks = bench.Ranks("gloo")
        assert ranks.dist is None and ranks.world == 1
        ranks.barrier()
        assert ranks.max(1.5) == 1.5 and ranks.sum(2) == 2.0
        assert ranks.gather([4, 5]) == [4, 5]
        ranks.close()
    finally:
        for k, v in saved.items():
            if v is not None:
                os.environ[k] = v
