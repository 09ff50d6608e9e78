"""Host-side driver of the serving loop: replays an arrival stream against a
``shasta.Server``, collects per-event latencies and summarises them, and
splits a stream over ranks (one server per GPU, no data-path collective).
"""
from __future__ import annotations

import time

import numpy as np


def shard(stream, rank, world):
    """Events of one rank: every world-th event of the stream, starting at
    `rank` (arrival times are kept, so each rank sees 1/world of the rate)."""
    return [ev for i, ev in enumerate(stream) if i % world == rank]


def summary(latencies):
    """p50 / p99 / mean / max of a list of latencies in seconds."""
    a = np.asarray(latencies, dtype=np.float64)
    if a.size == 0:
        return {"n": 0, "p50": None, "p99": None, "mean": None, "max": None}
    return {"n": int(a.size), "p50": float(np.percentile(a, 50)),
            "p99": float(np.percentile(a, 99)), "mean": float(a.mean()), "max": float(a.max())}


def gather(values, dist=None):
    """All ranks' lists concatenated (on every rank); the list itself
    without a process group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return list(values)
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, list(values))
    return [v for p in parts for v in p]


def replay(server, events, inputs, poll_every=0.001, retry_sleep=0.0005, timeout=600.0,
           keep=None):
    """Submits `events` (dicts with t_arrival, N, eos, steps) at their
    arrival times, measured from the call, and polls until all have
    finished.  inputs(ev) gives the five primitive arrays of an event.

    Returns one record per event: arrival and submit times and the server's
    timings, all on the server's clock, plus the number of EAGAIN refusals
    the client met (the queue was full) before the event was accepted.
    keep(i), if given, picks the events whose result e is kept in the record
    (key "e"); the others' results are dropped once polled."""
    clock0 = server.clock()
    wall0 = time.perf_counter()
    pending, records = {}, []
    i = 0
    deadline = wall0 + timeout
    while i < len(events) or pending:
        now = time.perf_counter()
        if now > deadline:
            raise TimeoutError(f"{len(pending)} events still pending")
        if i < len(events) and now - wall0 >= events[i]["t_arrival"]:
            ev = events[i]
            N = ev["N"]
            refusals = 0
            while True:
                try:
                    t = server.submit((N, N, N), inputs(ev), ev["steps"], eos=ev["eos"])
                    break
                except Exception as e:  # EAGAIN: queue full, try again shortly
                    if getattr(e, "status", None) != 3:
                        raise
                    refusals += 1
                    _poll(server, pending, records, keep)
                    time.sleep(retry_sleep)
            pending[t] = {"i": i, "N": N, "eos": ev["eos"], "refusals": refusals,
                          "t_arrival": clock0 + ev["t_arrival"]}
            i += 1
            continue
        _poll(server, pending, records, keep)
        time.sleep(poll_every)
    records.sort(key=lambda r: r["i"])
    return records


def _poll(server, pending, records, keep=None):
    for t in list(pending):
        r = server.poll(t)
        if r is None:
            continue
        rec = pending.pop(t)
        rec.update(t_submit=r["t_submit"], t_admit=r["t_admit"], t_done=r["t_done"],
                   steps=r["steps"])
        if keep is not None and keep(rec["i"]) and "prims" in r:
            rec["e"] = r["prims"]["e"]
        records.append(rec)
