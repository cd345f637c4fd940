"""Serving loop over a request trace: continuous batching versus one solve at a
time on the same GPU.

Requests are problem dicts with ``arrival_s`` (seconds after the start of the
run) and ``steps`` (see ``workloads.serving_trace``).  Both loops run in real
time: a request can be admitted only once its arrival time has passed, and its
latency is its completion time minus its arrival time (queueing included).
A request is complete when its whole force/torque series is back on the host.

``serve_batched`` keeps a queue of arrived requests and admits from it into a
``lbm.Batch`` while slots and the memory budget allow; the batch advances every
resident solve together, ``ticks_per_launch`` steps per graph replay, and
finished solves are read back and released between replays.
``serve_sequential`` solves the requests one after another, each as a
standalone ``lbm.Domain`` advanced by ``lbm_step``.  Both take the queue in
arrival order (``policy="fifo"``) or smallest work first (``policy="sjf"``:
cells x steps, ties in arrival order), the classic way to lower the median
latency of a queue.
"""
from __future__ import annotations

import time
from collections import deque

import numpy as np

from . import lbm
from .workloads import cells


def _summary(lat, makespan, cell_updates, n):
    lat = np.asarray(lat, dtype=float)
    return {
        "requests": int(n),
        "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
        "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
        "mean_s": float(lat.mean()) if lat.size else None,
        "makespan_s": float(makespan),
        "cell_updates": int(cell_updates),
        "mlups": float(cell_updates / makespan / 1e6) if makespan > 0 else None,
    }


def _wait_until(t0, t_abs):
    while True:
        now = time.perf_counter() - t0
        if now >= t_abs:
            return
        time.sleep(min(t_abs - now, 0.002))


def _work(r) -> int:
    return cells(r) * int(r["steps"])


def _next_index(waiting, policy: str) -> int:
    """index in `waiting` of the request to serve next"""
    if policy == "fifo" or len(waiting) < 2:
        return 0
    if policy == "sjf":
        return min(range(len(waiting)), key=lambda k: (_work(waiting[k]), k))
    raise ValueError(f"unknown policy {policy!r}")


def serve_batched(trace, budget_bytes: int, max_slots: int = 64, ticks_per_launch: int = 32,
                  launches_per_round: int = 1, device: int = 0, keep_series: bool = False, policy: str = "fifo"):
    """Continuous batching.  Returns (summary dict, {request id: force/torque
    series} if keep_series)."""
    reqs = sorted(trace, key=lambda r: r["arrival_s"])
    batch = lbm.Batch(budget_bytes, max_slots=max_slots, ticks_per_launch=ticks_per_launch, device=device)
    pending = deque(reqs)
    waiting = deque()
    slot_req = {}
    lat, series = [], {}
    updates = 0
    t0 = time.perf_counter()
    try:
        while pending or waiting or slot_req:
            now = time.perf_counter() - t0
            while pending and pending[0]["arrival_s"] <= now:
                waiting.append(pending.popleft())
            while waiting:
                k = _next_index(waiting, policy)
                r = waiting[k]
                slot = batch.admit(r)
                if slot is None:
                    if not slot_req:
                        raise lbm.LbmError(f"request {r.get('id')} does not fit an empty batch")
                    break
                del waiting[k]
                slot_req[slot] = r
            if not slot_req:
                if pending:
                    _wait_until(t0, pending[0]["arrival_s"])
                continue
            batch.run(launches_per_round)
            for slot in batch.poll():
                r = slot_req.pop(slot)
                ft = batch.force_torque(slot, "static")
                done = time.perf_counter() - t0
                lat.append(done - r["arrival_s"])
                updates += cells(r) * int(r["steps"])
                if keep_series:
                    series[r.get("id", len(series))] = ft
                batch.release(slot)
        makespan = time.perf_counter() - t0
    finally:
        batch.close()
    return _summary(lat, makespan, updates, len(reqs)), series


def serve_sequential(trace, device: int = 0, keep_series: bool = False, policy: str = "fifo"):
    """One solve at a time."""
    import torch
    pending = deque(sorted(trace, key=lambda r: r["arrival_s"]))
    n_req = len(pending)
    waiting = []
    lat, series = [], {}
    updates = 0
    t0 = time.perf_counter()
    while pending or waiting:
        now = time.perf_counter() - t0
        while pending and pending[0]["arrival_s"] <= now:
            waiting.append(pending.popleft())
        if not waiting:
            _wait_until(t0, pending[0]["arrival_s"])
            continue
        r = waiting.pop(_next_index(waiting, policy))
        dom = lbm.Domain(r, device=device, series_capacity=int(r["steps"]))
        try:
            dom.step(int(r["steps"]))
            ft = dom.force_torque("static")
        finally:
            dom.close()
        done = time.perf_counter() - t0
        lat.append(done - r["arrival_s"])
        updates += cells(r) * int(r["steps"])
        if keep_series:
            series[r.get("id", len(series))] = ft
    torch.cuda.synchronize(device)
    makespan = time.perf_counter() - t0
    return _summary(lat, makespan, updates, n_req), series


def main(argv=None):
    """python -m paper_1407_4524_gb300.serving: run the seeded serving trace."""
    import argparse
    import json

    from .workloads import serving_trace
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--requests", type=int, default=40)
    ap.add_argument("--rate", type=float, default=20.0, help="mean arrivals per second")
    ap.add_argument("--mode", choices=["batched", "sequential", "both"], default="both")
    ap.add_argument("--slots", type=int, default=256)
    ap.add_argument("--ticks", type=int, default=32, help="steps per graph replay")
    ap.add_argument("--budget-gb", type=float, default=64.0)
    ap.add_argument("--precision", default="fp16", choices=["fp32", "fp16"])
    ap.add_argument("--policy", default="fifo", choices=["fifo", "sjf"], help="queue order")
    args = ap.parse_args(argv)
    trace = serving_trace(n_requests=args.requests, rate_hz=args.rate, precision=args.precision)
    out = {"policy": args.policy}
    if args.mode in ("batched", "both"):
        out["batched"], _ = serve_batched(trace, int(args.budget_gb * (1 << 30)), max_slots=args.slots,
                                          ticks_per_launch=args.ticks, policy=args.policy)
    if args.mode in ("sequential", "both"):
        out["one_at_a_time"], _ = serve_sequential(trace, policy=args.policy)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
