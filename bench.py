#!/usr/bin/env python3
"""Benchmark of the fused LBM step with curved-wall links and momentum exchange.

Workload (default): D3Q19 periodic box 512x256x256, tau 0.6, fluid at rest,
64 spheres of radius U[6,12] (seed 1407): even index static, odd index
translating (|U| <= 0.02) and rotating (|W| <= 0.001); FP32 arithmetic with
populations stored as f - w in FP32; per-body force and torque every step;
cut-link lists and covered/uncovered sets rebuilt every step for the moving
bodies.  One "step" is the whole path: geometry of the moving bodies, wall
values + momentum exchange on every cut link, stream-collide of every cell,
impulsive terms / refill, per-body reduction.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead, on a bounded sample of the same workload.
Multi-GPU (torchrun): independent replicas, one per GPU (the path has no
exchange step between solves); value = all cells updated / max rank time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

if "OMP_NUM_THREADS" not in os.environ:
    os.environ["OMP_NUM_THREADS"] = str(os.cpu_count() or 1)

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

L2_BYTES = 129e6  # GB300 L2 (the larger-than-L2 test of the timing rules)
METRIC = "D3Q19 MLUPS + %HBM roofline w/ fused ME force; served-solve p50/p99 latency"
FALLBACK_HBM_GBS = 6800.0


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def _workload(name: str, precision: str, n=None, bodies=None):
    from paper_1407_4524_gb300 import workloads as W
    if name == "sphere_swarm_3d":
        if n is not None:
            return W.sphere_swarm_3d(precision=precision, n=n, n_bodies=bodies if bodies is not None else 64)
        return W.sphere_swarm_3d(precision=precision)
    if name == "sphere_channel_3d":
        return W.sphere_channel_3d(precision=precision)
    if name == "moving_cylinders_2d":
        return W.moving_cylinders_2d(precision=precision)
    if name == "channel_cylinder_2d":
        return W.channel_cylinder_2d(precision=precision)
    if name == "sedimenting_disc_2d":
        return W.sedimenting_disc_2d(precision=precision)
    if name == "sedimenting_ellipse_2d":
        return W.sedimenting_ellipse_2d(precision=precision)
    raise SystemExit(f"unknown workload {name}")


def _describe(spec) -> str:
    n = "x".join(str(v) for v in spec["n"])
    nb = len(spec.get("bodies", []))
    nm = sum(1 for b in spec.get("bodies", []) if any(np.abs(b.get("U", (0, 0, 0)))) or
             any(np.atleast_1d(b.get("W", 0.0))))
    return f"{spec['name']} {spec['lattice']} {n}, tau {spec['tau']}, {nb} bodies ({nm} moving)"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _barrier_max(x: float, world: int, device: str = "cuda"):
    """max of x over the ranks (NCCL on the GPU, gloo on the CPU)"""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_mlups(ms_local: float, cells: int, steps: int, world: int, device: str = "cuda"):
    """Replicas: every rank advances its own copy of the workload; the job
    time is the slowest rank's, the work is all ranks' cell updates."""
    ms = _barrier_max(ms_local, world, device)
    return ms, world * cells * steps / (ms * 1e-3) / 1e6


def cpu_baseline(spec, budget_s: float = 15.0):
    """The FP64 oracle as it stands, on a bounded sample of the workload: a
    periodic sub-box with the same lattice, tau and body density."""
    import oracle
    from paper_1407_4524_gb300 import workloads as W
    if spec["lattice"] == "D3Q19" and spec["name"] == "sphere_swarm_3d":
        sample = W.sphere_swarm_3d(precision="fp64", n=(128, 96, 96), n_bodies=2, seed=1407)
        desc = "periodic 128x96x96 sub-box, 2 spheres (1 moving), same tau / radii / speeds"
    else:
        sample = dict(spec)
        desc = "the full workload"
    o = oracle.Oracle(sample)
    cells = int(np.prod(o.shape))
    o.step(1)  # warm-up
    t0 = time.perf_counter()
    steps = 0
    while True:
        o.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or steps >= 200:
            break
    mlups = cells * steps / el / 1e6
    return {"value": round(mlups, 3), "unit": "MLUPS", "cores": oracle.threads(),
            "kind": "oracle", "sample": f"{desc}; {steps} steps, {el:.1f} s, FP64"}


def run_reference(args):
    world, rank, local = _dist()
    if rank != 0:
        return
    spec = _workload(args.workload, "fp64", args.n, args.bodies)
    import oracle
    from paper_1407_4524_gb300 import workloads as W
    budget = 150.0
    if args.workload == "sphere_swarm_3d":
        # size a periodic sub-box so that W + K oracle steps take a few minutes at most
        probe = W.sphere_swarm_3d(precision="fp64", n=(64, 64, 64), n_bodies=1, seed=1407)
        o = oracle.Oracle(probe)
        t0 = time.perf_counter()
        o.step(2)
        rate = 2 * 64 ** 3 / (time.perf_counter() - t0)  # cell updates per second
        cells_per_step = max(32 ** 3, min(512 * 256 * 256, rate * budget / max(1, args.steps + args.warmup)))
        nz = max(32, int(round((cells_per_step / 4) ** (1 / 3) / 8)) * 8)
        n = (4 * nz, nz, nz) if 4 * nz <= 512 else (512, min(256, nz), min(256, nz))
        nbod = max(1, int(round(64 * np.prod(n) / (512 * 256 * 256))))
        sample = W.sphere_swarm_3d(precision="fp64", n=n, n_bodies=nbod, seed=1407)
        what = f"periodic {'x'.join(map(str, n))} sub-box of the workload, {nbod} spheres"
        steps, warmup = args.steps, args.warmup
    else:
        # the whole domain; the step count is cut so that the run stays within the budget
        sample = spec
        n = tuple(spec["n"])
        o = oracle.Oracle(sample)
        t0 = time.perf_counter()
        o.step(1)
        per_step = time.perf_counter() - t0
        total = max(1, min(args.steps + args.warmup, int(budget / max(per_step, 1e-9))))
        warmup = min(args.warmup, max(0, total - 1))
        steps = max(1, total - warmup)
        what = f"the whole {'x'.join(map(str, n))} domain, {steps} timed steps"
    o = oracle.Oracle(sample)
    cells = int(np.prod(o.shape))
    o.step(warmup)
    t0 = time.perf_counter()
    o.step(steps)
    el = time.perf_counter() - t0
    mlups = cells * steps / el / 1e6
    cores = oracle.threads()  # the threads the oracle's loops really run on
    line = {
        "impl": "reference", "metric": METRIC, "value": round(mlups, 3), "unit": "MLUPS", "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": round(1e3 * el / max(1, steps), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": _describe(spec), "sample": what, "parallelism": "cpu"},
        "cpu_baseline": {"value": round(mlups, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": what},
        "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _device_timed(spec, args, dev, world, stream, sampler=None):
    """Build the domain, run exactly `warmup` untimed steps (stream-collide
    timing events on), then time `steps` steps between CUDA events on the
    launching stream.  Returns the open domain and the figures."""
    import torch
    from paper_1407_4524_gb300 import lbm
    dom = lbm.Domain(spec, device=dev, stream=stream, series_capacity=max(8192, args.steps + args.warmup + 16))
    # warm-up: exactly `warmup` steps, with the stream-collide kernel's timing
    # events already on.  The library replays captured 16-step graphs for runs
    # of >= 16 steps; the graph (with its timing events) is recorded here,
    # after the first warm-up step, outside the timed region.
    dom.set_kernel_timing(True)
    dom.step(1)
    dom.prepare_graph()
    dom.step(args.warmup - 1)
    torch.cuda.synchronize()
    dom.kernel_time()  # discard the warm-up windows
    if sampler:
        sampler.start()
        time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    dom.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    n_bulk, bulk_ms = dom.kernel_time()
    dom.set_kernel_timing(False)
    clocks = sampler.stop() if sampler else None
    ms, mlups = replica_mlups(ms, dom.N, args.steps, world)
    return dom, dict(ms=ms, mlups=mlups, n_bulk=n_bulk, bulk_ms=bulk_ms, clocks=clocks,
                     launches_per_step=dom.launches_per_step())


def _roofline(args, precision, dom, fluid_cells, n_bulk, bulk_ms):
    """roofline object of the stream-collide kernel: algorithmic bytes (one
    read and one write of Q stored values per fluid node) over its mean
    CUDA-event window, against the measured copy bandwidth"""
    peak, peak_kind = _peaks()
    sbytes = {"fp64": 8, "fp32": 4, "fp16": 2}[precision]
    bulk_avg_s = bulk_ms * 1e-3 / max(1, n_bulk)
    alg_bytes = 2.0 * dom.q * sbytes * fluid_cells
    achieved = alg_bytes / bulk_avg_s / 1e9
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(tpath) as fh:
            tj = json.load(fh)
        key = f"{args.workload}:{precision}"
        if key in tj and tj[key].get("kernel_rev") == _kernel_rev():
            traffic = tj[key]["bytes_per_launch"]
    except Exception:
        traffic = None
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": traffic, "peak_kind": peak_kind,
            "kernel": "k_bulk (pull-stream + BGK collide)", "kernel_ms": round(bulk_avg_s * 1e3, 4),
            "alg_bytes_per_launch": int(alg_bytes)}


def run_ours(args):
    import torch
    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    spec = _workload(args.workload, args.precision, args.n, args.bodies)
    stream = torch.cuda.Stream(dev)
    sampler = ClockSampler(dev) if rank == 0 else None
    dom, m = _device_timed(spec, args, dev, world, stream, sampler)
    cells = dom.N
    fluid_cells = dom.stats()["fluid_cells"]
    ms, mlups, clocks = m["ms"], m["mlups"], m["clocks"]
    launches_per_step = m["launches_per_step"]

    # end-to-end through the C ABI with host buffers: each step uploads the
    # bodies' kinematics (lbm_update_bodies: host array -> pinned staging ->
    # device) and reads the step's force/torque row back (lbm_get_force_torque)
    bodies = list(dom.bodies)
    nb = len(bodies)
    out = np.zeros((1, max(nb, 1), 6))
    e2e_steps = max(10, min(args.steps, 200))
    s0 = dom.stats()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    has_free = any(b.get("free", False) for b in bodies)
    t_first = dom.t
    t0 = time.perf_counter()
    # pipelined: the row of step k is read after step k+1 is enqueued, so the
    # host's read overlaps the GPU's next step; every row is read in the
    # timed region
    for _ in range(e2e_steps):
        if not has_free:  # free bodies take their kinematics from the flow: nothing to upload
            dom.update_bodies(bodies)
        dom.step(1)
        if dom.t >= 2 and dom.t - 2 >= t_first:
            dom.lib.lbm_get_force_torque(dom.h, dom.t - 2, 1, 0, out.ctypes.data)
    dom.lib.lbm_get_force_torque(dom.h, dom.t - 1, 1, 0, out.ctypes.data)
    torch.cuda.synchronize()
    e2e_s = _barrier_max(time.perf_counter() - t0, world)
    s1 = dom.stats()
    e2e = {"value": round(world * cells * e2e_steps / e2e_s / 1e6, 1), "unit": "MLUPS",
           "h2d_bytes_per_step": int((s1["h2d_bytes"] - s0["h2d_bytes"]) / e2e_steps),
           "d2h_bytes_per_step": int((s1["d2h_bytes"] - s0["d2h_bytes"]) / e2e_steps)}
    roofline = _roofline(args, args.precision, dom, fluid_cells, m["n_bulk"], m["bulk_ms"])
    # the bulk kernel's mean window over the mean step (the windows measured
    # cover the plain steps and the last graph replay, not every step)
    step_frac = (roofline["kernel_ms"] / max(1e-9, ms / args.steps)) if world == 1 else None
    dom.close()

    # the same workload with FP16 storage of f - w: its own device-timed run
    # (same steps and warm-up), reported beside the main line
    fp16 = None
    if args.precision == "fp32" and not args.no_fp16:
        spec16 = _workload(args.workload, "fp16", args.n, args.bodies)
        sampler16 = ClockSampler(dev) if rank == 0 else None
        dom16, m16 = _device_timed(spec16, args, dev, world, stream, sampler16)
        fc16 = dom16.stats()["fluid_cells"]
        fp16 = dict(value=round(m16["mlups"], 1), ms_per_step=round(m16["ms"] / args.steps, 4),
                    roofline=_roofline(args, "fp16", dom16, fc16, m16["n_bulk"], m16["bulk_ms"]),
                    clocks=m16["clocks"], launches_per_step=m16["launches_per_step"])
        dom16.close()

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    serving = run_serving(args, dev) if (world == 1 and args.serving_requests > 0) else None
    cpu = cpu_baseline(spec, budget_s=args.cpu_budget) if (world == 1 and not args.no_cpu) else None
    sbytes = {"fp64": 8, "fp32": 4, "fp16": 2}[args.precision]
    pop_bytes = 2 * dom.q * sbytes * cells
    line = {
        "metric": METRIC, "value": round(mlups, 1), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
        "data": "synthetic",
        "config": {"workload": _describe(spec), "cells": cells, "fluid_cells": fluid_cells,
                   "precision": args.precision + (" (f - w stored)" if args.precision != "fp64" else ""),
                   "l2": (("inputs larger than L2 (populations %.2f GB)" % (pop_bytes / 1e9)) if pop_bytes > L2_BYTES
                          else ("inputs fit in L2 (populations %.1f MB), steps back to back without a flush: "
                                "an L2-resident figure, not an HBM one" % (pop_bytes / 1e6))),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "bulk_share_of_step": round(step_frac, 4) if step_frac else None},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": int(launches_per_step * args.steps), "clocks": clocks,
    }
    if fp16:
        # FP16 storage (FP32 arithmetic): whole-job MLUPS of the same workload
        line["value_fp16"] = fp16["value"]
        line["ms_per_step_fp16"] = fp16["ms_per_step"]
        line["roofline_fp16"] = fp16["roofline"]
        line["clocks_fp16"] = fp16["clocks"]
        line["gpu_launches_fp16"] = int(fp16["launches_per_step"] * args.steps)
    line["serving"] = serving
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_serving(args, dev):
    """The serving stream: Poisson arrivals (20 req/s, seed 4524) of D2Q9 and
    D3Q19 channel solves of uneven sizes, FP32 arithmetic with FP16 f - w
    storage, run in real time twice on the same GPU: continuous batching
    (lbm_batch_*) and one solve at a time (lbm_step per solve), with first-come
    first-served queues and again with smallest-work-first queues.
    Latency = completion (series back on the host) - arrival."""
    from paper_1407_4524_gb300 import serving
    from paper_1407_4524_gb300 import workloads as W
    trace = W.serving_trace(n_requests=args.serving_requests, precision="fp16")
    free, _ = __import__("torch").cuda.mem_get_info(dev)
    budget = int(min(64 << 30, 0.5 * free))
    def rnd(d):
        return {k: (round(v, 4) if isinstance(v, float) else v) for k, v in d.items()}

    batched, _ = serving.serve_batched(trace, budget_bytes=budget, max_slots=args.serving_slots, ticks_per_launch=32,
                                       device=dev)
    seq, _ = serving.serve_sequential(trace, device=dev)
    # the same trace with smallest-work-first queues, for both loops (fewer
    # resident solves suit this order: the small ones are not slowed by sharing)
    sjf_b = {}
    for slots in (8,):
        sjf_b[slots], _ = serving.serve_batched(trace, budget_bytes=budget, max_slots=slots, ticks_per_launch=32,
                                                device=dev, policy="sjf")
    sjf_s, _ = serving.serve_sequential(trace, device=dev, policy="sjf")
    return {
        "trace": f"{len(trace)} requests, Poisson 20/s (seed 4524), D2Q9 {{128x64..1024x512}} / "
                 f"D3Q19 {{64^3..192x96x96}}, 2000-20000 steps, fp16 storage",
        "budget_bytes": budget,
        "slots": args.serving_slots,
        "batched": rnd(batched),
        "one_at_a_time": rnd(seq),
        "sjf": {"batched_by_slots": {str(k): rnd(v) for k, v in sjf_b.items()}, "one_at_a_time": rnd(sjf_s)},
        "mlups_ratio": round(batched["mlups"] / seq["mlups"], 3) if seq["mlups"] else None,
        "p50_s": round(batched["p50_s"], 4), "p99_s": round(batched["p99_s"], 4),
    }


# the sources that define the stream-collide kernel and its launch (the
# kernel the traffic figure belongs to)
BULK_SOURCES = ("lbm_dev.cuh", "lbm_step.cuh", "lbm_pair.cuh", "lbm_launch.cuh", "lbm_stage.cuh", "lbm_fp32.cu",
                "lbm_fp64.cu")


def _kernel_rev() -> str:
    """hash of the stream-collide kernel's sources the traffic figure was taken
    on (code only: comments and blank lines do not change it)"""
    import hashlib
    import re
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_1407_4524_gb300", "csrc")
    for f in BULK_SOURCES:
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        code = "\n".join(line.rstrip() for line in text.splitlines() if line.strip())
        h.update(code.encode())
    return h.hexdigest()[:12]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sphere_swarm_3d")
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "fp16"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp16", action="store_true", help="skip the FP16-storage run beside an FP32 one")
    ap.add_argument("--print-kernel-rev", action="store_true")
    ap.add_argument("--n", default=None, help="override the box size, e.g. 256,256,128 (profiling cases)")
    ap.add_argument("--bodies", type=int, default=None)
    ap.add_argument("--serving-requests", type=int, default=200,
                    help="requests of the serving trace (0: skip the serving measurement)")
    ap.add_argument("--serving-slots", type=int, default=16,
                    help="resident solves at most in the FIFO batched serving run")
    args = ap.parse_args()
    if args.n:
        args.n = tuple(int(v) for v in args.n.split(","))
    if args.print_kernel_rev:
        print(_kernel_rev())
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
