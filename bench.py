"""Benchmark of the coupled LBM-MEM step (MLUPS and fraction of the HBM roofline).

Default workload: a periodic 512^3 D3Q19 TRT box with one light sphere
(d = 40 cells, pi_p = 0.5, Ga = 200 at u_g = 0.01, C_v = 0.5), FP32
deviation storage, the full coupled step of Algorithm 1 per timed step.
The field (20.4 GB in FP32) is far larger than L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp16|fp64]
  python bench.py --impl reference ...   # the FP64 oracle on the host cores

Prints one JSON line on rank 0.  With torchrun (N > 1) every rank runs an
independent replica on its own GPU (weak scaling, no collective on the data
path); the time is the max over ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS of coupled LBM-MEM step (FP32/FP16 vs FP64) and % of HBM roofline"
BYTES_PER_POP = {"fp64": 8, "fp32": 4, "fp16": 2}
DTYPE = {"fp64": "f64", "fp32": "f32", "fp16": "f16-storage/f32-math"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "fp64"])
    ap.add_argument("--edge", type=int, default=512)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def workload(args):
    from paper_2103_10882_gb300 import workloads
    w = dict(workloads.ROOFLINE_512)
    e = args.edge
    w["shape"] = (e, e, e)
    return w


def workload_name(args):
    e = args.edge
    return "uniform %d^3 periodic D3Q19 TRT, 1 sphere d=40 pi_p=0.5 Ga=200 C_v=0.5, coupled step" % e


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profiled_traffic(args):
    """DRAM bytes per k_bulk launch from the committed ncu summary (captured
    at 256^3 and scaled by the cells processed); None when the summary does
    not exist or the kernel source changed since the capture."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "k_bulk_%s_uniform256.md" % args.precision)
    if args.edge != 512 or not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if ":" in line and line.strip().split(":")[0] in ("source_sha256_16", "traffic_bytes_per_launch_512"):
            k, v = line.strip().split(":", 1)
            fields[k] = v.strip()
    src = os.path.join(ROOT, "paper_2103_10882_gb300", "csrc", "uniform.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if fields.get("source_sha256_16") != sha:
        return None
    try:
        return int(fields["traffic_bytes_per_launch_512"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
                for nm, v in zip(names, r[4:8]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(args, w, seconds):
    """The FP64 oracle on the host cores, on a bounded sample of the same
    workload: a periodic slab of the same box (full x-y extent, 48 layers)
    through the sphere, same tau, sphere and gravity."""
    import numpy as np

    import oracle
    from paper_2103_10882_gb300 import workloads
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    e = w["shape"][0]
    shape = (e, e, 48)
    D, pi = w["diameter"], w["density_ratio"]
    nu = w["u_g"] * D / w["ga"]
    tau = 3 * nu + 0.5
    gm = w["u_g"] ** 2 / (abs(pi - 1) * D)
    o = oracle.UniformSim(shape, tau=tau)
    pos = np.array([e / 2, e / 2, 24.0]) + workloads.sub_cell_offset(0)
    o.add_sphere(pos, D, pi, cv=w["cv"])
    o.set_gravity((0, 0, -gm))
    o.init_equilibrium()
    ncells = shape[0] * shape[1] * shape[2]
    t0 = time.perf_counter()
    steps = 0
    while True:
        o.step(1)
        steps += 1
        dt = time.perf_counter() - t0
        if dt >= seconds:
            break
    o.close()
    return {"value": ncells * steps / dt / 1e6, "unit": "MLUPS", "cores": threads, "kind": "oracle",
            "sample": "%dx%dx%d periodic slab through the sphere, %d steps, %.1f s" % (shape + (steps, dt))}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = workload(args)
    per = max(args.cpu_seconds / max(args.steps, 1), 1.0)
    cb = cpu_baseline(args, w, per * max(args.steps, 1))
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(args), "precision": "fp64 oracle"},
            "cpu_baseline": cb, "e2e": {"value": cb["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch

    import paper_2103_10882_gb300 as L
    from paper_2103_10882_gb300 import workloads

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    w = workload(args)
    shape, D, pi = w["shape"], w["diameter"], w["density_ratio"]
    sim = L.Simulation(shape, precision=args.precision)
    pos = np.array(shape, dtype=float) / 2 + workloads.sub_cell_offset(rank)
    pos[2] = 0.25 * shape[2] + workloads.sub_cell_offset(rank)[2]
    sim.add_sphere(pos, D, pi, cv=w["cv"])
    sim.set_ga(w["ga"], w["u_g"], (0.0, 0.0, -1.0))
    sim.init_fluid()
    ncells = sim.ncells

    # warm-up
    sim.step(args.warmup)
    torch.cuda.synchronize()
    stream = sim.stream
    c0 = sim.counters()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        sim.profile(True)
        start.record(stream)
        sim.step_async(args.steps)
        stop.record(stream)
        torch.cuda.synchronize()
    sim.check()
    ms = start.elapsed_time(stop)
    bulk_ms, bulk_n, _, _ = sim.profile_result()
    sim.profile(False)
    c1 = sim.counters()
    launches = int(c1[2] - c0[2])
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = world * ncells * args.steps / (ms_max * 1e-3) / 1e6

    # end to end through the public API with host buffers: each step uploads
    # the gravity vector (host array), advances one step (status read back)
    # and reads the particle record into a host array
    g_host = np.array([0.0, 0.0, -(w["u_g"] ** 2) / (abs(pi - 1) * D)])
    e0 = sim.counters()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        sim.set_gravity(g_host)
        sim.step(1)
        rec = sim.particle()
    t1 = time.perf_counter()
    e1 = sim.counters()
    e2e_value = ncells * args.e2e_steps / (t1 - t0) / 1e6
    h2d = (e1[3] - e0[3]) / args.e2e_steps
    d2h = (e1[4] - e0[4]) / args.e2e_steps
    assert np.all(np.isfinite(rec))

    bpp = BYTES_PER_POP[args.precision]
    alg_bytes = 2 * 19 * bpp * ncells
    bulk_avg_s = bulk_ms / max(bulk_n, 1) * 1e-3
    achieved = alg_bytes / bulk_avg_s / 1e9
    peak, peak_kind = measured_peaks()
    traffic = profiled_traffic(args)

    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
        "config": {"workload": workload_name(args), "cells": ncells, "precision": args.precision,
                   "l2": "inputs larger than L2 (%.1f GB field)" % (2 * alg_bytes / 2 / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "kernel": "k_bulk (stream + TRT collide, %s)" % args.precision,
                     "peak_kind": peak_kind, "bytes_per_cell_update": 2 * 19 * bpp},
        "e2e": {"value": e2e_value, "unit": "MLUPS", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": args.e2e_steps},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "step_ms_breakdown": {"bulk_ms_avg": bulk_ms / max(bulk_n, 1), "step_ms_avg": ms_max / args.steps},
    }
    sim.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, w, args.cpu_seconds)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
