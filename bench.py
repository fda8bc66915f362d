"""Benchmark of the coupled LBM-MEM step: MLUPS and fraction of the HBM roofline.

Default workload (the single rising light sphere on a refined grid): level-0
box of 64 x 64 x 256 cells in 16^3 blocks, 3 levels (finest 256 x 256 x
1024), sphere of 20 finest cells, density ratio 0.5, Ga = 200 at u_g = 0.01,
C_v = 0.5, no-slip walls on x and y, periodic z, regrid every 50 level-0
steps with the particle criterion and the flow-based curl sensor (Sec.
4.2.2: sigma_c = 1e-3, c = 0.2), FP32 deviation storage.  A timed step is one level-0 step of the full
coupled method (Algorithm 1 on the finest level, sub-cycling, explosion and
coalescence, regrids when due).  MLUPS counts real cell updates of all levels.
The headline value is a window of --steps level-0 steps of the developed run
(from level-0 step 2000 on, the wake has grown the finest level) placed so
that it holds one regrid; the line also carries the first steps from rest
(cold_start), a long developed window (developed_long, one regrid per 50
steps) and the same developed window in FP16 storage and FP64.

Also reported (key "uniform512"): a periodic 512^3 box with a sphere of 40
cells, the bandwidth case of the stream-collide kernel; "uniform512_mrt" is
the same case with the paper's MRT collision (bulk factor 100).  Both fields are far
larger than L2 (no flush needed).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp16|fp64]
  python bench.py --impl reference ...   # the FP64 oracle on the host cores

Prints one JSON line on rank 0.  With torchrun (N > 1) every rank runs an
independent replica on its own GPU (weak scaling, no collective on the data
path); the time is the max over ranks.
"""
import argparse
import hashlib
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

REFINED = dict(shape=(64, 64, 256), levels=3, diameter=20.0, density_ratio=0.5, ga=200.0, u_g=0.01, cv=0.5,
               bc=("noslip", "noslip", "periodic"), regrid=50, sensor=(1e-3, 0.2))
UNIFORM = dict(shape=(512, 512, 512), diameter=40.0, density_ratio=0.5, ga=200.0, u_g=0.01, cv=0.5)
# the large refined case: FP16 storage against FP64 on terminal velocity and lateral drift (seeded start offset
# and a lateral velocity perturbation of 1e-3 u_g in a seeded direction)
LARGE = dict(shape=(128, 128, 512), levels=4, diameter=40.0, density_ratio=0.1, ga=300.0, u_g=0.01, cv=0.5,
             bc=("noslip", "noslip", "periodic"), regrid=50, sensor=(1e-3, 0.2), perturbation=1e-3, seed=1)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100, help="timed level-0 steps of the refined workload")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "fp64"])
    ap.add_argument("--workload", default="refined", choices=["refined", "uniform"])
    ap.add_argument("--edge", type=int, default=512, help="edge of the uniform bandwidth case")
    ap.add_argument("--uniform-steps", type=int, default=30)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--long-steps", type=int, default=1000,
                    help="level-0 steps of the long developed window of the headline workload (FP32 line)")
    ap.add_argument("--cuda-profiler-window", action="store_true",
                    help="bracket the developed window of the headline precision with cudaProfilerStart/Stop (for "
                         "ncu --profile-from-start off)")
    ap.add_argument("--no-other-precisions", action="store_true",
                    help="skip the FP16-storage and FP64 windows of the headline workload")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-uniform", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-mrt", action="store_true", help="skip the MRT (bulk factor 100) variant of the uniform case")
    ap.add_argument("--batch-steps", type=int, default=20)
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--validate", type=int, default=0,
                    help="instead of timing: run the refined workload this many level-0 steps in FP64, FP32 and FP16 "
                         "and report the reduced precisions' errors on the particle's path")
    ap.add_argument("--adjoint-reps", type=int, default=3)
    ap.add_argument("--validate-workload", default="refined", choices=["refined", "large"],
                    help="workload of --validate: the headline refined case or the large FP16 case")
    ap.add_argument("--rotation", action="store_true",
                    help="instead of timing: the rotating virtual-mass test (Sec. 3.4, Table 3) and one JSON line")
    ap.add_argument("--stability", action="store_true",
                    help="instead of timing: the stability-limit study (lowest stable density ratio per diameter at "
                         "Ga = 100, plain MEM and virtual mass) and one JSON line")
    return ap.parse_args()


REFINED_NAME = ("refined rising sphere: level-0 64x64x256 (16^3 blocks), 3 levels, d=20 finest, pi_p=0.5, Ga=200, "
                "C_v=0.5, walls x/y, periodic z, regrid every 50 level-0 steps (particle + curl sensor sigma_c=1e-3, "
                "c=0.2)")
# The paper's only performance figures (Table 4, CPU, context only: another machine, method, workload and metric):
# the uniform-grid rising sphere at d_p = 100 on SuperMUC-NG took 10.27 h on 36,864 processes for about 3.6e5 finest
# steps of 3.06e9 cells (derived: about 29.8 GLUPS in total, 0.81 MLUPS per process); the adaptive run took 6.58 h
# on 768 processes with 3.78e7 cells on average.
PAPER_CONTEXT = {"source": "Table 4 (SuperMUC-NG, MPI CPU processes)",
                 "uniform_grid": {"processes": 36864, "cells": 3.06e9, "hours": 10.27,
                                  "derived_glups_total": 29.8, "derived_mlups_per_process": 0.81},
                 "adaptive_grid": {"processes": 768, "mean_cells": 3.78e7, "hours": 6.58}}
# level-0 step from which the run counts as developed: the wake has grown the finest level (3.3 -> 4-5 M
# cell updates per level-0 step) and regrids change the hierarchy
DEVELOPED_STEP = 2000


def uniform_name(edge, prec):
    return "uniform %d^3 periodic, 1 sphere d=40 pi_p=0.5 Ga=200 C_v=0.5, %s" % (edge, prec)


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profiled_traffic(name, scale_cells):
    """DRAM bytes per launch of a kernel from a committed ncu summary
    (fields traffic_bytes_per_launch_* and source_sha256_16 of its source
    file); None if absent or the source changed since the capture."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if ":" in line:
            k, v = line.strip().split(":", 1)
            fields[k.strip()] = v.strip()
    src = os.path.join(ROOT, "paper_2103_10882_gb300", "csrc", fields.get("source_file", "uniform.cu"))
    if not os.path.exists(src):
        return None
    if fields.get("source_sha256_16") != hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]:
        return None
    try:
        return int(fields[scale_cells])
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
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
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


def ga_tau_g(ga, u_g, d, pi):
    nu = u_g * d / ga
    return 3 * nu + 0.5, u_g ** 2 / (abs(pi - 1) * d)


def refined_start(shape, levels, d, seed=0):
    f = 1 << (levels - 1)
    from paper_2103_10882_gb300 import workloads
    off = workloads.sub_cell_offset(seed)
    # lateral centre, 0.6 d above the bottom (finest units)
    return (shape[0] * f / 2 + off[0], shape[1] * f / 2 + off[1], 0.6 * d + off[2])


def refined_sim(L, prec, history_capacity=1 << 16, w=None):
    """A refined rising-sphere workload (the headline one unless w is given)
    through the public API: hierarchy, sphere, gravity from Ga, refinement
    sensor, fluid at rest, and the sphere's seeded lateral perturbation."""
    import math
    from paper_2103_10882_gb300 import workloads
    w = REFINED if w is None else w
    seed = w.get("seed", 0)
    tau, _ = ga_tau_g(w["ga"], w["u_g"], w["diameter"], w["density_ratio"])
    sim = L.Simulation(w["shape"], precision=prec, tau=tau, bc=w["bc"], levels=w["levels"],
                       regrid_interval=w["regrid"], history_capacity=history_capacity)
    sim.add_sphere(refined_start(w["shape"], w["levels"], w["diameter"], seed), w["diameter"], w["density_ratio"],
                   cv=w["cv"])
    sim.set_ga(w["ga"], w["u_g"], (0.0, 0.0, -1.0))
    sim.set_refinement_sensor(*w["sensor"])
    if w.get("perturbation"):
        theta = 2.0 * math.pi * float(workloads.uniform01(seed + 1000, 1)[0])
        v = w["perturbation"] * w["u_g"]
        sim.set_particle_velocity((v * math.cos(theta), v * math.sin(theta), 0.0))
    sim.init_fluid()
    return sim


def cpu_baseline(seconds, max_steps=None, warmup=0):
    """The FP64 refined oracle on the host cores, on a bounded sample of the
    same workload: the same hierarchy and sphere, `warmup` untimed level-0
    steps (at most one), then timed level-0 steps until `seconds` have passed
    or `max_steps` are done (at least one), first on all host cores (the
    oracle's OpenMP loops, bit-identical results), then on one core for
    half as long."""
    import oracle
    w = REFINED
    tau, gm = ga_tau_g(w["ga"], w["u_g"], w["diameter"], w["density_ratio"])
    cores = os.cpu_count() or 1

    def sample(threads, budget):
        oracle.set_threads(threads)
        o = oracle.RefinedSim(w["shape"], w["levels"], tau=tau, periodic=(0, 0, 1))
        o.add_sphere(refined_start(w["shape"], w["levels"], w["diameter"]), w["diameter"], w["density_ratio"],
                     cv=w["cv"])
        o.set_gravity((0, 0, -gm))
        o.set_sensor(*w["sensor"])
        o.init_equilibrium()
        upd = sum((o.block_map(l) >= 0).sum() * 4096 * (1 << l) for l in range(w["levels"]))
        if warmup > 0:
            o.step(1)
        t0 = time.perf_counter()
        steps = 0
        while True:
            o.step(1)
            steps += 1
            dt = time.perf_counter() - t0
            if dt >= budget or (max_steps is not None and steps >= max_steps):
                break
        o.close()
        return upd * steps / dt / 1e6, steps, dt

    v_all, n_all, t_all = sample(cores, seconds)
    v_one, n_one, t_one = sample(1, 0.5 * seconds)
    oracle.set_threads(cores)
    return {"value": v_all, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "value_1_core": v_one,
            "sample": "refined workload (same hierarchy and sphere): %d level-0 steps in %.1f s on %d threads, "
                      "%d in %.1f s on one" % (n_all, t_all, cores, n_one, t_one)}


def run_reference(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    cb = cpu_baseline(max(args.cpu_seconds, 1.0), max_steps=max(args.steps, 1), warmup=args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f64",
            "data": "synthetic", "config": {"workload": REFINED_NAME}, "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def timed(sim, steps, stream, torch, profile):
    """CUDA events around `steps` steps on the simulation's stream.  With
    profile=True the library also brackets every stream-collide launch with
    events (which keeps the refined engine off its CUDA graphs)."""
    c0 = sim.counters()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if profile:
        sim.profile(True)
    start.record(stream)
    sim.step_async(steps)
    stop.record(stream)
    torch.cuda.synchronize()
    sim.check()
    ms = start.elapsed_time(stop)
    prof = None
    if profile:
        prof = sim.profile_result()
        sim.profile(False)
    c1 = sim.counters()
    return ms, prof, c0, c1


def e2e(sim, steps, g_host):
    """Same metric end to end through the C ABI with host buffers: each step
    uploads the gravity vector from a host array, advances one level-0 step
    (reading the status word back) and reads the particle record into a host
    array."""
    import numpy as np
    e0 = sim.counters()
    t0 = time.perf_counter()
    rec = None
    for _ in range(steps):
        sim.set_gravity(g_host)
        sim.step(1)
        rec = sim.particle()
    t1 = time.perf_counter()
    e1 = sim.counters()
    assert np.all(np.isfinite(rec))
    return {"value": (e1[1] - e0[1]) / (t1 - t0) / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": (e1[3] - e0[3]) / steps, "d2h_bytes_per_step": (e1[4] - e0[4]) / steps,
            "steps": steps}


def roofline(prof, kernel, traffic):
    kms, launches, _, _, bytes_, _ = prof
    peak, kind = measured_peak()
    achieved = bytes_ / (kms * 1e-3) / 1e9 if kms > 0 else 0.0
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": kernel, "peak_kind": kind, "launches": int(launches),
            "kernel_ms_total": kms}


def validate(args):
    """The refined rising-sphere workload run for args.validate level-0 steps
    in FP64, FP32 and FP16 storage: rise velocity, lateral drift and
    trajectory of the reduced precisions against the FP64 run, and each run's
    MLUPS (one JSON line)."""
    import numpy as np
    import torch
    import paper_2103_10882_gb300 as L
    w = LARGE if args.validate_workload == "large" else REFINED
    runs = {}
    for prec in ("fp64", "fp32", "fp16"):
        sim = refined_sim(L, prec, history_capacity=1 << 19, w=w)
        c0 = sim.counters()
        start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        start.record(sim.stream)
        sim.step_async(args.validate)
        stop.record(sim.stream)
        torch.cuda.synchronize()
        sim.check()
        c1 = sim.counters()
        h = sim.history()
        runs[prec] = dict(hist=h, mlups=(c1[1] - c0[1]) / (start.elapsed_time(stop) * 1e-3) / 1e6)
        sim.close()
    ref = runs["fp64"]["hist"]
    d = w["diameter"]
    name = ("large refined case: level-0 128x128x512, 4 levels, d=40, pi_p=0.1, Ga=300, seeded offset and 1e-3 u_g "
            "lateral perturbation" if w is LARGE else "refined rising sphere (headline workload)")
    q = len(ref) // 4   # the last quarter of the finest steps: the terminal mean, less sensitive to path oscillations
    out = {"validate": "%s, %d level-0 steps = %d finest steps" % (name, args.validate, len(ref)),
           "fp64": {"u_z_end": ref[-1, 11], "u_z_mean_last_quarter": float(ref[-q:, 11].mean()), "z_end": ref[-1, 8],
                    "mlups": runs["fp64"]["mlups"]}}
    for prec in ("fp32", "fp16"):
        h = runs[prec]["hist"]
        n = min(len(h), len(ref))
        traj = np.sqrt(((h[:n, 6:9] - ref[:n, 6:9]) ** 2).sum(axis=1))
        lat = np.sqrt((h[n - 1, 6] - h[0, 6]) ** 2 + (h[n - 1, 7] - h[0, 7]) ** 2)
        lat_ref = np.sqrt((ref[n - 1, 6] - ref[0, 6]) ** 2 + (ref[n - 1, 7] - ref[0, 7]) ** 2)
        mean, mref = float(h[n - q:n, 11].mean()), float(ref[n - q:n, 11].mean())
        out[prec] = {"u_z_end": h[n - 1, 11],
                     "u_z_rel_err": abs(h[n - 1, 11] - ref[n - 1, 11]) / abs(ref[n - 1, 11]),
                     "u_z_mean_last_quarter": mean, "u_z_mean_rel_err": abs(mean - mref) / abs(mref),
                     "trajectory_max_err_over_d": float(traj.max() / d),
                     "lateral_drift": float(lat), "lateral_drift_fp64": float(lat_ref),
                     "mlups": runs[prec]["mlups"], "speedup_over_fp64": runs[prec]["mlups"] / runs["fp64"]["mlups"]}
    print(json.dumps(out))
    return 0


def stability_study(args):
    """Lowest stable density ratio per sphere diameter at Ga = 100 (Sec. 3.2,
    Table 1) with the plain momentum exchange method, by bisection in
    log(pi_p), with the paper's collision (MRT, bulk factor 100) and its
    force-oscillation criterion next to the status word; the same with TRT;
    and the virtual-mass correction (C_v = 0.5) at pi_p = 0.001.  The
    paper's Table 1 alongside as context."""
    import paper_2103_10882_gb300 as L
    from paper_2103_10882_gb300 import studies, workloads
    table = {10: 0.13, 15: 0.09, 20: 0.066, 30: 0.045, 40: 0.034}   # Table 1 of the paper (context)
    prec = args.precision
    out = {"study": "stability limit of light rising spheres, Ga=100, u_g=0.01, box (6.4, 6.4, 12.8) d_p, "
                    "stable = neither the force-oscillation criterion (step-to-step change of the hydrodynamic force "
                    "above 100 |F_g|) nor the status word trips before t_n = 10", "precision": prec,
           "mem_mrt100": {}, "mem_trt": {}, "vm_mem": {}}
    t0 = time.time()
    for d in workloads.STABILITY["diameters"]:
        for key, bulk in (("mem_mrt100", 100.0), ("mem_trt", 1.0)):
            s, u, runs = studies.density_ratio_limit(L, d, 0.0, table[d] / 4, table[d] * 4, iters=4, precision=prec,
                                                     bulk=bulk)
            trip = [dict(pi=r["density_ratio"], t_n_force=r["t_n_force"], t_n_status=r["t_n_status"]) for r in runs
                    if not r["stable"]]
            out[key][str(d)] = {"pi_min": s, "highest_unstable": u, "paper_table1": table[d], "runs": len(runs),
                                "unstable_runs": trip}
        r = studies.rising_sphere_run(L, d, 0.001, 0.5, precision=prec)
        out["vm_mem"][str(d)] = {"density_ratio": 0.001, "stable": r["stable"], "u_z_over_u_g": r["u_z_over_u_g"]}
        print("d %d: MEM (MRT 100) pi_min %s, MEM (TRT) %s (paper %.3f); VM-MEM at 0.001 stable %s"
              % (d, out["mem_mrt100"][str(d)]["pi_min"], out["mem_trt"][str(d)]["pi_min"], table[d], r["stable"]),
              file=sys.stderr, flush=True)
    out["seconds"] = time.time() - t0
    print(json.dumps(out))
    return 0


def rotation_study(args):
    """The rotating virtual-mass test (Sec. 3.4, Table 3): omega_n over t_n
    for pi_p = 0.1 and 1.1 with MEM and VM-MEM (C_v = 0.5), and pi_p = 0.001
    with both; the mean and terminal relative errors of VM-MEM against MEM
    (Table 3's measures) and the paper's values alongside as context."""
    import numpy as np
    import paper_2103_10882_gb300 as L
    from paper_2103_10882_gb300 import studies, workloads
    w = workloads.ROTATION
    table3 = {0.1: (0.46e-3, 0.01e-3), 1.1: (0.15e-3, 0.0)}   # Table 3 of the paper (context)
    out = {"study": "rotating sphere with virtual mass: (12.8, 6.4, 4.8) d_p, walls on z, upper wall u_w=0.1, "
                    "Couette start, d_p=%d, Re_p=110, translation held, rotation released after %g t_c, monitored "
                    "for %g t_c" % (w["diameter"], w["develop_tc"], w["monitor_tc"]), "precision": args.precision,
           "runs": {}}
    t0 = time.time()
    runs = {}
    for pi in w["density_ratios"]:
        for name, cv in (("mem", 0.0), ("vm_mem", 0.5)):
            r = studies.rotating_sphere_run(L, pi, cv, precision=args.precision)
            runs[(pi, name)] = r
            om = np.asarray(r["omega_n"])
            out["runs"]["%s_%g" % (name, pi)] = {
                "stable": r["stable"], "samples": len(om), "omega_n_end": float(om[-1]) if len(om) else None,
                "omega_n_at": {str(t): float(om[int(round(t * r["t_c"] / 10)) - 1]) for t in (0.5, 1, 2, 4, 8)
                               if len(om) >= int(round(t * r["t_c"] / 10))}}
            print("pi_p %g %s: stable %s, omega_n end %s" % (pi, name, r["stable"], out["runs"]["%s_%g" % (name, pi)]["omega_n_end"]),
                  file=sys.stderr, flush=True)
    out["errors_vm_vs_mem"] = {}
    for pi in (0.1, 1.1):
        if runs[(pi, "mem")]["stable"] and runs[(pi, "vm_mem")]["stable"]:
            mean, term = studies.rotation_errors(runs[(pi, "vm_mem")], runs[(pi, "mem")])
            out["errors_vm_vs_mem"][str(pi)] = {"mean_rel": mean, "terminal_rel": term,
                                                "paper_table3": {"mean_rel": table3[pi][0], "terminal_rel": table3[pi][1]}}
    out["seconds"] = time.time() - t0
    print(json.dumps(out))
    return 0


def adjoint_line(L, workloads, torch, prec, reps):
    """Gradient of the mean drag on the differentiation workload: forward
    (500 steps, checkpoints every 50) and backward (recompute + reverse
    sweep) timed with CUDA events, and the roofline of the reverse-step
    kernel from events around each of its launches."""
    import numpy as np
    c = workloads.ADJOINT_64
    off = workloads.sub_cell_offset(7)
    pos = tuple(0.5 * n + o for n, o in zip(c["shape"], off))
    sim = L.Simulation(c["shape"], precision=prec, tau=c["tau"])
    sim.add_sphere(pos, c["diameter"], 1.0)
    sim.set_fixed(True)
    sim.set_body_force((c["body_force"], 0.0, 0.0))
    dev = torch.device("cuda")
    u0 = torch.tensor(workloads.fourier_velocity_field(c["shape"], c["kmax"], c["amplitude"], 7),
                      dtype=torch.float64, device=dev)
    J = torch.empty((), dtype=torch.float64, device=dev)
    one = torch.ones((), dtype=torch.float64, device=dev)
    gt = torch.empty((), dtype=torch.float64, device=dev)
    gf = torch.empty(3, dtype=torch.float64, device=dev)
    gu = torch.empty_like(u0)
    N, K = c["steps"], c["checkpoint"]

    def fwd():
        L.lbmp_drag_forward(sim.h, u0.data_ptr(), N, K, 0, J.data_ptr())

    def bwd():
        L.lbmp_drag_backward(sim.h, one.data_ptr(), gt.data_ptr(), gf.data_ptr(), gu.data_ptr())

    fwd()
    bwd()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    tf, tb = [], []
    for _ in range(reps):
        ev[0].record(sim.stream)
        fwd()
        ev[1].record(sim.stream)
        bwd()
        ev[2].record(sim.stream)
        torch.cuda.synchronize()
        tf.append(ev[0].elapsed_time(ev[1]))
        tb.append(ev[1].elapsed_time(ev[2]))
    sim.check()
    sim.profile(True)
    bwd()
    torch.cuda.synchronize()
    prof = sim.profile_result()
    sim.profile(False)
    n = int(np.prod(c["shape"]))
    out = {
        "workload": "gradient of the mean drag over 500 steps: 64^3 periodic, fixed sphere d=12, g_x=1e-6, "
                    "Fourier u0 |k|<=4 amplitude 1e-3, checkpoints every 50, %s" % prec,
        "ms_forward": float(np.median(tf)), "ms_backward": float(np.median(tb)),
        "reverse_mlups": N * n / (float(np.median(tb)) * 1e-3) / 1e6,
        "J": J.item(), "dJ_dtau": gt.item(), "dJ_dgx": gf[0].item(),
        "roofline": roofline(prof, "k_adj_plain (reverse stream-collide, %s)" % prec,
                             profiled_traffic("k_adj_plain_%s_adjoint64.md" % prec, "traffic_bytes_per_launch")),
        "bytes_per_cell_reverse": 19 * (8 if prec == "fp64" else 4) * 3,
    }
    sim.close()
    return out


def replica_context(backend="nccl"):
    """(world, rank, local rank, torch.distributed or None) from the torchrun
    environment; with more than one rank the process group is joined (NCCL
    between GPUs).  Every rank runs an independent replica of the workload."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)
    return world, rank, local, dist


def max_over_ranks(value, dist, device):
    """The largest of the ranks' values (every rank gets it): the job's time."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(world, updates_per_rank, ms_max):
    """Whole-job throughput of weak-scaled replicas: all ranks' cell updates
    over the slowest rank's time."""
    return world * updates_per_rank / (ms_max * 1e-3) / 1e6


def refined_runs(L, prec, args, torch, local, dist, world, full):
    """The headline workload in one precision.  After the warm-up: a cold-start
    window (the first steps from rest); the run is then advanced untimed to
    the developed state and a window of args.steps level-0 steps is timed that
    holds one regrid (value); with full=True also a long developed window
    (args.long_steps, one regrid per 50 steps), the per-launch profile of the
    level update (roofline) and the end-to-end measurement through the C ABI."""
    import numpy as np
    w = REFINED
    bpp = BYTES_PER_POP[prec]
    tau, gm = ga_tau_g(w["ga"], w["u_g"], w["diameter"], w["density_ratio"])
    sim = refined_sim(L, prec)
    sim.step(args.warmup)
    out = {}
    with ClockSampler(local) as clk:
        cms, _, c0, c1 = timed(sim, args.steps, sim.stream, torch, profile=False)
        out["cold_start"] = {"value": job_mlups(world, c1[1] - c0[1], max_over_ranks(cms, dist, "cuda")),
                             "unit": "MLUPS", "ms_per_step": cms / args.steps, "start_step": int(c0[0]),
                             "steps": args.steps, "cell_updates_per_step": (c1[1] - c0[1]) / args.steps,
                             "note": "first steps from rest after the warm-up (the initial hierarchy)"}
        # developed state: the window (start, start + K] holds the regrid after level-0 step DEVELOPED_STEP + 50
        interval = w["regrid"]
        regrid_at = DEVELOPED_STEP + interval
        start = regrid_at - (args.steps + 1) // 2
        sim.step(max(start - int(sim.counters()[0]), 0))
        start = int(sim.counters()[0])
        maps0 = [sim.block_map(l).copy() for l in range(w["levels"])]
        window = full and args.cuda_profiler_window
        if window:
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
        ms, _, d0, d1 = timed(sim, args.steps, sim.stream, torch, profile=False)
        if window:
            torch.cuda.profiler.stop()
        maps1 = [sim.block_map(l) for l in range(w["levels"])]
        ms_max = max_over_ranks(ms, dist, "cuda")
        regrids = sum(1 for s_ in range(start + 1, start + args.steps + 1) if s_ % interval == 0)
        out["value"] = job_mlups(world, d1[1] - d0[1], ms_max)
        out["ms_per_step"] = ms_max / args.steps
        out["gpu_launches"] = int(d1[2] - d0[2])
        out["config"] = {"start_step": start, "steps": args.steps, "regrids_in_window": regrids,
                         "hierarchy_changed_in_window": any(not np.array_equal(a, b) for a, b in zip(maps0, maps1)),
                         "cell_updates_per_step": (d1[1] - d0[1]) / args.steps,
                         "real_blocks_per_level": [int((m >= 0).sum()) for m in maps1],
                         "launches_per_step": int(sim.updates_per_step()[1]),
                         "l2": "inputs larger than L2 (no flush)"}
        if full:
            lms, _, e0, e1 = timed(sim, args.long_steps, sim.stream, torch, profile=False)
            out["developed_long"] = {
                "value": job_mlups(world, e1[1] - e0[1], max_over_ranks(lms, dist, "cuda")), "unit": "MLUPS",
                "ms_per_step": lms / args.long_steps, "start_step": int(e0[0]), "steps": args.long_steps,
                "regrids": args.long_steps // interval, "cell_updates_per_step": (e1[1] - e0[1]) / args.long_steps}
        # per-launch events around every level update (no CUDA graph): the roofline of k_update
        pms, prof, _, _ = timed(sim, max(10, args.steps // 2), sim.stream, torch, profile=True)
    out["clocks"] = clk.summary()
    out["roofline"] = roofline(prof, "k_update (refined stream + collide / coalescence, %s)" % prec,
                               profiled_traffic("k_update_%s_refined.md" % prec, "traffic_bytes_per_launch"))
    out["roofline"]["bytes_per_cell_update"] = 38 * bpp
    out["profiled_pass"] = {"steps": int(prof[3]), "ms_per_step": prof[2] / max(prof[3], 1),
                            "start_step": int(sim.counters()[0] - prof[3]), "note": "per-launch events, no CUDA graph"}
    if full:
        out["e2e"] = e2e(sim, args.e2e_steps, np.array([0.0, 0.0, -gm]))
        part = sim.particle()
        out["particle_after"] = {"step": int(sim.counters()[0]), "z": part[8], "u_z": part[11]}
    sim.close()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.validate > 0:
        return validate(args)
    if args.stability:
        return stability_study(args)
    if args.rotation:
        return rotation_study(args)
    import numpy as np
    import torch

    import paper_2103_10882_gb300 as L
    from paper_2103_10882_gb300 import workloads

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))   # before the NCCL group is joined
    world, rank, local, dist = replica_context("nccl")
    prec = args.precision
    bpp = BYTES_PER_POP[prec]
    line = {}

    # ------------------------------------------------- refined (headline)
    ref = refined_runs(L, prec, args, torch, local, dist, world, full=True)
    line.update({
        "metric": METRIC, "value": ref["value"], "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ref["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE[prec], "data": "synthetic",
        "paper_context": PAPER_CONTEXT,
        "config": dict(ref["config"], workload=REFINED_NAME, precision=prec,
                       parallelism="replicas" if world > 1 else "single GPU"),
    })
    for k in ("roofline", "profiled_pass", "e2e", "gpu_launches", "clocks", "cold_start", "developed_long",
              "particle_after"):
        if k in ref:
            line[k] = ref[k]
    # the same windows in the other two precisions (FP16 deviation storage with FP32 arithmetic; FP64)
    if not args.no_other_precisions:
        others = {}
        for p2 in ("fp16", "fp64", "fp32"):
            if p2 != prec:
                r2 = refined_runs(L, p2, args, torch, local, dist, world, full=False)
                others[p2] = {"value": r2["value"], "unit": "MLUPS", "ms_per_step": r2["ms_per_step"], "dtype": DTYPE[p2],
                              "config": r2["config"], "roofline": r2["roofline"], "clocks": r2["clocks"]}
                if p2 == "fp64":   # the memory fraction is stated, but GB300's FP64 arithmetic bounds this path
                    others[p2]["roofline"]["note"] = ("FP64 arithmetic-bound: about 200 FP64 operations per cell "
                                                      "update; the HBM fraction is shown for comparison")
        f64 = others["fp64"]["value"] if "fp64" in others else ref["value"]
        line["speedup_over_fp64"] = ref["value"] / f64
        for p2, r2 in others.items():
            r2["speedup_over_fp64"] = r2["value"] / f64
            line["refined_" + p2] = r2

    # --------------------------------------------- uniform bandwidth case
    def uniform_case(bulk):
        e = args.edge
        uw = UNIFORM
        tau_u, gm_u = ga_tau_g(uw["ga"], uw["u_g"], uw["diameter"], uw["density_ratio"])
        us = L.Simulation((e, e, e), precision=prec, tau=tau_u, bulk=bulk)
        pos = np.array([e / 2, e / 2, e / 4]) + workloads.sub_cell_offset(rank)
        us.add_sphere(pos, uw["diameter"], uw["density_ratio"], cv=uw["cv"])
        us.set_gravity((0.0, 0.0, -gm_u))
        us.init_fluid()
        us.step(3)
        with ClockSampler(local) as clk_u:
            ums, uprof, u0, u1 = timed(us, args.uniform_steps, us.stream, torch, profile=True)
        us.close()
        model = "TRT" if bulk == 1.0 else "MRT, bulk factor %g" % bulk
        return {
            "workload": uniform_name(e, prec) + ("" if bulk == 1.0 else ", " + model),
            "value": (u1[1] - u0[1]) / (ums * 1e-3) / 1e6, "unit": "MLUPS",
            "ms_per_step": ums / args.uniform_steps,
            "roofline": roofline(uprof, "k_bulk (stream + %s collide, %s)" % (model, prec),
                                 profiled_traffic("k_bulk_%s_uniform256.md" % prec, "traffic_bytes_per_launch_512")
                                 if e == 512 and bulk == 1.0 else None),
            "roofline_mlups": measured_peak()[0] * 1e9 / (38 * bpp) / 1e6,
            "clocks": clk_u.summary(),
        }

    if not args.no_uniform:
        line["uniform512"] = uniform_case(1.0)
        if not args.no_mrt:   # the paper's default collision (Sec. 2.1: Lambda_b = 100)
            line["uniform512_mrt"] = uniform_case(100.0)
    # --------------------------------------------- batched parameter sweep
    if not args.no_batch:
        sims = []
        for d in workloads.batch_sweep(0, 64):
            e = d["edge"]
            tau_b, gm_b = ga_tau_g(d["ga"], 0.01, d["diameter"], d["density_ratio"])
            sims.append(dict(edge=e, pos=e / 2 + d["offset"], diameter=d["diameter"],
                             density_ratio=d["density_ratio"], cv=0.5, tau=tau_b, gravity=(0.0, 0.0, -gm_b)))
        bs = L.BatchSimulation(sims, precision=prec)
        bs.autotune(5)
        info = bs.info()
        bs.step(4)
        with ClockSampler(local) as clk_b:
            bms, _, b0, b1 = timed(bs, args.batch_steps, bs.stream, torch, profile=False)
            _, bprof, _, _ = timed(bs, 4, bs.stream, torch, profile=True)
        bs.close()
        line["batch64"] = {
            "workload": "64 independent periodic boxes, edges from {32,48,64,96}, d = edge/6, pi_p in [0.1,0.9], "
                        "Ga in [100,400], C_v=0.5, seed 0, %s" % prec,
            "value": (b1[1] - b0[1]) / (bms * 1e-3) / 1e6, "unit": "MLUPS", "cells": int(info[1]),
            "ms_per_step": bms / args.batch_steps, "launches_per_step": (b1[2] - b0[2]) / args.batch_steps,
            "autotuner": {"threads_per_tile": int(info[2]), "z_cells_per_thread": int(info[3]),
                          "candidate_us": [v / 1e3 for v in info[4:8]]},
            "roofline": roofline(bprof, "k_batch_bulk (%s)" % prec,
                                 profiled_traffic("k_batch_bulk_%s_batch64.md" % prec, "traffic_bytes_per_launch")),
            "clocks": clk_b.summary(),
        }
    # --------------------------------------------- differentiation (adjoint)
    if not args.no_adjoint:
        line["adjoint64"] = adjoint_line(L, workloads, torch, "fp64" if prec == "fp64" else "fp32", args.adjoint_reps)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
