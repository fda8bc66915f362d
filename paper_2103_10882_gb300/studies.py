"""Validation studies of the coupled method through the public API.

Stability limit for light spheres (Sec. 3.2, Table 1): the lowest density
ratio pi_p for which a sphere rising at a given Galileo number runs
without instability until it reaches its terminal velocity, with the plain
momentum exchange method (C_v = 0) or with the virtual-mass correction
(C_v > 0, Sec. 3.3).  A run is the paper's setup: a periodic box of
(6.4, 6.4, 12.8) d_p (rounded to whole cells), the sphere starting at
(3.2, 3.2, 0.6) d_p, gravity and viscosity from Ga at u_g = 0.01, fluid at
rest, t_n = t u_g / d_p = 10, and the paper's collision (MRT with the bulk
factor Lambda_b = 100, Sec. 2.1) unless another is asked for.  Two
instability criteria are reported:
  - the paper's: growing oscillations of the hydrodynamic force.  Read here
    as the step-to-step change of the hydrodynamic force on the sphere
    exceeding 100 |F_g| (|F_g| the buoyancy-gravity force that drives the
    sphere) or not being finite.  The momentum exchange force jumps whenever
    the sphere covers or uncovers cells; in stable runs at d_p = 10 and 20
    those jumps stayed below 50 |F_g|, while unstable runs grew by orders of
    magnitude within a few steps;
  - the library's status word (fluid velocity above 0.3 or not finite, the
    sphere jumping more than half a cell in a step), where such
    oscillations end.
A run is stable when neither trips before t_n = 10.

Rotating sphere with virtual mass (Sec. 3.4, Table 3): a (12.8, 6.4, 4.8)
d_p box with no-slip walls on z, the upper one moving with u_w = 0.1 in x,
the fluid starting from the Couette profile, the sphere at the centre held
in place until the flow around it has developed and then free to rotate
(translation still held); its angular velocity omega_y over time, in
t_n = t / t_c and omega_n = omega_y / omega_c with t_c = d_p / u_p,
omega_c = u_p / d_p, u_p = u_w / 2.
"""
import math

import numpy as np

from . import workloads


def rising_sphere_run(L, d, density_ratio, cv, bulk=100.0, precision="fp32", ga=None, chunk=500,
                      force_criterion=True):
    """One rising-sphere run.  Returns a dict: stable (neither criterion
    tripped before t_n = 10), steps done, u_z / u_g at the end (NaN when the
    status word stopped the run), and for each criterion the t_n at which
    it tripped (None if it did not)."""
    w = workloads.STABILITY
    ga = w["ga"] if ga is None else ga
    u_g = w["u_g"]
    shape = tuple(int(round(f * d)) for f in w["box"])
    nu = u_g * d / ga
    cap = chunk + 1
    sim = L.Simulation(shape, precision=precision, tau=3.0 * nu + 0.5, bulk=bulk, history_capacity=cap)
    out = dict(stable=True, steps=0, u_z_over_u_g=float("nan"), t_n_force=None, t_n_status=None)
    try:
        sim.add_sphere(tuple(f * d for f in w["start"]), float(d), float(density_ratio), cv=float(cv))
        sim.set_ga(ga, u_g, (0.0, 0.0, -1.0))
        sim.init_fluid()
        fg = u_g ** 2 * math.pi * d ** 2 / 6.0   # |F_g| = |pi_p - 1| g V with u_g^2 = |pi_p - 1| g d_p
        steps = int(round(w["t_n"] * d / u_g))
        first = True
        done = 0
        while done < steps:
            k = min(chunk, steps - done)
            tripped = False
            try:
                sim.step(k)
            except L.LbmpError as e:
                if e.status != 4:   # LBMP_ERR_UNSTABLE
                    raise
                # the status word is read after each chunk: it tripped by the chunk's end
                out.update(stable=False, t_n_status=(done + k) * u_g / d)
                tripped = True
            if force_criterion:
                # the records of this chunk (with the last one before it): step-to-step changes
                hist = sim.history()
                new = min(k, int(sim.counters()[0]) - done)
                h = hist[-(new + (0 if first else 1)):, 0:3]
                if first:
                    h = np.vstack([h[:1], h])
                first = False
                with np.errstate(invalid="ignore"):
                    jump = np.abs(np.diff(h, axis=0)).max(axis=1)
                over = np.nonzero(~np.isfinite(jump) | (jump > 100.0 * fg))[0]
                if len(over) and out["t_n_force"] is None:
                    out["t_n_force"] = (done + int(over[0]) + 1) * u_g / d
                    out["stable"] = False
            if tripped:
                break
            done += k
        out["steps"] = done
        if out["t_n_status"] is None:
            out["u_z_over_u_g"] = sim.particle()[11] / u_g
        return out
    finally:
        sim.close()


def density_ratio_limit(L, d, cv, lo, hi, iters=5, **kw):
    """Bisection in log(pi_p) between an unstable lo and a stable hi (both
    checked); returns (lowest stable, highest unstable, runs)."""
    runs = []

    def stable(pi):
        r = rising_sphere_run(L, d, pi, cv, **kw)
        runs.append(dict(r, density_ratio=pi))
        return r["stable"]

    if not stable(hi):
        return None, hi, runs
    if stable(lo):
        return lo, None, runs
    for _ in range(iters):
        mid = math.sqrt(lo * hi)
        if stable(mid):
            hi = mid
        else:
            lo = mid
    return hi, lo, runs


def rotating_sphere_run(L, density_ratio, cv, d=None, precision="fp32", bulk=1.0, develop_tc=None,
                        monitor_tc=None, record_every=10):
    """One run of the rotating virtual-mass test (Sec. 3.4).  Returns a dict:
    stable (no status-word error), t_n and omega_n sampled every
    record_every steps after the release, and the run's parameters."""
    import torch
    w = workloads.ROTATION
    d = w["diameter"] if d is None else d
    develop_tc = w["develop_tc"] if develop_tc is None else develop_tc
    monitor_tc = w["monitor_tc"] if monitor_tc is None else monitor_tc
    u_w = w["u_w"]
    u_p = 0.5 * u_w
    nu = u_p * d / w["re_p"]
    shape = tuple(int(round(f * d)) for f in w["box"])
    t_c = d / u_p
    omega_c = u_p / d
    sim = L.Simulation(shape, precision=precision, tau=3.0 * nu + 0.5, bc=("periodic", "periodic", "noslip"),
                       bulk=bulk, history_capacity=record_every)
    out = dict(density_ratio=density_ratio, cv=cv, d=d, shape=shape, tau=3.0 * nu + 0.5, t_c=t_c, omega_c=omega_c,
               stable=True, t_n=[], omega_n=[])
    try:
        sim.add_sphere(tuple(0.5 * n for n in shape), float(d), float(density_ratio), cv=float(cv))
        sim.set_fixed(True)
        sim.set_wall_velocity(2, 1, (u_w, 0.0, 0.0))
        nz = shape[2]
        prof = u_w * (torch.arange(nz, dtype=torch.float64, device="cuda") + 0.5) / nz
        uf = torch.zeros((3, nz, shape[1], shape[0]), dtype=torch.float64, device="cuda")
        uf[0] = prof[:, None, None]
        sim.init_fluid(u_field=uf)
        del uf
        sim.step(int(round(develop_tc * t_c)))
        sim.set_fixed("translation")
        n = int(round(monitor_tc * t_c))
        done = 0
        while done < n:
            k = min(record_every, n - done)
            try:
                sim.step(k)
            except L.LbmpError as e:
                if e.status != 4:
                    raise
                out["stable"] = False
                break
            done += k
            out["t_n"].append(done / t_c)
            out["omega_n"].append(sim.particle()[13] / omega_c)
        return out
    finally:
        sim.close()


def rotation_errors(vm, mem):
    """Mean and terminal relative error of omega_n of a virtual-mass run
    against the plain-MEM run of the same density ratio (Table 3's
    measures), over the samples both have."""
    a, b = np.asarray(vm["omega_n"]), np.asarray(mem["omega_n"])
    n = min(len(a), len(b))
    a, b = a[:n], b[:n]
    rel = np.abs(a - b) / np.abs(b).max()
    return float(rel.mean()), float(abs(a[-1] - b[-1]) / abs(b[-1]))

