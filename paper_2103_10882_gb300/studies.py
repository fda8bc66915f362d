"""Stability limit of the coupled method for light spheres (Sec. 3.2,
Table 1): the lowest density ratio pi_p for which a sphere rising at a
given Galileo number runs without instability until it reaches its
terminal velocity, with the plain momentum exchange method (C_v = 0) or
with the virtual-mass correction (C_v > 0, Sec. 3.3).

A run is the paper's setup through the public API: a periodic box of
(6.4, 6.4, 12.8) d_p (rounded to whole cells), the sphere starting at
(3.2, 3.2, 0.6) d_p, gravity and viscosity from Ga at u_g = 0.01, fluid at
rest, t_n = t u_g / d_p = 10.  It counts as unstable when the library's
status word reports it (fluid velocity above 0.3 or not finite, or the
sphere jumping more than half a cell in a step), which is where the
growing force oscillations the paper describes end.
"""
import math

from . import workloads


def rising_sphere_run(L, d, density_ratio, cv, bulk=1.0, precision="fp32", ga=None, chunk=500):
    """One run; returns (stable, steps_done, u_z / u_g at the end or NaN)."""
    w = workloads.STABILITY
    ga = w["ga"] if ga is None else ga
    u_g = w["u_g"]
    shape = tuple(int(round(f * d)) for f in w["box"])
    nu = u_g * d / ga
    sim = L.Simulation(shape, precision=precision, tau=3.0 * nu + 0.5, bulk=bulk, history_capacity=1)
    try:
        sim.add_sphere(tuple(f * d for f in w["start"]), float(d), float(density_ratio), cv=float(cv))
        sim.set_ga(ga, u_g, (0.0, 0.0, -1.0))
        sim.init_fluid()
        steps = int(round(w["t_n"] * d / u_g))
        done = 0
        while done < steps:
            k = min(chunk, steps - done)
            try:
                sim.step(k)
            except L.LbmpError as e:
                if e.status != 4:   # LBMP_ERR_UNSTABLE
                    raise
                return False, done, float("nan")
            done += k
        return True, done, sim.particle()[11] / u_g
    finally:
        sim.close()


def density_ratio_limit(L, d, cv, lo, hi, iters=5, **kw):
    """Bisection in log(pi_p) between an unstable lo and a stable hi (both
    checked); returns (lowest stable, highest unstable, runs)."""
    runs = []

    def stable(pi):
        ok, done, uz = rising_sphere_run(L, d, pi, cv, **kw)
        runs.append(dict(density_ratio=pi, stable=ok, steps=done, u_z_over_u_g=uz))
        return ok

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
