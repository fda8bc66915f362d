"""Pins of the tangent-linear drag oracle (oracle/tangent.cpp).

Its primal must be the uniform oracle's own step (per-step forces equal bit
for bit); its derivative must match central differences of the uniform
oracle, two closed forms derived by hand from the CLI rule and the TRT
collision for the first steps from rest, and the linearity every tangent
model has.
"""
import math

import numpy as np
import pytest

from lattice_ref import C, W, opposite
from paper_2103_10882_gb300 import workloads

SHAPE = (16, 16, 16)
POS = (8.3, 7.6, 8.1)
D = 5.0


def uniform_drag(orc, tau, force, u0, steps, axis=0):
    """Mean drag from the uniform oracle with the sphere held fixed."""
    o = orc.UniformSim(SHAPE, tau=tau, body_force=force)
    o.add_sphere(POS, D, 1.0, fixed=True)
    o.init_equilibrium(u_field=u0)
    o.step(steps)
    h = o.history()
    return math.fsum(h[:, axis]) / steps, h


def link_table(orc):
    o = orc.UniformSim(SHAPE, tau=0.7)
    o.add_sphere(POS, D, 1.0, fixed=True)
    cell, q, delta = o.links()
    flags = o.flags()
    nx, ny, nz = SHAPE
    far_ok = np.empty(len(cell), dtype=bool)
    far = np.empty(len(cell), dtype=np.int64)
    for m, (x, k) in enumerate(zip(cell, q)):
        i, j, kk = x % nx, (x // nx) % ny, x // (nx * ny)
        f = ((i - C[k, 0]) % nx) + nx * (((j - C[k, 1]) % ny) + ny * ((kk - C[k, 2]) % nz))
        far[m] = f
        far_ok[m] = flags.ravel()[f] == 0
    kappa = np.where(far_ok, (1 - 2 * delta) / (1 + 2 * delta), 0.0)
    return cell, q, kappa, far, far_ok


def test_primal_is_the_uniform_oracle(orc):
    u0 = workloads.fourier_velocity_field(SHAPE, 2, 1e-2, 3)
    J, _, forces = orc.drag_tangent(SHAPE, 0.7, POS, D, 12, u0=u0, body_force=(1e-5, 0, 0))
    Ju, h = uniform_drag(orc, 0.7, (1e-5, 0, 0), u0, 12)
    assert np.array_equal(forces, h[:, 0:3])
    assert J == pytest.approx(Ju, rel=1e-14, abs=0)


def test_force_derivative_two_steps_from_rest(orc):
    """From rest with F = 0: g^1 = 3 w_q c_q.F to first order, so
    dJ/dF_x over two steps is (1/2) sum_links 6 w_k c_kx^2 (1 + kappa0)."""
    cell, q, kappa, _, _ = link_table(orc)
    expect = 0.5 * sum(6 * W[k] * C[k, 0] ** 2 * (1 + kap) for k, kap in zip(q, kappa))
    _, dJ, _ = orc.drag_tangent(SHAPE, 0.7, POS, D, 2, dforce=(1, 0, 0))
    assert dJ == pytest.approx(expect, rel=1e-12)
    # nothing reaches the force at the first step
    _, dJ1, _ = orc.drag_tangent(SHAPE, 0.7, POS, D, 1, dforce=(1, 0, 0))
    assert dJ1 == 0.0
    _, dJt, _ = orc.drag_tangent(SHAPE, 0.7, POS, D, 1, u0=workloads.fourier_velocity_field(SHAPE, 2, 1e-2, 4),
                                 dtau=1.0)
    assert dJt == 0.0


def test_velocity_derivative_one_step_from_rest(orc):
    """One step from rest: dJ = sum_links 3 w_k c_kx [(2 + kappa0) c_k.du(x) + kappa0 c_k.du(x - c_k)]."""
    cell, q, kappa, far, far_ok = link_table(orc)
    du = workloads.fourier_velocity_field(SHAPE, 3, 1.0, 11).reshape(3, -1)
    expect = 0.0
    for x, k, kap, f in zip(cell, q, kappa, far):
        ck = C[k].astype(float)
        expect += 3 * W[k] * ck[0] * ((2 + kap) * (ck @ du[:, x]) + kap * (ck @ du[:, f]))
    _, dJ, _ = orc.drag_tangent(SHAPE, 0.7, POS, D, 1, du0=du.reshape(3, 16, 16, 16))
    assert dJ == pytest.approx(expect, rel=1e-12)


@pytest.mark.parametrize("what", ["tau", "force", "u0"])
def test_against_central_differences(orc, what):
    """20 steps of a forced, swirling flow past the sphere: the tangent
    against central differences of the uniform oracle."""
    tau, F, steps = 0.7, 1e-5, 20
    u0 = workloads.fourier_velocity_field(SHAPE, 2, 1e-2, 3)
    du = workloads.fourier_velocity_field(SHAPE, 3, 1.0, 17)
    if what == "tau":
        _, dJ, _ = orc.drag_tangent(SHAPE, tau, POS, D, steps, u0=u0, body_force=(F, 0, 0), dtau=1.0)
        h = 1e-4
        jp = uniform_drag(orc, tau + h, (F, 0, 0), u0, steps)[0]
        jm = uniform_drag(orc, tau - h, (F, 0, 0), u0, steps)[0]
    elif what == "force":
        _, dJ, _ = orc.drag_tangent(SHAPE, tau, POS, D, steps, u0=u0, body_force=(F, 0, 0), dforce=(1, 0, 0))
        h = 1e-6
        jp = uniform_drag(orc, tau, (F + h, 0, 0), u0, steps)[0]
        jm = uniform_drag(orc, tau, (F - h, 0, 0), u0, steps)[0]
    else:
        _, dJ, _ = orc.drag_tangent(SHAPE, tau, POS, D, steps, u0=u0, body_force=(F, 0, 0), du0=du)
        h = 1e-6
        jp = uniform_drag(orc, tau, (F, 0, 0), u0 + h * du, steps)[0]
        jm = uniform_drag(orc, tau, (F, 0, 0), u0 - h * du, steps)[0]
    fd = (jp - jm) / (2 * h)
    assert dJ == pytest.approx(fd, rel=1e-6)


def test_tangent_is_linear_in_the_direction(orc):
    u0 = workloads.fourier_velocity_field(SHAPE, 2, 1e-2, 3)
    du = workloads.fourier_velocity_field(SHAPE, 3, 1.0, 17)
    args = (SHAPE, 0.7, POS, D, 8)
    kw = dict(u0=u0, body_force=(1e-5, 0, 0))
    _, a, _ = orc.drag_tangent(*args, dtau=1.0, **kw)
    _, b, _ = orc.drag_tangent(*args, dforce=(1, 0, 0), **kw)
    _, c, _ = orc.drag_tangent(*args, du0=du, **kw)
    _, a2, _ = orc.drag_tangent(*args, dtau=2.0, **kw)
    _, abc, _ = orc.drag_tangent(*args, dtau=1.0, dforce=(1, 0, 0), du0=du, **kw)
    assert a2 == 2 * a
    assert abc == pytest.approx(a + b + c, rel=1e-12, abs=1e-12 * (abs(a) + abs(b) + abs(c)))
