"""Pins of the oracle parts the rotating virtual-mass test needs (Sec. 3.4):
a no-slip domain wall that moves (the upper wall of the Couette flow) and a
sphere whose translation is held while its rotation is free.

- a domain wall with velocity u_w reproduces plane Couette flow exactly;
- the domain wall equals the CLI plane wall of Sec. 2.3 at delta = 1/2,
  pinned separately in test_oracle_pins;
- a held translation keeps position and velocity exactly; a rotation
  released after a held phase follows the same virtual-mass closed form
  (Sec. 3.3) from the release on as a rotation free from the start.
"""
import numpy as np
import pytest

from lattice_ref import moments


@pytest.mark.parametrize("tau", [0.56, 0.9])
def test_moving_domain_wall_couette_exact(orc, tau):
    """Walls on z at the half-way planes z = 0 and z = nz, the upper one
    moving with u_w in x: the steady state is u_x = u_w (z + 1/2) / nz
    exactly (bounce-back with the moving-wall term is exact for a linear
    profile).  A wrong sign or factor of the moving-wall term changes the
    wall velocity the fluid sees and fails by far more than the bound."""
    nz, v = 12, 0.02
    s = orc.UniformSim((2, 2, nz), tau=tau, periodic=(1, 1, 0))
    s.set_wall_velocity(2, 1, (v, 0.0, 0.0))
    s.init_equilibrium()
    s.step(6000 if tau > 0.7 else 20000)
    _, u = moments(s.populations(), s.shape)
    z = np.arange(nz) + 0.5
    exact = np.tile(v * z / nz, (4, 1)).T.reshape(-1)   # cells are x fastest
    assert np.abs(u[0] - exact).max() < 1e-11 * v
    assert np.abs(u[1]).max() < 1e-15 and np.abs(u[2]).max() < 1e-15


def test_domain_wall_equals_plane_wall_at_half_cell(orc):
    """The moving domain wall of a 4 x 4 x 12 box is the CLI plane wall of
    Sec. 2.3 at delta = 1/2: a 4 x 4 x 14 periodic box whose first and last
    layers are solid (planes at z = 1 and z = 13, the same wall
    velocities) gives the same fluid populations after 60 steps of a drifting
    flow, to rounding.  Both walls move, in different directions."""
    vlo, vhi = (-0.004, 0.001, 0.0), (0.01, 0.003, 0.0)
    a = orc.UniformSim((4, 4, 12), tau=0.7, periodic=(1, 1, 0))
    a.set_wall_velocity(2, 0, vlo)
    a.set_wall_velocity(2, 1, vhi)
    b = orc.UniformSim((4, 4, 14), tau=0.7)
    b.set_planes(2, 1.0, 13.0, v_lo=vlo, v_hi=vhi)
    rng = np.random.default_rng(5)
    ua = rng.uniform(-0.01, 0.01, size=(3, 4 * 4 * 12))
    ub = np.zeros((3, 4 * 4 * 14))
    ub.reshape(3, 14, 16)[:, 1:13, :] = ua.reshape(3, 12, 16)
    a.init_equilibrium(u_field=ua)
    b.init_equilibrium(u_field=ub)
    a.step(60)
    b.step(60)
    ga = a.populations().reshape(19, 12, 16)
    gb = b.populations().reshape(19, 14, 16)[:, 1:13, :]
    assert np.abs(ga).max() > 1e-4
    assert np.abs(ga - gb).max() < 1e-15


def _sphere(orc, fixed):
    s = orc.UniformSim((8, 8, 8), tau=0.6)
    s.add_sphere((4.0, 4.0, 4.0), 4.0, 0.1, cv=0.5, cv_omega=1.0, fixed=fixed)
    s.set_particle_velocity((0.001, -0.002, 0.0005), (0.0, 0.0, 0.0))
    return s


def test_translation_held_rotation_free(orc):
    """fixed = translation: under a constant force and torque the centre and
    the translational velocity stay exactly as set, the translational
    acceleration record is zero (so the virtual force is zero), and the
    rotation follows the virtual-mass closed form of Sec. 3.3,
    beta(n) = T / I (1 - r^(n+1)), r = C_vw / (rho_p + C_vw), with the
    kick-drift-kick angular velocity omega(n) = beta(0)/2 + beta(1) + ... +
    beta(n) (the first step has no completing half kick; each later step
    completes the previous half step and starts the next with its own
    beta)."""
    s = _sphere(orc, "translation")
    p0 = s.particle()
    D, rho_p, cvw = 4.0, 0.1, 1.0
    V = np.pi * D ** 3 / 6
    I_true = 0.4 * rho_p * V * (D / 2) ** 2
    r = cvw / (rho_p + cvw)
    F = np.array([1e-4, 2e-4, -3e-4])
    T = np.array([0.0, 2e-4, -1e-4])
    betas = []
    for n in range(25):
        s.particle_only_step(F, T)
        p = s.particle()
        assert np.array_equal(p[6:9], p0[6:9]) and np.array_equal(p[9:12], p0[9:12])
        assert np.all(p[15:18] == 0.0)
        betas.append(T / I_true * (1 - r ** (n + 1)))
        np.testing.assert_allclose(p[18:21], betas[-1], rtol=1e-12, atol=1e-30)
        np.testing.assert_allclose(p[12:15], np.sum(betas, axis=0) - 0.5 * betas[0], rtol=1e-12, atol=1e-30)


def test_rotation_released_after_hold_starts_afresh(orc):
    """Held completely for 7 steps (angular velocity kept, zero angular
    acceleration), then rotation released: from the release on the angular
    velocity and acceleration are those of a sphere whose rotation is free
    from its first step under the same torque.  Catches a release that
    completes a half kick never started, or a virtual torque built from an
    acceleration the held sphere never had."""
    T = np.array([1e-4, -2e-4, 3e-4])
    F = np.array([2e-4, 0.0, 0.0])
    held = _sphere(orc, True)
    for _ in range(7):
        held.particle_only_step(F, T)
        p = held.particle()
        assert np.all(p[12:15] == 0.0) and np.all(p[18:21] == 0.0)
    held.set_fixed("translation")
    free = _sphere(orc, "translation")
    for _ in range(20):
        held.particle_only_step(F, T)
        free.particle_only_step(F, T)
        ph, pf = held.particle(), free.particle()
        np.testing.assert_array_equal(ph[12:15], pf[12:15])
        np.testing.assert_array_equal(ph[18:21], pf[18:21])
