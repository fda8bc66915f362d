"""Pins of the oracle's MRT collision (Sec. 2.1: C = M^-1 S M with the bulk
factor Lambda_b; Lambda_b = 1 is TRT).

- Lambda_b = 1 + 1e-12 takes the MRT code path and must reproduce the TRT
  path (forced flow past a moving sphere), which pins the moment basis
  (complete, orthogonal, even/odd classes), the relaxation classes and the
  source treatment;
- sound waves decay at the linearised compressible Navier-Stokes rate
  k^2/2 (4 nu/3 + nu_b) with the paper's nu_b = (2/3) c_s^2 (1/s_b - 1/2):
  the bulk rate acts on the bulk mode;
- shear waves decay at nu k^2 whatever Lambda_b: the shear modes keep s_nu;
- mass and momentum are conserved to rounding with Lambda_b = 100.
"""
import math

import numpy as np
import pytest

from lattice_ref import C, W

TAU = 0.6
NU = (TAU - 0.5) / 3.0


def test_mrt_at_unit_bulk_factor_equals_trt(orc):
    runs = []
    for bulk in (1.0, 1.0 + 1e-12):
        s = orc.UniformSim((24, 24, 24), tau=TAU, body_force=(2e-6, -1e-6, 3e-6), bulk=bulk)
        s.add_sphere((12.3, 11.8, 12.6), 8.0, 0.5, cv=0.5)
        s.set_gravity((0, 0, -2.5e-5))
        rng = np.random.default_rng(4)
        u = rng.uniform(-5e-3, 5e-3, size=(3, 24 * 24 * 24))
        s.init_equilibrium(u_field=u)
        s.step(30)
        runs.append((s.populations(), s.history()))
    (g0, h0), (g1, h1) = runs
    scale = np.abs(g0).max()
    assert np.abs(g1 - g0).max() <= 1e-10 * scale
    assert np.abs(h1[:, 0:6] - h0[:, 0:6]).max() <= 1e-9 * np.abs(h0[:, 0:3]).max()


def _wave(orc, bulk, kind, n=64, steps=400):
    """Amplitude history of a long wave along x in a periodic n x 4 x 4 box."""
    s = orc.UniformSim((n, 4, 4), tau=TAU, bulk=bulk)
    x = (np.arange(n) + 0.5)
    k = 2 * math.pi / n
    ncell = n * 16
    xs = np.tile(x, 16)                      # x fastest
    amp = 1e-4
    g = np.zeros((19, ncell))
    if kind == "sound":                      # density wave, fluid at rest
        drho = amp * np.cos(k * xs)
        g[:] = W[:, None] * drho[None, :]
    else:                                    # shear wave u_y = amp sin(k x)
        uy = amp * np.sin(k * xs)
        cu = C[:, 1][:, None] * uy[None, :]
        g[:] = W[:, None] * (3 * cu + 4.5 * cu ** 2 - 1.5 * uy[None, :] ** 2)
    s.set_populations(g)
    e = []
    cosk, sink = np.cos(k * xs), np.sin(k * xs)
    for t in range(steps):
        gp = s.populations()
        rho = gp.sum(axis=0)
        j = gp.T @ C.astype(float)
        if kind == "sound":
            # acoustic energy of the mode: c_s^2 |rho_k|^2 + |j_k|^2 (constant without damping)
            rk = 2 * (rho @ cosk) / ncell
            jk = 2 * (j[:, 0] @ sink) / ncell
            e.append(rk ** 2 / 3.0 + jk ** 2)
        else:
            e.append((2 * (j[:, 1] @ sink) / ncell) ** 2)
        s.step(1)
    return k, np.array(e)


def _rate(e, skip=50):
    t = np.arange(len(e))[skip:]
    slope = np.polyfit(t, np.log(e[skip:]), 1)[0]
    return -0.5 * slope


@pytest.mark.parametrize("bulk,n,rel", [(1.0, 64, 0.02), (10.0, 64, 0.02), (100.0, 256, 0.05)])
def test_sound_wave_decays_at_the_bulk_viscosity_rate(orc, bulk, n, rel):
    """The closed form is the hydrodynamic limit: the bulk mode must relax
    fast against the wave (omega (1/s_b - 1/2) << 1), so Lambda_b = 100
    (1/s_b - 1/2 = 10 at tau = 0.6) takes a four times longer wave."""
    k, e = _wave(orc, bulk, "sound", n=n)
    nu_b = (2.0 / 3.0) * (1.0 / 3.0) * bulk * (TAU - 0.5)      # (2/3) c_s^2 (1/s_b - 1/2)
    want = 0.5 * k * k * (4.0 * NU / 3.0 + nu_b)
    got = _rate(e)
    assert abs(got - want) <= rel * want, (got, want)


@pytest.mark.parametrize("bulk", [1.0, 100.0])
def test_shear_wave_rate_independent_of_bulk_factor(orc, bulk):
    k, e = _wave(orc, bulk, "shear", steps=300)
    got = _rate(e, skip=0)
    assert abs(got - NU * k * k) <= 2e-3 * NU * k * k


def test_mrt_conserves_mass_and_momentum(orc):
    s = orc.UniformSim((16, 16, 16), tau=0.55, bulk=100.0)
    rng = np.random.default_rng(9)
    g = W[:, None] * rng.uniform(-1e-2, 1e-2, size=(19, 16 ** 3))
    s.set_populations(g)
    m0 = g.sum()
    p0 = g.sum(axis=1) @ C.astype(float)
    s.step(20)
    g1 = s.populations()
    assert abs(g1.sum() - m0) < 1e-12
    assert np.abs(g1.sum(axis=1) @ C.astype(float) - p0).max() < 1e-12


def _mode(name):
    """Per-direction values of one D3Q19 moment (Duenweg's orthogonal basis,
    built here from the lattice velocities)."""
    cx, cy, cz = (C[:, a].astype(float) for a in range(3))
    c2 = cx * cx + cy * cy + cz * cz
    return {
        "bulk": c2 - 1.0,                                        # |c|^2 - 1
        "quartic": 3.0 * c2 * c2 - 6.0 * c2 + 1.0,               # isotropic fourth order
        "shear": cx * cy,                                        # a shear mode
        "normal_stress": cy * cy - cz * cz,                      # a shear mode
        "third_order": (cy * cy - cz * cz) * cx,                 # an odd third-order mode
        "third_order_iso": (3.0 * c2 - 5.0) * cx,                # the other kind of odd third-order mode
        "aniso_quartic": (2.0 * c2 - 3.0) * (cy * cy - cz * cz),  # an anisotropic fourth-order mode
    }[name]


@pytest.mark.parametrize("bulk", [10.0, 100.0])
def test_each_moment_relaxes_at_its_class_rate(orc, bulk):
    """A spatially uniform state does not change under streaming, so only the
    collision acts.  A deviation along one non-conserved moment, with weights
    (g_q = a w_q e_q: orthogonal to density and momentum, zero equilibrium at
    rest), stays along it and shrinks by (1 - s) per step.  The reading of
    Sec. 2.1's relaxation counts: s_b for the bulk and the isotropic
    fourth-order moments, s_nu for the shear and the anisotropic fourth-order
    ones, s_minus (TRT's odd rate) for the third-order ones; this pins the
    isotropic fourth-order rate, which the hydrodynamic tests cannot see."""
    s_nu = 1.0 / TAU
    s_minus = 1.0 / (0.5 + (3.0 / 16.0) / (1.0 / s_nu - 0.5))
    s_b = 1.0 / (0.5 + bulk * (1.0 / s_nu - 0.5))
    rates = {"bulk": s_b, "quartic": s_b, "shear": s_nu, "normal_stress": s_nu, "aniso_quartic": s_nu,
             "third_order": s_minus, "third_order_iso": s_minus}
    for name, s in rates.items():
        e = _mode(name)
        assert abs(W @ e) < 1e-15 and np.abs(W @ (e[:, None] * C)).max() < 1e-15   # not density, not momentum
        sim = orc.UniformSim((4, 4, 4), tau=TAU, bulk=bulk)
        g0 = 1e-4 * np.tile((W * e)[:, None], (1, 64))
        sim.set_populations(g0)
        for n in (1, 2, 5):
            sim.step(1 if n != 5 else 3)
            g = sim.populations()
            want = (1.0 - s) ** n * g0
            assert np.abs(g - want).max() <= 1e-13 * np.abs(g0).max(), (name, n)
