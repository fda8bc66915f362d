"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it checks and the mistake it would catch.
None of these compares the oracle with itself: the expected values are
closed forms, conservation laws, exact identities of the scheme, or brute
force recomputations from the definitions in lattice_ref.py.
"""
import numpy as np
import pytest

from lattice_ref import C, W, cell_centres, moments, opposite


# ------------------------------------------------------------------ lattice
def test_equilibrium_moments(orc):
    """Sec. 2.1, Eq. (rho_f, rho_0 u_f): the equilibrium carries rho and
    rho_0 u, and its second moment is rho c_s^2 I + rho_0 u u (He & Luo
    incompressible form).  Catches a wrong weight or coefficient."""
    rng = np.random.default_rng(1)
    s = orc.UniformSim((4, 3, 2), tau=0.8)
    n = s.ncells
    uf = rng.uniform(-0.05, 0.05, size=(3, n))
    s.init_equilibrium(rho=1.013, u=(0, 0, 0), u_field=uf)
    g = s.populations()
    rho, u = moments(g, s.shape)
    np.testing.assert_allclose(rho, 1.013, rtol=0, atol=1e-15)
    np.testing.assert_allclose(u, uf, rtol=0, atol=1e-16)
    f = g + W[:, None]
    Cf = C.astype(np.float64)
    Pi = np.einsum("qa,qb,qn->abn", Cf, Cf, f)
    expect = rho[None, None, :] / 3.0 * np.eye(3)[:, :, None] + uf[:, None, :] * uf[None, :, :]
    np.testing.assert_allclose(Pi, expect, rtol=0, atol=1e-15)


def test_rest_state_is_unchanged(orc):
    """Rest state with a sphere at rest and no gravity stays at rest: CLI
    returns w_q for every link and the MEM link forces reduce to 2 w_q c_q,
    whose sum over a closed surface is zero.  The oracle evaluates both on
    full populations f = w + g, so the deviations stay at rounding level."""
    for boundary in ("cli", "sbb"):
        s = orc.UniformSim((16, 16, 16), tau=0.6, boundary=boundary)
        s.add_sphere((8.21, 7.93, 8.47), 6.0, 0.5, cv=0.5)
        s.init_equilibrium()
        flags0 = s.flags()
        s.step(20)
        assert np.abs(s.populations()).max() < 1e-16
        assert np.array_equal(s.flags(), flags0)
        p = s.particle()
        assert np.abs(p[0:6]).max() < 1e-15
        assert np.abs(p[9:15]).max() < 1e-15


def test_mass_momentum_conservation_periodic(orc):
    """TRT collision conserves rho and rho_0 u locally and the periodic
    stream conserves them globally (Sec. 2.1)."""
    rng = np.random.default_rng(2)
    shape = (8, 6, 5)
    s = orc.UniformSim(shape, tau=0.7)
    g0 = rng.normal(scale=1e-3, size=(19, s.ncells))
    s.set_populations(g0)
    rho0, u0 = moments(g0, shape)
    s.step(50)
    rho1, u1 = moments(s.populations(), shape)
    assert abs(rho1.sum() - rho0.sum()) < 1e-12
    np.testing.assert_allclose(u1.sum(axis=1), u0.sum(axis=1), rtol=0, atol=1e-14)


def test_shear_wave_viscosity(orc):
    """Sec. 2.1: nu = c_s^2 (1/s_nu - 1/2).  A shear wave u_x = A sin(k y)
    decays as exp(-nu k^2 t).  Catches a wrong s+ (e.g. a 1/(tau+1/2))."""
    ny = 64
    tau = 0.8
    nu = (tau - 0.5) / 3.0
    s = orc.UniformSim((1, ny, 1), tau=tau)
    y = np.arange(ny) + 0.5
    k = 2 * np.pi / ny
    A = 1e-4
    uf = np.zeros((3, ny))
    uf[0] = A * np.sin(k * y)
    s.init_equilibrium(u_field=uf)
    T = 400
    s.step(T)
    _, u = moments(s.populations(), s.shape)
    amp = 2.0 / ny * np.sum(u[0] * np.sin(k * y))
    expect = A * np.exp(-nu * k * k * T)
    # O(k^2) lattice dispersion leaves ~5e-4 here; a wrong viscosity law is off by >10%
    assert abs(amp / expect - 1.0) < 1e-3


def _poiseuille(orc, magic):
    ny = 10
    tau = 0.9
    F = 1e-6
    s = orc.UniformSim((1, ny, 1), tau=tau, magic=magic, periodic=(1, 0, 1), body_force=(F, 0, 0))
    s.init_equilibrium()
    s.step(20000)
    rho, u = moments(s.populations(), s.shape)
    # the stored field is post-collision: its momentum already holds the full
    # force of the step, the physical velocity is half a force step earlier
    ux = u[0] - 0.5 * F
    nu = (tau - 0.5) / 3.0
    y = np.arange(ny) + 0.5
    exact = F / (2 * nu) * y * (ny - y)
    return np.abs(ux - exact).max() / exact.max()


def test_poiseuille_exact_with_magic_3_16(orc):
    """Sec. 2.1: with the magic parameter Lambda = 3/16 the TRT bounce-back
    wall sits exactly half-way, so force-driven Poiseuille flow is the exact
    parabola.  With another Lambda it is not: that catches a wrong s-."""
    err = _poiseuille(orc, 3.0 / 16.0)
    assert err < 1e-10
    err_other = _poiseuille(orc, 0.25)
    assert err_other > 1e-4


@pytest.mark.parametrize("lo,hi", [(0.8, 14.3), (1.45, 13.9), (0.55, 14.05)])
def test_couette_cli_exact(orc, lo, hi):
    """Sec. 2.3: CLI places a moving wall at x + delta c_q and is exact for a
    linear profile for any delta.  Catches a wrong kappa_0 or alpha (in
    particular the garbled factor 3 in the printed moving-wall term)."""
    ny = 16
    v = 0.01
    s = orc.UniformSim((1, ny, 1), tau=0.75)
    s.set_planes(1, lo, hi, v_lo=(0, 0, 0), v_hi=(v, 0, 0))
    s.init_equilibrium()
    s.step(12000)
    flags = s.flags()
    _, u = moments(s.populations(), s.shape)
    y = np.arange(ny) + 0.5
    fluid = flags == 0
    exact = v * (y - lo) / (hi - lo)
    err = np.abs(u[0][fluid] - exact[fluid]).max()
    assert err < 1e-12 * 1e3 * v   # steady state reached to ~1e-11 relative


def test_momentum_balance_fixed_sphere(orc):
    """Sec. 2.3: the link force is the momentum the fluid loses through the
    wall, so with a fixed sphere and a body force the fluid momentum changes
    each step by exactly N_fluid F_body - F_hyd.  Catches a dropped term or a
    sign error in the link-force formula, for CLI and bounce-back."""
    for boundary in ("cli", "sbb"):
        F = np.array([2e-6, -1e-6, 5e-7])
        shape = (16, 16, 16)
        s = orc.UniformSim(shape, tau=0.7, body_force=F, boundary=boundary)
        s.add_sphere((8.3, 7.6, 8.9), 7.0, 1.0, fixed=True)
        s.init_equilibrium()
        s.step(30)
        fluid = s.flags() == 0
        nf = fluid.sum()
        for _ in range(5):
            _, u0 = moments(s.populations(), shape)
            P0 = u0[:, fluid].sum(axis=1)
            s.step(1)
            _, u1 = moments(s.populations(), shape)
            P1 = u1[:, fluid].sum(axis=1)
            Fh = s.particle()[0:3]
            # the link forces are sums of O(w_q) terms that cancel to O(1e-3):
            # their rounding is ~1e-14 absolute; a wrong term is ~1e-3
            np.testing.assert_allclose(P1 - P0, nf * F - Fh, rtol=0, atol=1e-13)


def test_mass_conserved_sbb_fixed_sphere(orc):
    """Simple bounce-back on a fixed sphere conserves fluid mass exactly."""
    rng = np.random.default_rng(3)
    shape = (12, 12, 12)
    s = orc.UniformSim(shape, tau=0.65, boundary="sbb")
    s.add_sphere((6.1, 6.2, 5.8), 5.0, 1.0, fixed=True)
    fluid = s.flags() == 0
    g0 = rng.normal(scale=1e-3, size=(19, s.ncells)) * fluid[None, :]
    s.set_populations(g0)
    m0 = g0.sum()
    s.step(40)
    assert abs(s.populations().sum() - m0) < 1e-13


# ---------------------------------------------------------------- mapping
def test_flags_and_links_brute_force(orc):
    """Sec. 2.3 mapping: solid iff the cell centre lies in the sphere; links
    join a fluid cell to a solid neighbour; x_b = x + delta c_q lies on the
    sphere surface.  Brute force in numpy over every cell and direction,
    including a sphere that wraps through the periodic boundary."""
    for pos in [(8.37, 7.71, 8.02), (0.4, 15.2, 7.9)]:
        shape = (16, 16, 16)
        D = 7.3
        s = orc.UniformSim(shape, tau=0.6)
        s.add_sphere(pos, D, 0.5)
        X = cell_centres(shape)
        d = X - np.asarray(pos)[:, None]
        L = np.asarray(shape, dtype=float)[:, None]
        d = np.where(d > L / 2, d - L, np.where(d < -L / 2, d + L, d))
        solid = (d ** 2).sum(axis=0) <= (D / 2) ** 2
        flags = s.flags()
        assert np.array_equal(flags == 1, solid)
        cell, q, delta = s.links()
        # expected link set
        nx, ny, nz = shape
        idx = np.arange(s.ncells)
        i, j, k = idx % nx, (idx // nx) % ny, idx // (nx * ny)
        exp = []
        for qq in range(1, 19):
            nb = ((i + C[qq, 0]) % nx) + nx * (((j + C[qq, 1]) % ny) + ny * ((k + C[qq, 2]) % nz))
            sel = (~solid) & solid[nb]
            exp += [(c, qq) for c in idx[sel]]
        exp.sort()
        got = sorted(zip(cell.tolist(), q.tolist()))
        assert got == exp
        xb = d[:, cell] + delta[None, :] * C[q].T
        np.testing.assert_allclose(np.sqrt((xb ** 2).sum(axis=0)), D / 2, rtol=0, atol=1e-12)
        assert np.all((delta > 0) & (delta <= 1))


# --------------------------------------------------------------- particle
def test_velocity_verlet_constant_force(orc):
    """Sec. 2.2 Velocity Verlet is exact for a constant force:
    x(n) = x0 + F n^2 / (2 m), u(n) = F n / m, with m = rho_p V, V = pi D^3/6."""
    s = orc.UniformSim((8, 8, 8), tau=0.6, plain_mem=True)
    x0 = np.array([4.1, 3.9, 4.2])
    D, rho_p = 3.0, 0.7
    s.add_sphere(x0, D, rho_p)
    F = np.array([1e-3, -2e-3, 5e-4])
    m = rho_p * np.pi * D ** 3 / 6
    for n in range(1, 11):
        s.particle_only_step(F)
        p = s.particle()
        np.testing.assert_allclose(p[6:9], x0 + F * n * n / (2 * m), rtol=1e-14, atol=1e-14)
        # stored u is the drift velocity u(t + 1/2)
        np.testing.assert_allclose(p[9:12], F * (n - 0.5) / m, rtol=1e-13, atol=1e-18)


def test_gravity_buoyancy(orc):
    """Sec. 2.2: F_g = (rho_p - rho_f) g V; a light sphere (rho_p < 1) in
    gravity -z accelerates upward with a = (rho_p - 1) g V / m."""
    s = orc.UniformSim((8, 8, 8), tau=0.6, plain_mem=True)
    D, rho_p = 3.0, 0.25
    s.add_sphere((4.0, 4.0, 4.0), D, rho_p)
    g = np.array([0.0, 0.0, -1e-4])
    s.set_gravity(g)
    s.particle_only_step(np.zeros(3))
    V = np.pi * D ** 3 / 6
    np.testing.assert_allclose(s.particle()[15:18], (rho_p - 1) * g * V / (rho_p * V), rtol=1e-14)


def test_virtual_mass_acceleration_closed_form(orc):
    """Sec. 3.3, Eqs. (virtual force) with a_{p,t-1}: under a constant
    hydrodynamic force F the VM-corrected acceleration is the geometric
    series a(n) = F/(rho_p V) (1 - r^(n+1)), r = C_v / (rho_p + C_v), and it
    converges to the true F / (rho_p V).  Same for the torque with C_vw."""
    s = orc.UniformSim((8, 8, 8), tau=0.6)
    D, rho_p, cv, cvw = 4.0, 0.1, 0.5, 1.0
    s.add_sphere((4.0, 4.0, 4.0), D, rho_p, cv=cv, cv_omega=cvw)
    V = np.pi * D ** 3 / 6
    I_true = 0.4 * rho_p * V * (D / 2) ** 2
    F = np.array([1e-4, 0.0, -3e-4])
    T = np.array([0.0, 2e-4, 1e-4])
    r = cv / (rho_p + cv)
    rw = cvw / (rho_p + cvw)
    for n in range(30):
        s.particle_only_step(F, T)
        p = s.particle()
        np.testing.assert_allclose(p[15:18], F / (rho_p * V) * (1 - r ** (n + 1)), rtol=1e-12)
        np.testing.assert_allclose(p[18:21], T / I_true * (1 - rw ** (n + 1)), rtol=1e-12)


def test_force_average_two_steps(orc):
    """Algorithm 1: the hydrodynamic force is averaged over two steps before
    it enters the particle update (first step: no previous value)."""
    s = orc.UniformSim((8, 8, 8), tau=0.6, plain_mem=True)
    D, rho_p = 3.0, 2.0
    s.add_sphere((4.0, 4.0, 4.0), D, rho_p)
    m = rho_p * np.pi * D ** 3 / 6
    F1, F2 = np.array([1e-3, 0, 0]), np.array([3e-3, 0, 0])
    s.particle_only_step(F1)
    np.testing.assert_allclose(s.particle()[15:18], F1 / m, rtol=1e-15)
    s.particle_only_step(F2)
    np.testing.assert_allclose(s.particle()[15:18], 0.5 * (F1 + F2) / m, rtol=1e-15)


def test_vm_with_zero_coefficients_is_plain_mem(orc):
    """Sec. 3.3: with C_v = C_vw = 0 the VM-MEM reduces to plain MEM
    (m_p = rho_p V, F_v = 0) -- bit-identical trajectories and fields over a
    coupled run of a rising light sphere."""
    res = []
    for plain in (False, True):
        s = orc.UniformSim((16, 16, 24), tau=0.6, plain_mem=plain)
        s.add_sphere((8.2, 7.7, 6.3), 6.0, 0.6, cv=0.0, cv_omega=0.0)
        s.set_gravity((0, 0, -2e-4))
        s.init_equilibrium()
        s.step(60)
        res.append((s.populations(), s.history()))
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])


def test_refill_uncovered_cells(orc):
    """Sec. 2.3 with the equilibrium refill: after the sphere moves, each
    uncovered cell holds f_eq(rho_fill, u_p + omega_p x (x - x_p)) with
    rho_fill the mean density of its neighbours that are fluid before and
    after the move; covered cells hold nothing."""
    shape = (16, 16, 16)
    s = orc.UniformSim(shape, tau=0.6)
    s.add_sphere((8.0, 8.0, 8.0), 6.0, 50.0)
    s.set_particle_velocity((0.45, 0.2, 0.1), (0.0, 0.02, 0.0))
    rng = np.random.default_rng(4)
    fluid0 = s.flags() == 0
    s.set_populations(rng.normal(scale=1e-4, size=(19, s.ncells)) * fluid0[None, :])
    # run one step by hand except the remap: compare against the oracle's remap
    before_flags = s.flags()
    s.step(1)
    after_flags = s.flags()
    g = s.populations()
    p = s.particle()
    xp, up, wp = p[6:9], p[9:12], p[12:15]
    uncovered = np.nonzero((before_flags == 1) & (after_flags == 0))[0]
    covered = np.nonzero((before_flags == 0) & (after_flags == 1))[0]
    assert len(uncovered) > 0 and len(covered) > 0
    assert np.all(g[:, covered] == 0)
    nx, ny, nz = shape
    rho, _ = moments(g, shape)
    X = cell_centres(shape)
    for c in uncovered:
        i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
        nb = [((i + C[q, 0]) % nx) + nx * (((j + C[q, 1]) % ny) + ny * ((k + C[q, 2]) % nz)) for q in range(1, 19)]
        ok = [b for b in nb if before_flags[b] == 0 and after_flags[b] == 0]
        rf = np.mean(rho[ok]) if ok else 1.0
        r = X[:, c] - xp
        u = up + np.cross(wp, r)
        cu = C @ u
        expect = W * ((rf - 1) + 3 * cu + 4.5 * cu ** 2 - 1.5 * u @ u)
        np.testing.assert_allclose(g[:, c], expect, rtol=0, atol=1e-15)


@pytest.mark.slow
def test_hasimoto_periodic_sphere_array(orc):
    """Sec. 2.3 force on a fixed sphere in a periodic cubic array driven by a
    body force, against Hasimoto's (1959) expansion for Stokes drag,
    F = 6 pi mu a U / K, K = 1 - 1.7601 phi^(1/3) + phi - 1.5593 phi^2,
    with U the superficial velocity.  The CLI wall and the truncated series
    agree within 2% at d = 6 cells (measured -1.9%) and 1.5% at d = 8
    (-1.2%), and the difference shrinks with the resolution (the sphere's
    hydrodynamic radius converges to its geometric one; -0.9% at d = 12); a
    missing term of the link force or a wrong viscosity would be far off."""
    ratios = []
    for D, L, steps, tol in ((6.0, 24, 4500, 0.02), (8.0, 32, 8000, 0.015)):
        tau, F = 1.5, 1e-6
        s = orc.UniformSim((L, L, L), tau=tau, body_force=(F, 0, 0))
        s.add_sphere((L / 2 + 0.13, L / 2 - 0.21, L / 2 + 0.07), D, 1.0, fixed=True)
        s.init_equilibrium()
        s.step(steps)
        fluid = s.flags() == 0
        _, u = moments(s.populations(), s.shape)
        U = (u[0][fluid] - 0.5 * F).sum() / L ** 3
        Fh = s.particle()[0]
        assert abs(Fh / (fluid.sum() * F) - 1) < 1e-3   # steady state: drag balances the body force
        nu = (tau - 0.5) / 3
        phi = np.pi * D ** 3 / 6 / L ** 3
        K = 1 - 1.7601 * phi ** (1 / 3) + phi - 1.5593 * phi ** 2
        ratio = Fh / (6 * np.pi * nu * (D / 2) * U / K)
        assert abs(ratio - 1) < tol, (D, ratio)
        ratios.append(ratio)
    assert abs(ratios[1] - 1) < abs(ratios[0] - 1)
