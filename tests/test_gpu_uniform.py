"""GPU parity of the uniform-grid coupled step against the FP64 oracle.

All calls go through the C ABI (via the thin ctypes binding).  Tolerances:
  FP64 path: populations within 1e-10 of max|g| (max-norm), forces within
             1e-10 of max(|F_hyd|, |F_g|), positions/velocities 1e-10
             relative; flags and boundary-link sets bit-exact.
  FP32/FP16: stated per test (storage rounding accumulates over steps).
"""
import numpy as np
import pytest

from paper_2103_10882_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2103_10882_gb300 as L
    L._native.load()
    return L


def ga_to_tau_g(ga, u_g, D, pi):
    """Ga = u_g D / nu, u_g = sqrt(|pi - 1| g D)  (Sec. 3.1), nu = (tau - 1/2)/3."""
    nu = u_g * D / ga
    return 3 * nu + 0.5, u_g ** 2 / (abs(pi - 1) * D)


def make_pair(orc, lib, shape, precision="fp64", tau=0.6, magic=3 / 16, bc=("periodic",) * 3, boundary="cli",
              sphere=None, gravity=(0, 0, 0), body_force=(0, 0, 0), fixed=False, velocity=None, force_average=True):
    periodic = tuple(1 if b == "periodic" else 0 for b in bc)
    o = orc.UniformSim(shape, tau=tau, magic=magic, periodic=periodic, body_force=body_force, boundary=boundary,
                       force_average=force_average)
    g = lib.Simulation(shape, precision=precision, tau=tau, magic=magic, bc=bc, boundary=boundary,
                       force_average=force_average)
    g.set_body_force(body_force)
    if sphere is not None:
        pos, D, pi, cv = sphere
        o.add_sphere(pos, D, pi, cv=cv, fixed=fixed)
        g.add_sphere(pos, D, pi, cv=cv)
        if fixed:
            g.set_fixed(True)
        o.set_gravity(gravity)
        g.set_gravity(gravity)
        if velocity is not None:
            o.set_particle_velocity(*velocity)
            g.set_particle_velocity(*velocity)
    o.init_equilibrium()
    g.init_fluid()
    return o, g


def assert_pops_close(o, g, rel):
    a, b = g.populations(), o.populations()
    scale = max(np.abs(b).max(), 1e-300)
    err = np.abs(a - b).max() / scale
    assert err <= rel, "population error %.3e > %.1e" % (err, rel)
    return err


def assert_links_equal(o, g):
    oc, oq, od = o.links()
    gc, gq, gd = g.links()
    ko = np.lexsort((oq, oc))
    kg = np.lexsort((gq, gc))
    assert np.array_equal(oc[ko], gc[kg])
    assert np.array_equal(oq[ko], gq[kg])
    np.testing.assert_allclose(gd[kg], od[ko], rtol=0, atol=1e-12)


def assert_history_close(o, g, rel, Fscale):
    ho, hg = o.history(), g.history()
    assert ho.shape == hg.shape
    np.testing.assert_allclose(hg[:, 0:6], ho[:, 0:6], rtol=0, atol=rel * Fscale)
    np.testing.assert_allclose(hg[:, 6:9], ho[:, 6:9], rtol=rel, atol=rel)
    vs = max(np.abs(ho[:, 9:15]).max(), 1e-30)
    np.testing.assert_allclose(hg[:, 9:15], ho[:, 9:15], rtol=0, atol=rel * vs)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_single_sphere_fp64_parity(orc, lib, seed):
    """32^3 periodic, D = 8, pi_p = 0.5, C_v = 0.5, tau = 0.6, Lambda = 3/16,
    g from u_g = 0.01, 200 steps; sphere at the centre plus a seeded offset."""
    w = workloads.SINGLE_SPHERE_32
    D, pi = w["diameter"], w["density_ratio"]
    g_mag = w["u_g"] ** 2 / (abs(pi - 1) * D)
    pos = np.array(w["shape"]) / 2 + workloads.sub_cell_offset(seed)
    o, g = make_pair(orc, lib, w["shape"], tau=w["tau"], sphere=(pos, D, pi, w["cv"]), gravity=(0, 0, -g_mag))
    assert np.array_equal(o.flags(), g.flags())
    assert_links_equal(o, g)
    Fscale = abs(pi - 1) * g_mag * np.pi * D ** 3 / 6
    for _ in range(2):
        o.step(100)
        g.step(100)
        assert_pops_close(o, g, 1e-10)
        assert np.array_equal(o.flags(), g.flags())
        assert_links_equal(o, g)
    assert_history_close(o, g, 1e-10, Fscale)
    # the sphere moved by more than a cell: remap and refill were exercised
    assert np.abs(g.particle()[6:9] - pos).max() > 1e-3


def test_ga100_small_tau_fp64_parity(orc, lib):
    """Ga = 100 at u_g = 0.01: tau = 0.5024 (nu = 8e-4), 150 steps."""
    D, pi = 8.0, 0.5
    tau, gm = ga_to_tau_g(100.0, 0.01, D, pi)
    pos = np.array([16.0, 16.0, 14.0]) + workloads.sub_cell_offset(7)
    o, g = make_pair(orc, lib, (32, 32, 32), tau=tau, sphere=(pos, D, pi, 0.5), gravity=(0, 0, -gm))
    o.step(150)
    g.step(150)
    assert_pops_close(o, g, 1e-10)
    assert_links_equal(o, g)
    assert_history_close(o, g, 1e-10, abs(pi - 1) * gm * np.pi * D ** 3 / 6)


def test_literal_ga100_tau06_short(orc, lib):
    """The literal combination tau = 0.6, D = 8, Ga = 100 (g = 0.043): the
    sphere accelerates past 0.1 lattice speed within a few steps; arithmetic
    parity over 10 steps."""
    D, pi = 8.0, 0.5
    nu = (0.6 - 0.5) / 3
    u_g = 100.0 * nu / D
    gm = u_g ** 2 / (abs(pi - 1) * D)
    pos = np.array([16.0, 16.0, 16.0]) + workloads.sub_cell_offset(3)
    o, g = make_pair(orc, lib, (32, 32, 32), tau=0.6, sphere=(pos, D, pi, 0.5), gravity=(0, 0, -gm))
    o.step(10)
    g.step(10)
    assert_pops_close(o, g, 1e-10)
    assert_history_close(o, g, 1e-10, abs(pi - 1) * gm * np.pi * D ** 3 / 6)


def test_sbb_and_no_average_parity(orc, lib):
    pos = np.array([12.3, 11.8, 10.6])
    o, g = make_pair(orc, lib, (24, 24, 28), tau=0.7, boundary="sbb", force_average=False,
                     sphere=(pos, 7.0, 0.3, 1.0), gravity=(0, 0, -4e-5))
    o.step(80)
    g.step(80)
    assert_pops_close(o, g, 1e-10)
    assert_links_equal(o, g)
    assert_history_close(o, g, 1e-10, 0.7 * 4e-5 * np.pi * 343 / 6)


def test_sphere_across_periodic_boundary(orc, lib):
    """Sphere centred near the corner: the solid region, links and the box
    of the remap wrap around three periodic boundaries."""
    pos = np.array([0.7, 31.6, 0.2])
    o, g = make_pair(orc, lib, (32, 32, 32), tau=0.65, sphere=(pos, 9.0, 0.5, 0.5), gravity=(2e-5, -1e-5, 3e-5),
                     velocity=((0.01, -0.02, 0.015), (0.001, 0.0, -0.002)))
    for _ in range(3):
        o.step(40)
        g.step(40)
        assert np.array_equal(o.flags(), g.flags())
        assert_links_equal(o, g)
    assert_pops_close(o, g, 1e-10)


def test_noslip_walls_and_ragged_extents(orc, lib):
    """No-slip walls on x and y, periodic z, extents that are not multiples
    of the thread-block width; a sphere rising between the walls."""
    shape = (37, 29, 41)
    pos = np.array([18.2, 14.9, 12.4])
    o, g = make_pair(orc, lib, shape, tau=0.62, bc=("noslip", "noslip", "periodic"),
                     sphere=(pos, 8.0, 0.5, 0.5), gravity=(0, 0, -5e-5))
    o.step(120)
    g.step(120)
    assert_pops_close(o, g, 1e-10)
    assert np.array_equal(o.flags(), g.flags())
    assert_links_equal(o, g)


def test_body_force_fixed_rotating_sphere(orc, lib):
    """Fluid body force, fixed sphere spinning at a given angular velocity:
    exercises the forcing term and the omega x r wall velocity."""
    pos = np.array([10.4, 9.7, 10.1])
    o, g = make_pair(orc, lib, (20, 20, 20), tau=0.8, body_force=(1e-6, 2e-6, -1e-6), sphere=(pos, 8.0, 1.5, 0.0),
                     fixed=True, velocity=((0, 0, 0), (0.0, 0.0, 0.003)))
    o.step(100)
    g.step(100)
    assert_pops_close(o, g, 1e-10)
    p_o, p_g = o.particle(), g.particle()
    np.testing.assert_allclose(p_g[0:6], p_o[0:6], rtol=0, atol=1e-10 * np.abs(p_o[0:6]).max())


def test_fluid_only_and_degenerate_extents(orc, lib):
    """No sphere; 1-cell-thick periodic axes and a Poiseuille channel."""
    rng = np.random.default_rng(5)
    for shape, bc in [((1, 10, 1), ("periodic", "noslip", "periodic")), ((5, 1, 3), ("periodic",) * 3),
                      ((33, 2, 7), ("noslip", "periodic", "noslip"))]:
        o, g = make_pair(orc, lib, shape, tau=0.9, bc=bc, body_force=(1e-6, 0, 5e-7))
        g0 = rng.normal(scale=1e-4, size=(19, o.ncells))
        o.set_populations(g0)
        g.set_populations(g0)
        o.step(50)
        g.step(50)
        assert_pops_close(o, g, 1e-10)


def test_rest_state_gpu(lib):
    """Rest state stays at rest to rounding on every precision."""
    for prec in ("fp64", "fp32", "fp16"):
        s = lib.Simulation((32, 32, 32), precision=prec)
        s.add_sphere((16.2, 15.7, 16.4), 8.0, 0.5, cv=0.5)
        s.init_fluid()
        s.step(20)
        assert np.abs(s.populations()).max() < 1e-12
        assert np.abs(s.particle()[0:6]).max() < 1e-12


@pytest.mark.parametrize("precision,pop_rel,force_rel", [("fp32", 1e-5, 1e-4), ("fp16", 5e-3, 2e-2)])
def test_reduced_precision_against_oracle(orc, lib, precision, pop_rel, force_rel):
    """FP32 deviations and FP16 scaled deviations (FP32 arithmetic) against
    the FP64 oracle on the 32^3 single-sphere case after 100 steps."""
    w = workloads.SINGLE_SPHERE_32
    D, pi = w["diameter"], w["density_ratio"]
    gm = w["u_g"] ** 2 / (abs(pi - 1) * D)
    pos = np.array(w["shape"]) / 2 + workloads.sub_cell_offset(0)
    o, g = make_pair(orc, lib, w["shape"], precision=precision, tau=w["tau"], sphere=(pos, D, pi, w["cv"]),
                     gravity=(0, 0, -gm))
    o.step(100)
    g.step(100)
    assert_pops_close(o, g, pop_rel)
    Fscale = abs(pi - 1) * gm * np.pi * D ** 3 / 6
    ho, hg = o.history(), g.history()
    assert np.abs(hg[:, 0:3] - ho[:, 0:3]).max() <= force_rel * Fscale
    assert np.abs(hg[-1, 6:9] - ho[-1, 6:9]).max() < 1e-4


def test_uniform_flow_invariant_large(lib):
    """At the bandwidth-benchmark size (512^3, FP32): a uniform flow without
    a sphere is an exact fixed point of stream + collide, so every sampled
    cell keeps its equilibrium to FP32 rounding after 3 steps."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    if free < 30e9:
        pytest.skip("needs ~25 GB of device memory")
    s = lib.Simulation((512, 512, 512), precision="fp32")
    u = (0.02, -0.01, 0.005)
    s.init_fluid(1.0, u)
    s.step(3)
    cells = np.arange(0, s.ncells, 9973, dtype=np.int64)
    g = s.gather(cells).T
    from lattice_ref import C, W
    uu = np.dot(u, u)
    cu = C @ np.asarray(u)
    eq = W * (3 * cu + 4.5 * cu ** 2 - 1.5 * uu)
    assert np.abs(g - eq[:, None]).max() < 1e-7


@pytest.mark.parametrize("shape,bc,wall", [
    ((38, 29, 41), ("noslip", "noslip", "periodic"), None),      # even nx: two cells per thread, walls on x and y
    ((37, 29, 41), ("noslip", "noslip", "periodic"), None),      # odd nx: one cell per thread
    ((70, 24, 20), ("periodic", "periodic", "noslip"), (0.03, 0.01, 0.0)),   # a row longer than a warp's pairs, moving wall
])
def test_fp16_pairs_walls_against_oracle(orc, lib, shape, bc, wall):
    """FP16 storage on grids with walls and rows of any length: the update
    that reads aligned pairs of halves (even nx, shuffles across lanes, the
    last pair of each row and each warp loading its outer half) and the one
    cell per thread form (odd nx) both stay within the FP16 tolerance of the
    FP64 oracle, with a light sphere moving and, in the last case, the upper
    z wall moving."""
    pos = np.array(shape, dtype=float) / 2 + np.array([0.3, -0.4, 0.2])
    o, g = make_pair(orc, lib, shape, precision="fp16", tau=0.62, bc=bc, sphere=(pos, 8.0, 0.5, 0.5),
                     gravity=(0, 0, -5e-5))
    if wall is not None:
        o.set_wall_velocity(2, 1, wall)
        g.set_wall_velocity(2, 1, wall)
    o.step(120)
    g.step(120)
    assert_pops_close(o, g, 5e-3)
    Fscale = 0.5 * 5e-5 * np.pi * 8.0 ** 3 / 6
    assert np.abs(g.history()[:, 0:3] - o.history()[:, 0:3]).max() <= 2e-2 * Fscale * (10 if wall else 1)
