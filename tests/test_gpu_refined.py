"""GPU parity of the refined-grid engine against the refined oracle.

Integer work (block maps, boundary links) is compared bit-exactly; FP64
populations within 1e-10 of their largest magnitude, forces within 1e-10 of
the buoyancy scale; FP32 with the tolerances stated per test.  All calls go
through the C ABI.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2103_10882_gb300 as L
    L._native.load()
    return L


def pair(orc, lib, shape, levels, tau, precision="fp64", rescale=False, bc=("periodic",) * 3, box=None,
         sphere=None, gravity=(0, 0, 0)):
    periodic = tuple(1 if b == "periodic" else 0 for b in bc)
    o = orc.RefinedSim(shape, levels, tau=tau, periodic=periodic, rescale=rescale)
    g = lib.Simulation(shape, precision=precision, tau=tau, bc=bc, levels=levels, rescale=rescale)
    if box is not None:
        o.refine_box(*box)
        g.refine_box(*box)
    if sphere is not None:
        pos, D, pi, cv = sphere
        o.add_sphere(pos, D, pi, cv=cv)
        g.add_sphere(pos, D, pi, cv=cv)
        o.set_gravity(gravity)
        g.set_gravity(gravity)
    return o, g


def same_maps(o, g, levels):
    for l in range(levels):
        assert o.level_shape(l) == g.level_shape(l)
        assert np.array_equal(o.block_map(l), g.block_map(l)), "block map of level %d differs" % l


def same_integer_work(o, g, levels):
    """Block maps, finest-level flags (solid, next to the sphere, fluid) and
    the boundary links bit-exact; link wall distances within 1e-12."""
    same_maps(o, g, levels)
    f = levels - 1
    assert np.array_equal(o.flags(), g.level_flags(f)), "finest-level flags differ"
    oc, oq, od = o.links()
    gc, gq, gd = g.links()
    a, b = np.lexsort((oq, oc)), np.lexsort((gq, gc))
    assert np.array_equal(oc[a], gc[b]) and np.array_equal(oq[a], gq[b]), "boundary links differ"
    if len(od):
        assert np.abs(od[a] - gd[b]).max() < 1e-12


def cells_close(o, g, levels, rel):
    for l in range(levels):
        xo, fo = o.real_cells(l)
        xg, fg = g.level_cells(l)
        assert np.array_equal(xo, xg)
        if len(fo):
            scale = max(np.abs(fo).max(), 1e-300)
            err = np.abs(fg - fo).max() / scale
            assert err <= rel, "level %d: population error %.3e > %.1e" % (l, err, rel)


@pytest.mark.parametrize("levels,shape", [(2, (32, 32, 48)), (3, (48, 48, 64))])
def test_box_refinement_shear_fp64(orc, lib, levels, shape):
    """Box refinement (edges and corners), shear wave plus drift: block maps
    bit-exact, populations of every level within 1e-10 after a few coarse steps."""
    f = 1 << (levels - 1)
    box = ((9 * f, 13 * f, 15 * f), (21 * f, 19 * f, 29 * f))
    o, g = pair(orc, lib, shape, levels, tau=0.8, box=box)
    same_maps(o, g, levels)
    o.init_equilibrium(u=(0.01, 0.004, -0.007), shear=0.01, shear_dir=0, shear_axis=2)
    g.init_fluid_wave(1.0, (0.01, 0.004, -0.007), 0.01, 0, 2)
    cells_close(o, g, levels, 1e-12)
    steps = 3 if levels == 3 else 5
    o.step(steps)
    g.step(steps)
    cells_close(o, g, levels, 1e-10)


def test_uniform_flow_and_conservation_gpu(lib):
    """Uniform flow stays exact on every level; with the plain transfer the
    GPU conserves mass and momentum of a shear wave to rounding."""
    shape, levels = (32, 32, 48), 2
    g = lib.Simulation(shape, precision="fp64", tau=0.7, levels=levels)
    g.refine_box((18, 26, 30), (42, 38, 58))
    u = np.array([0.02, -0.01, 0.005])
    g.init_fluid(1.0, u)
    g.step(3)
    from lattice_ref import C, W
    cu = C @ u
    e = W * (3 * cu + 4.5 * cu ** 2 - 1.5 * u @ u)
    for l in range(levels):
        _, f = g.level_cells(l)
        assert np.abs(f - e[None, :]).max() < 2e-16
    g2 = lib.Simulation((48, 48, 64), precision="fp64", tau=0.8, levels=levels)
    g2.refine_box((18, 26, 30), (42, 38, 58))
    g2.init_fluid_wave(1.0, (0.01, 0.004, -0.007), 0.01, 0, 2)

    def totals():
        m, p, s = [], [[], [], []], []
        for l in range(levels):
            _, f = g2.level_cells(l)
            vol = 8.0 ** (levels - 1 - l)
            m.extend((f.sum(axis=1) * vol).tolist())
            for k in range(3):
                mk = (f @ C[:, k].astype(float)) * vol
                p[k].extend(mk.tolist())
                s.extend(np.abs(mk).tolist())
        return math.fsum(m), np.array([math.fsum(v) for v in p]), math.fsum(s)

    m0, p0, scale = totals()
    g2.step(4)
    m1, p1, _ = totals()
    assert abs(m1 - m0) < 1e-14 * scale
    assert np.abs(p1 - p0).max() < 1e-14 * scale


@pytest.mark.parametrize("levels,shape,box0,box1", [
    (2, (32, 32, 48), ((18, 26, 30), (42, 38, 58)), ((40, 10, 50), (60, 40, 90))),
    (3, (32, 32, 64), ((36, 44, 40), (84, 76, 92)), ((20, 24, 150), (60, 56, 200))),
])
def test_rescaled_regrid_parity(orc, lib, levels, shape, box0, box1):
    """The non-equilibrium rescaling of cells that change level in a regrid
    (kappa per TRT part when refined, 1/kappa when coarsened) follows the
    oracle: a shear wave with drift, three steps, a regrid that both refines
    and coarsens, then two more steps."""
    o, g = pair(orc, lib, shape, levels, tau=0.8, rescale=True, box=box0)
    o.init_equilibrium(u=(0.01, 0.0, 0.0), shear=0.01, shear_dir=0, shear_axis=2)
    g.init_fluid_wave(1.0, (0.01, 0.0, 0.0), 0.01, 0, 2)
    o.step(3)
    g.step(3)
    before = [o.block_map(l).copy() for l in range(levels)]
    o.refine_box(*box1)
    g.refine_box(*box1)
    after = [o.block_map(l) for l in range(levels)]
    f = levels - 1
    assert np.any((before[f] >= 0) & (after[f] < 0)) and np.any((before[f] < 0) & (after[f] >= 0))
    same_maps(o, g, levels)
    cells_close(o, g, levels, 1e-12)
    o.step(2)
    g.step(2)
    cells_close(o, g, levels, 1e-10)


def test_refined_sphere_fp64(orc, lib):
    """Three levels around a light sphere (d = 10 finest cells): maps, links,
    populations and the particle history against the oracle."""
    pos = (30.7, 33.2, 31.6)
    o, g = pair(orc, lib, (16, 16, 16), 3, tau=0.7, sphere=(pos, 10.0, 0.3, 0.5), gravity=(0, 0, -2e-4))
    same_maps(o, g, 3)
    o.init_equilibrium()
    g.init_fluid()
    o.step(3)
    g.step(3)
    same_maps(o, g, 3)
    cells_close(o, g, 3, 1e-10)
    ho, hg = o.history(), g.history()
    assert ho.shape == hg.shape == (12, 15)
    Fs = 0.7 * 2e-4 * math.pi * 1000 / 6
    np.testing.assert_allclose(hg[:, 0:6], ho[:, 0:6], rtol=0, atol=1e-10 * Fs)
    np.testing.assert_allclose(hg[:, 6:9], ho[:, 6:9], rtol=1e-10, atol=1e-10)
    same_integer_work(o, g, 3)
    assert len(g.links()[0]) > 0


def test_host_changes_between_steps_fp64(orc, lib):
    """The host changes the particle record between steps (a new sphere
    velocity) and then the fluid (re-initialised): the next steps re-form the
    sphere's frames and explode the active ghost cells again, and stay
    within 1e-10 of the oracle doing the same on three levels."""
    pos = (30.7, 33.2, 31.6)
    o, g = pair(orc, lib, (16, 16, 16), 3, tau=0.7, sphere=(pos, 10.0, 0.3, 0.5), gravity=(0, 0, -2e-4))
    o.init_equilibrium()
    g.init_fluid()
    o.step(2)
    g.step(2)
    u, w = (0.012, -0.02, 0.015), (0.001, 0.0, -0.002)
    o.set_particle_velocity(u, w)
    g.set_particle_velocity(u, w)
    o.step(2)
    g.step(2)
    cells_close(o, g, 3, 1e-10)
    same_integer_work(o, g, 3)
    o.init_equilibrium()
    g.init_fluid()
    o.step(2)
    g.step(2)
    cells_close(o, g, 3, 1e-10)
    same_integer_work(o, g, 3)
    ho, hg = o.history(), g.history()
    assert ho.shape == hg.shape == (24, 15)
    Fs = 0.7 * 2e-4 * math.pi * 1000 / 6
    np.testing.assert_allclose(hg[:, 0:6], ho[:, 0:6], rtol=0, atol=1e-10 * Fs)
    np.testing.assert_allclose(hg[:, 6:15], ho[:, 6:15], rtol=1e-10, atol=1e-10)


def test_moving_sphere_with_regrids(orc, lib):
    """A fast light sphere crosses block boundaries; both sides regrid every
    coarse step: block maps stay bit-exact and populations within 1e-10."""
    pos = (30.3, 31.6, 42.6)   # bounding box (+1 cell) ends 0.4 cells below a block boundary
    o, g = pair(orc, lib, (32, 32, 48), 2, tau=0.6, sphere=(pos, 8.0, 0.2, 0.5), gravity=(0, 0, -1e-2))
    o.init_equilibrium()
    g.init_fluid()
    maps0 = [g.block_map(l).copy() for l in range(2)]
    for step in range(8):
        o.step(1)
        g.step(1)
        o.regrid()
        g.regrid()
        same_integer_work(o, g, 2)
    cells_close(o, g, 2, 1e-10)
    ho, hg = o.history(), g.history()
    np.testing.assert_allclose(hg[:, 6:9], ho[:, 6:9], rtol=1e-10, atol=1e-10)
    assert hg[-1, 8] - pos[2] > 0.5   # it rose ...
    assert any(not np.array_equal(maps0[l], g.block_map(l)) for l in range(2))   # ... and the grid followed


def test_refined_fp32_against_fp64_oracle(orc, lib):
    """FP32 deviations on three levels against the FP64 oracle."""
    pos = (30.7, 33.2, 31.6)
    o, g = pair(orc, lib, (16, 16, 16), 3, tau=0.7, precision="fp32", sphere=(pos, 10.0, 0.3, 0.5),
                gravity=(0, 0, -2e-4))
    o.init_equilibrium()
    g.init_fluid()
    o.step(3)
    g.step(3)
    cells_close(o, g, 3, 1e-4)
    ho, hg = o.history(), g.history()
    Fs = 0.7 * 2e-4 * math.pi * 1000 / 6
    assert np.abs(hg[:, 0:3] - ho[:, 0:3]).max() < 1e-3 * Fs


def test_refined_walls(orc, lib):
    """No-slip walls on x and y (as in the rising-sphere channel) with a box
    refinement touching nothing but the interior."""
    o, g = pair(orc, lib, (32, 32, 48), 2, tau=0.75, bc=("noslip", "noslip", "periodic"),
                box=((20, 20, 30), (44, 44, 60)))
    same_maps(o, g, 2)
    o.init_equilibrium(u=(0.0, 0.0, 0.01), shear=0.01, shear_dir=2, shear_axis=0)
    g.init_fluid_wave(1.0, (0.0, 0.0, 0.01), 0.01, 2, 0)
    o.step(4)
    g.step(4)
    cells_close(o, g, 2, 1e-10)


def test_refined_fp16_against_fp64_oracle(orc, lib):
    """FP16 deviation storage (2^11-scaled, FP32 arithmetic) on three levels
    against the FP64 oracle: populations within 5e-3 of their largest
    magnitude, forces within 2e-2 of the buoyancy scale."""
    pos = (30.7, 33.2, 31.6)
    o, g = pair(orc, lib, (16, 16, 16), 3, tau=0.7, precision="fp16", sphere=(pos, 10.0, 0.3, 0.5),
                gravity=(0, 0, -2e-4))
    o.init_equilibrium()
    g.init_fluid()
    o.step(3)
    g.step(3)
    cells_close(o, g, 3, 5e-3)
    ho, hg = o.history(), g.history()
    Fs = 0.7 * 2e-4 * math.pi * 1000 / 6
    assert np.abs(hg[:, 0:3] - ho[:, 0:3]).max() < 2e-2 * Fs


def test_long_rising_sphere_run_stays_sane(lib):
    """The headline workload (64x64x256 level 0, three levels, d = 20, Ga = 200,
    pi_p = 0.5, regrid every 50 level-0 steps with the particle criterion and
    the curl sensor) for its full 5000 level-0 steps: the status word stays
    clean, the record stays finite, the sphere keeps rising with a small
    lateral drift, the history is continuous (no step jumps more than the
    velocity allows), and the sensor keeps the wake refined (the finer levels
    hold more blocks than the sphere alone asks for)."""
    import bench
    w = bench.REFINED
    sim = bench.refined_sim(lib, "fp32", history_capacity=1 << 15)
    start = bench.refined_start(w["shape"], w["levels"], w["diameter"])
    first = [int((sim.block_map(l) >= 0).sum()) for l in range(w["levels"])]
    grew = False
    for _ in range(50):
        sim.step(100)   # checks the status word
        now = [int((sim.block_map(l) >= 0).sum()) for l in range(w["levels"])]
        grew |= now[-1] > first[-1]
    p = sim.particle()
    assert np.all(np.isfinite(p))
    h = sim.history()
    assert len(h) == 20000 and np.all(np.isfinite(h))
    assert h[-1, 8] > start[2] + 100.0 and h[-1, 11] > 0.01       # rose at about the terminal velocity
    assert np.abs(np.diff(h[:, 6:9], axis=0)).max() < 0.1         # continuous path
    assert abs(h[-1, 6] - start[0]) < 10.0 and abs(h[-1, 7] - start[1]) < 10.0
    assert grew
    sim.close()


def test_sensor_regrids_walls_100_finest_steps_fp64(orc, lib):
    """Three levels, no-slip walls on x and y, a light sphere (d = 10) and
    the curl sensor (sigma_c = 1e-5, c = 0.2): 25 level-0 steps (100
    finest steps) with a regrid every 5, three of which change the forest
    through the sensor and the sphere.  After every regrid the maps, the
    finest-level flags and the boundary links are bit-exact; at the end the
    populations of every level are within 1e-10 and the force history within
    1e-10 of the buoyancy scale.  Before each regrid the oracle's block
    values are checked to stay clear of the thresholds, so the FP64 maps are
    decided the same way on both sides."""
    sigma, cfac = 1e-5, 0.2
    pos, D, pi, gz = (62.3, 65.6, 90.2), 10.0, 0.3, 1e-3
    o, g = pair(orc, lib, (32, 32, 96), 3, tau=0.7, bc=("noslip", "noslip", "periodic"), sphere=(pos, D, pi, 0.5),
                gravity=(0, 0, gz))
    o.set_sensor(sigma, cfac)
    g.set_refinement_sensor(sigma, cfac)
    o.init_equilibrium()
    g.init_fluid()
    same_integer_work(o, g, 3)
    changed = 0
    for k in range(5):
        o.step(5)
        g.step(5)
        vals = np.concatenate([o.block_sensor(l) for l in range(3)])
        for thr in (sigma, cfac * sigma):
            assert np.abs(vals / thr - 1).min() > 1e-6
        before = [o.block_map(l).copy() for l in range(3)]
        o.regrid()
        g.regrid()
        changed += any(not np.array_equal(before[l], o.block_map(l)) for l in range(3))
        same_integer_work(o, g, 3)
    assert changed >= 3
    assert all(len(o.real_cells(l)[0]) > 0 for l in range(3))
    cells_close(o, g, 3, 1e-10)
    ho, hg = o.history(), g.history()
    assert ho.shape == hg.shape == (100, 15)
    Fs = (1 - pi) * gz * math.pi * D ** 3 / 6
    np.testing.assert_allclose(hg[:, 0:6], ho[:, 0:6], rtol=0, atol=1e-10 * Fs)
    np.testing.assert_allclose(hg[:, 6:9], ho[:, 6:9], rtol=1e-10, atol=1e-10)


def test_headline_size_fp64(orc, lib):
    """The bench's refined workload at its full size (level-0 64x64x256 in
    16^3 blocks, three levels, d = 20 finest cells, pi_p = 0.5, Ga = 200,
    walls on x and y, curl sensor on), built by the bench's own helper and
    stepped in the launch configuration the bench times (CUDA graphs of two
    level-0 steps, the coarser levels on their own streams), in the FP64
    path: after three level-0 steps (twelve coupled finest sub-steps) the
    block maps, finest flags and links are bit-exact with the oracle on the
    host cores and every population of every level is within 1e-10."""
    import os
    import bench
    w = bench.REFINED
    tau, gm = bench.ga_tau_g(w["ga"], w["u_g"], w["diameter"], w["density_ratio"])
    orc.set_threads(os.cpu_count() or 1)
    o = orc.RefinedSim(w["shape"], w["levels"], tau=tau, periodic=(0, 0, 1))
    o.add_sphere(bench.refined_start(w["shape"], w["levels"], w["diameter"]), w["diameter"], w["density_ratio"],
                 cv=w["cv"])
    o.set_gravity((0, 0, -gm))
    o.set_sensor(*w["sensor"])
    o.init_equilibrium()
    g = bench.refined_sim(lib, "fp64")
    o.step(3)
    g.step(3)
    same_integer_work(o, g, w["levels"])
    cells_close(o, g, w["levels"], 1e-10)
    ho, hg = o.history(), g.history()
    assert ho.shape == hg.shape == (12, 15)
    Fg = abs(w["density_ratio"] - 1) * gm * math.pi * w["diameter"] ** 3 / 6
    np.testing.assert_allclose(hg[:, 0:6], ho[:, 0:6], rtol=0, atol=1e-10 * Fg)
    np.testing.assert_allclose(hg[:, 6:15], ho[:, 6:15], rtol=1e-10, atol=1e-12)
    o.close()
    g.close()
