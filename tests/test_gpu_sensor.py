"""GPU parity of the flow-based refinement sensor (Sec. 4.2.2) against the
refined oracle, through the C ABI.

The per-block scaled curl is compared with the oracle's (FP64 within 1e-9
relative, FP32 within 1e-3 of the largest value); the block maps after
sensor-driven regrids are compared bit-exactly on cases whose block values
stay clear of the thresholds (checked on the oracle's values first), and the
populations after the migration within 1e-10.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SIGMA, CF = 1e-3, 0.2


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2103_10882_gb300 as L
    L._native.load()
    return L


def pair(orc, lib, shape, levels, tau, precision="fp64", box=None, sphere=None, gravity=(0, 0, 0),
         regrid_interval=0):
    o = orc.RefinedSim(shape, levels, tau=tau)
    g = lib.Simulation(shape, precision=precision, tau=tau, levels=levels, regrid_interval=regrid_interval)
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
        assert np.array_equal(o.block_map(l), g.block_map(l)), "block map of level %d differs" % l


def cells_close(o, g, levels, rel):
    for l in range(levels):
        xo, fo = o.real_cells(l)
        xg, fg = g.level_cells(l)
        assert np.array_equal(xo, xg)
        if len(fo):
            err = np.abs(fg - fo).max() / max(np.abs(fo).max(), 1e-300)
            assert err <= rel, "level %d: population error %.3e > %.1e" % (l, err, rel)


def clear_of_thresholds(o, levels, margin=1e-6):
    for l in range(levels):
        phi = o.block_sensor(l)
        for t in (SIGMA, CF * SIGMA):
            assert np.all(np.abs(phi / t - 1.0) > margin), "a block value sits on a threshold; pick another case"


def test_block_sensor_values_fp64_and_fp32(orc, lib):
    levels = 2
    for precision, rel in (("fp64", 1e-9), ("fp32", 1e-3)):
        o, g = pair(orc, lib, (64, 64, 64), levels, tau=0.6, precision=precision,
                    sphere=((45.0, 46.5, 50.2), 10.0, 0.5, 0.5), gravity=(0, 0, 2e-5))
        o.init_equilibrium(shear=3e-3, shear_dir=1, shear_axis=0)
        g.init_fluid_wave(1.0, (0.0, 0.0, 0.0), 3e-3, 1, 0)
        o.step(3)
        g.step(3)
        for l in range(levels):
            po, pg = o.block_sensor(l), g.block_sensor(l)
            assert po.shape == pg.shape and po.size > 0
            scale = po.max()
            assert scale > 0
            if precision == "fp64":
                np.testing.assert_allclose(pg, po, rtol=rel, atol=1e-12 * scale)
            else:
                assert np.abs(pg - po).max() <= rel * scale
        g.close()


def test_sensor_regrids_match_oracle_fp64(orc, lib):
    """A refined box plus shear waves of falling amplitude: the sensor
    refines, keeps and coarsens blocks; block maps bit-exact after each
    regrid, populations within 1e-10 after the migrations and a few steps."""
    levels = 3
    o, g = pair(orc, lib, (32, 32, 64), levels, tau=0.55, box=((20.0, 20.0, 20.0), (40.0, 40.0, 40.0)))
    o.set_sensor(SIGMA, CF)
    g.set_refinement_sensor(SIGMA, CF)
    maps = []
    for k, amp in enumerate([2e-2, 8e-3, 2.1e-3, 1e-4]):
        d = k % 2
        o.init_equilibrium(u=(0.0, 0.0, 0.002), shear=amp, shear_dir=d, shear_axis=2)
        g.init_fluid_wave(1.0, (0.0, 0.0, 0.002), amp, d, 2)
        clear_of_thresholds(o, levels)
        o.regrid()
        g.regrid()
        same_maps(o, g, levels)
        maps.append([g.block_map(l).copy() for l in range(levels)])
        cells_close(o, g, levels, 1e-12)
        o.step(2)
        g.step(2)
        cells_close(o, g, levels, 1e-10)
    # the forest did change between rounds
    assert any(not np.array_equal(maps[i][l], maps[i + 1][l]) for i in range(3) for l in range(levels))


def test_periodic_sensor_regrid_without_sphere(orc, lib):
    """regrid_interval = 2 with the sensor on and no sphere: the engine regrids
    on its own after two level-0 steps, like the oracle's explicit regrid."""
    levels = 2
    o, g = pair(orc, lib, (32, 32, 48), levels, tau=0.6, regrid_interval=2)
    o.set_sensor(SIGMA, CF)
    g.set_refinement_sensor(SIGMA, CF)
    o.init_equilibrium(shear=1e-2, shear_dir=0, shear_axis=2)
    g.init_fluid_wave(1.0, (0.0, 0.0, 0.0), 1e-2, 0, 2)
    before = g.block_map(1).copy()
    o.step(2)
    clear_of_thresholds(o, levels)
    o.regrid()
    g.step(2)
    same_maps(o, g, levels)
    assert not np.array_equal(before, g.block_map(1))
    cells_close(o, g, levels, 1e-10)


def test_sensor_argument_checks(lib):
    g = lib.Simulation((32, 32, 32), precision="fp32", tau=0.6, levels=2)
    with pytest.raises(lib.LbmpError):
        g.set_refinement_sensor(SIGMA, 0.36)
    with pytest.raises(lib.LbmpError):
        g.set_refinement_sensor(-1.0, 0.2)
    with pytest.raises(lib.LbmpError):
        g.block_sensor(5)
    g.set_refinement_sensor(0.0, 0.0)          # off
    g.close()
    u = lib.Simulation((32, 32, 32), precision="fp32", tau=0.6)
    with pytest.raises(lib.LbmpError):
        u.set_refinement_sensor(SIGMA, CF)
    u.close()
