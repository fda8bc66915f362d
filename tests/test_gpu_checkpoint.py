"""Checkpoint and resume through the C ABI: a run saved part-way and
continued equals, bit for bit, a fresh handle that loads the file and
steps on (uniform grid with a moving sphere; refined grid with a moving
sphere, the curl sensor and periodic regrids); a different grid, a missing
file and batched handles are refused."""
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


def test_uniform_resume_is_exact(lib, tmp_path):
    path = str(tmp_path / "u.ckpt")
    a = lib.Simulation((32, 32, 32), precision="fp32", tau=0.6)
    a.add_sphere((16.3, 15.8, 16.4), 8.0, 0.3, cv=0.5)
    a.set_gravity((0, 0, -1e-3))
    a.set_body_force((1e-6, 0, 0))
    a.init_fluid()
    a.step(30)
    a.save(path)
    a.step(20)
    b = lib.Simulation((32, 32, 32), precision="fp32", tau=0.6)
    b.load(path)
    b.step(20)
    assert np.array_equal(a.populations(), b.populations())
    assert np.array_equal(a.flags(), b.flags())
    assert np.array_equal(a.particle(), b.particle())
    assert np.array_equal(a.history(), b.history())
    assert a.particle()[8] - 16.4 > 0.1       # the sphere moved, so the remap ran after the load
    a.close()
    b.close()


@pytest.mark.parametrize("levels,shape,pos,gz", [(2, (32, 32, 48), (30.3, 31.6, 40.6), -1e-2),
                                                 (3, (16, 16, 32), (30.7, 33.2, 60.6), -2e-3)])
def test_refined_resume_is_exact(lib, tmp_path, levels, shape, pos, gz):
    """Two and three levels: the loaded handle explodes its ghost cells and
    forms the sphere's frames again before its first step."""
    path = str(tmp_path / "r.ckpt")

    def make():
        s = lib.Simulation(shape, precision="fp32", tau=0.6, levels=levels, regrid_interval=3)
        s.set_refinement_sensor(1e-3, 0.2)
        return s

    a = make()
    a.add_sphere(pos, 8.0, 0.2, cv=0.5)
    a.set_gravity((0, 0, gz))
    a.init_fluid()
    a.step(7)
    a.save(path)
    a.step(8)
    b = make()
    b.load(path)
    b.step(8)
    for l in range(levels):
        assert np.array_equal(a.block_map(l), b.block_map(l))
        xa, ga = a.level_cells(l)
        xb, gb = b.level_cells(l)
        assert np.array_equal(xa, xb) and np.array_equal(ga, gb)
    assert np.array_equal(a.particle(), b.particle())
    a.close()
    b.close()


def test_refusals(lib, tmp_path):
    path = str(tmp_path / "x.ckpt")
    a = lib.Simulation((32, 32, 32), precision="fp32")
    a.init_fluid()
    a.save(path)
    with pytest.raises(lib.LbmpError):
        lib.Simulation((32, 32, 16), precision="fp32").load(path)
    with pytest.raises(lib.LbmpError):
        lib.Simulation((32, 32, 32), precision="fp64").load(path)
    with pytest.raises(lib.LbmpError):
        a.load(str(tmp_path / "missing.ckpt"))
    sims = [dict(edge=16, pos=(8.2, 7.9, 8.1), diameter=4.0, density_ratio=0.5, cv=0.5, tau=0.6,
                 gravity=(0.0, 0.0, -1e-5))]
    bs = lib.BatchSimulation(sims)
    with pytest.raises(lib.LbmpError):
        lib.lbmp_save(bs.h, path)
    bs.close()
    a.close()
