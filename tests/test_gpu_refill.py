"""GPU parity of the Grad refill of uncovered cells (Sec. 2.3, read as
Grad's approximation from the local strain rate) against the oracle, through
the C ABI: fast light spheres that uncover cells every few steps on a
uniform grid (FP64 within 1e-10, FP32 within 1e-5), on three refined levels
with regrids, and in an uneven batch; and that the option reaches the
kernels (the result differs from the equilibrium refill)."""
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


POS = (12.3, 11.8, 12.6)


def uniform_run(orc, lib, precision, refill, steps=40):
    o = orc.UniformSim((24, 24, 24), tau=0.6, refill=refill)
    g = lib.Simulation((24, 24, 24), precision=precision, tau=0.6, refill=refill)
    for s in (o, g):
        s.add_sphere(POS, 8.0, 0.2, cv=0.5)
        s.set_gravity((0, 0, -2e-3))
    o.init_equilibrium()
    g.init_fluid()
    o.step(steps)
    g.step(steps)
    return o, g


@pytest.mark.parametrize("precision,rel", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_uniform_grad_refill(orc, lib, precision, rel):
    o, g = uniform_run(orc, lib, precision, "grad")
    assert np.array_equal(o.flags(), g.flags())
    go, gg = o.populations(), g.populations()
    assert np.abs(gg - go).max() <= rel * np.abs(go).max()
    ho, hg = o.history(), g.history()
    assert hg[-1, 8] - hg[0, 8] > 0.5
    Fs = 0.8 * 2e-3 * math.pi * 512 / 6
    assert np.abs(hg[:, 0:6] - ho[:, 0:6]).max() <= 10 * rel * Fs
    g.close()


def test_refill_option_reaches_the_kernels(orc, lib):
    _, ge = uniform_run(orc, lib, "fp64", "equilibrium", steps=20)
    _, gg = uniform_run(orc, lib, "fp64", "grad", steps=20)
    assert np.abs(gg.populations() - ge.populations()).max() > 1e-8
    ge.close()
    gg.close()


def test_refined_grad_refill_with_regrids(orc, lib):
    pos = (30.3, 31.6, 42.6)
    o = orc.RefinedSim((32, 32, 48), 2, tau=0.6, refill="grad")
    g = lib.Simulation((32, 32, 48), precision="fp64", tau=0.6, levels=2, refill="grad")
    for s in (o, g):
        s.add_sphere(pos, 8.0, 0.2, cv=0.5)
        s.set_gravity((0, 0, -1e-2))
    o.init_equilibrium()
    g.init_fluid()
    for _ in range(6):
        o.step(1)
        g.step(1)
        o.regrid()
        g.regrid()
    for l in range(2):
        assert np.array_equal(o.block_map(l), g.block_map(l))
        xo, fo = o.real_cells(l)
        xg, fg = g.level_cells(l)
        assert np.array_equal(xo, xg)
        if len(fo):
            assert np.abs(fg - fo).max() <= 1e-10 * np.abs(fo).max(), "level %d" % l
    assert g.history()[-1, 8] - pos[2] > 0.5
    g.close()


def test_batch_grad_refill(orc, lib):
    sims = []
    for e, d, pi in ((32, 6.0, 0.2), (16, 4.0, 0.3)):
        sims.append(dict(edge=e, pos=(e / 2 + 0.31, e / 2 - 0.22, e / 2 + 0.13), diameter=d, density_ratio=pi,
                         cv=0.5, tau=0.6, gravity=(0.0, 0.0, -2e-3)))
    b = lib.BatchSimulation(sims, precision="fp64", refill="grad")
    b.step(30)
    for i, s in enumerate(sims):
        e = s["edge"]
        o = orc.UniformSim((e, e, e), tau=s["tau"], refill="grad")
        o.add_sphere(s["pos"], s["diameter"], s["density_ratio"], cv=s["cv"])
        o.set_gravity(s["gravity"])
        o.init_equilibrium()
        o.step(30)
        go, gb = o.populations(), b.populations(i)
        assert np.abs(gb - go).max() <= 1e-10 * np.abs(go).max(), "simulation %d" % i
        assert b.history(i)[-1, 8] - s["pos"][2] > 0.2
    b.close()
