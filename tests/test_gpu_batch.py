"""Batched sweep: every simulation of a batch against the FP64 oracle run on
its own, and FP32 batches against single-simulation GPU runs."""
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


def small_batch(seed=0):
    """Uneven boxes, sphere size edge/6 rounded, pi_p and Ga drawn as in the sweep."""
    u = workloads.uniform01(seed, 5 * 4).reshape(4, 5)
    sims = []
    for i, e in enumerate((32, 16, 48, 32)):
        d = float(round(e / 6.0)) if e > 16 else 5.0
        pi = 0.1 + 0.8 * u[i, 0]
        ga = 100 + 300 * u[i, 1]
        nu = 0.01 * d / ga
        g = 0.01 ** 2 / (abs(pi - 1) * d)
        sims.append(dict(edge=e, pos=e / 2 + u[i, 2:5], diameter=d, density_ratio=pi, cv=0.5, tau=3 * nu + 0.5,
                         gravity=(0.0, 0.0, -g)))
    return sims


def test_batch_fp64_matches_oracle_per_simulation(orc, lib):
    sims = small_batch(0)
    b = lib.BatchSimulation(sims, precision="fp64")
    b.step(60)
    for i, s in enumerate(sims):
        e = s["edge"]
        o = orc.UniformSim((e, e, e), tau=s["tau"])
        o.add_sphere(s["pos"], s["diameter"], s["density_ratio"], cv=s["cv"])
        o.set_gravity(s["gravity"])
        o.init_equilibrium()
        o.step(60)
        go, gb = o.populations(), b.populations(i)
        assert np.abs(gb - go).max() <= 1e-10 * np.abs(go).max(), "simulation %d" % i
        ho, hb = o.history(), b.history(i)
        Fs = abs(s["density_ratio"] - 1) * abs(s["gravity"][2]) * np.pi * s["diameter"] ** 3 / 6
        assert np.abs(hb[:, 0:6] - ho[:, 0:6]).max() <= 1e-10 * Fs
        np.testing.assert_allclose(hb[:, 6:9], ho[:, 6:9], rtol=1e-10, atol=1e-10)


def test_batch_fp32_matches_single_runs_and_graphs(lib):
    """The batched kernels do the single-simulation arithmetic (up to FP32
    rounding: the two engines' boundary kernels are different code); odd
    step counts exercise the graph (two steps) and the plain path together.
    Forces, torques and accelerations are compared against the largest
    component of their group, positions and velocities relatively."""
    sims = small_batch(1)
    b = lib.BatchSimulation(sims, precision="fp32")
    b.autotune(3)
    info = b.info()
    assert info[0] == 4 and info[1] == sum(s["edge"] ** 3 for s in sims)
    b.step(7)
    b.step(6)
    for i, s in enumerate(sims):
        e = s["edge"]
        g = lib.Simulation((e, e, e), precision="fp32", tau=s["tau"])
        g.add_sphere(s["pos"], s["diameter"], s["density_ratio"], cv=s["cv"])
        g.set_gravity(s["gravity"])
        g.init_fluid()
        g.step(13)
        a, c = g.populations(), b.populations(i)
        assert np.abs(a - c).max() <= 1e-6 * max(np.abs(a).max(), 1e-12)
        pb, ps = b.particle(i), g.particle()
        for lo, hi in ((0, 3), (3, 6), (15, 18), (18, 21), (21, 24)):
            scale = max(np.abs(ps[lo:hi]).max(), 1e-30)
            assert np.abs(pb[lo:hi] - ps[lo:hi]).max() <= 1e-5 * scale, (lo, pb[lo:hi], ps[lo:hi])
        np.testing.assert_allclose(pb[6:9], ps[6:9], rtol=1e-9)
        np.testing.assert_allclose(pb[9:15], ps[9:15], rtol=1e-5, atol=1e-5 * np.abs(ps[9:15]).max())


def test_batch_rest_state_and_errors(lib):
    sims = [dict(edge=16, pos=(8.2, 7.9, 8.1), diameter=5.0, density_ratio=0.5, cv=0.5, tau=0.7)]
    b = lib.BatchSimulation(sims, precision="fp16")
    b.step(10)
    assert np.abs(b.populations(0)).max() < 1e-12
    bad = [dict(edge=20, pos=(10, 10, 10), diameter=5.0, density_ratio=0.5, tau=0.7)]
    with pytest.raises(lib.LbmpError):
        lib.BatchSimulation(bad)
