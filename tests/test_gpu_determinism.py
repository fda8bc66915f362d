"""Run-to-run determinism of the refined step through the C ABI.

The refined step runs kernels side by side on three streams: the boundary
kernel beside the finest update, the remap after every second finest
sub-step beside the coarser levels' update, and the explosion into level 1
beside the first finest sub-steps.  Its force sums are fixed-order (per-lane
TwoSum sums, block sums in a fixed tree, a last-block hand-off).  Two fresh
handles that run the same case must therefore agree bit for bit: the
populations of every level, the block layout after regrids, the particle
record and the force history.  A race between the streams, or an order that
depends on scheduling, would show as a difference.
"""
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


def _run(lib, precision, levels, steps):
    s = lib.Simulation((32, 32, 48), precision=precision, tau=0.6, levels=levels, regrid_interval=4,
                       history_capacity=4096)
    s.set_refinement_sensor(1e-3, 0.2)
    f = 1 << (levels - 1)
    s.add_sphere((16.0 * f + 0.31, 16.0 * f - 0.22, 12.0 * f + 0.4), 10.0, 0.3, cv=0.5)
    s.set_gravity((0, 0, -2e-3))
    s.set_particle_velocity((1e-3, -5e-4, 0.0))
    s.init_fluid()
    s.step(steps)
    out = {
        "maps": [s.block_map(l).copy() for l in range(levels)],
        "cells": [s.level_cells(l) for l in range(levels)],
        "particle": s.particle(),
        "history": s.history(),
    }
    s.close()
    return out


@pytest.mark.parametrize("precision,levels", [("fp32", 3), ("fp64", 3), ("fp32", 2), ("fp16", 3)])
def test_refined_runs_are_bitwise_identical(lib, precision, levels):
    steps = 13   # odd: graph replays and a plain step; three regrids
    a = _run(lib, precision, levels, steps)
    b = _run(lib, precision, levels, steps)
    for l in range(levels):
        assert np.array_equal(a["maps"][l], b["maps"][l]), "level %d layout" % l
        xa, ga = a["cells"][l]
        xb, gb = b["cells"][l]
        assert np.array_equal(xa, xb), "level %d cells" % l
        assert np.array_equal(ga, gb), "level %d populations" % l
    assert np.array_equal(a["particle"], b["particle"])
    assert np.array_equal(a["history"], b["history"])
    # the case exercised the moving-sphere path: the sphere left its start by more than a cell's hundredth
    f = 1 << (levels - 1)
    start = np.array([16.0 * f + 0.31, 16.0 * f - 0.22, 12.0 * f + 0.4])
    assert np.abs(a["particle"][6:9] - start).max() > 1e-2
