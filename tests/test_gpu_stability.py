"""Stability-limit study (Sec. 3.2, Table 1; virtual mass, Sec. 3.3) on the
GPU, through the public API: a qualitative pin against the paper's Table 1
(tests/golden/table1_pi_min_ga100.txt).

- the plain momentum exchange method (C_v = 0) has a lowest stable density
  ratio of the same order as Table 1 (within a factor 3) at d_p = 10 and 20,
  and it falls as the resolution grows;
- with the virtual-mass correction (C_v = 0.5) the sphere rises stably at
  pi_p = 0.001 (the paper's lightest case), far below that limit, at a
  plausible terminal velocity.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_pi_min_ga100.txt")


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2103_10882_gb300 as L
    L._native.load()
    return L


def table1():
    rows = np.loadtxt(GOLDEN)
    return {int(d): float(p) for d, p in rows}


def test_mem_limit_same_order_as_table1_and_falls_with_resolution(lib):
    from paper_2103_10882_gb300 import studies
    t = table1()
    lim = {}
    for d in (10, 20):
        stable, unstable, runs = studies.density_ratio_limit(lib, d, 0.0, t[d] / 4, t[d] * 4, iters=4)
        assert stable is not None and unstable is not None, runs
        assert unstable < stable
        lim[d] = stable
        assert t[d] / 3 <= stable <= 3 * t[d], (d, stable, t[d])
    assert lim[20] < lim[10]


def test_virtual_mass_stable_far_below_the_mem_limit(lib):
    from paper_2103_10882_gb300 import studies
    ok, done, uz = studies.rising_sphere_run(lib, 10, 0.001, 0.5)
    assert ok and done == 10000
    assert 0.8 < uz < 1.4
    ok_mem, _, _ = studies.rising_sphere_run(lib, 10, 0.001, 0.0)
    assert not ok_mem
