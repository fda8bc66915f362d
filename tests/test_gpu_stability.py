"""Stability-limit study (Sec. 3.2, Table 1; virtual mass, Sec. 3.3) on the
GPU, through the public API, with the paper's collision (MRT, bulk factor
100, Sec. 2.1): a pin against the paper's Table 1
(tests/golden/table1_pi_min_ga100.txt).

- the plain momentum exchange method (C_v = 0) has its lowest stable density
  ratio between 1.5 and 2.5 times Table 1's at d_p = 10 and 20 (the full
  study measured 1.7-2.0 times at every d_p from 10 to 40: the coupling
  details of the paper's own runs are not given), and it falls about as
  1/d_p, as in Table 1;
- every unstable run trips the force-oscillation criterion (the paper's
  growing force oscillations) no later than the status word;
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


def test_mem_limit_against_table1_and_falls_with_resolution(lib):
    from paper_2103_10882_gb300 import studies
    t = table1()
    lim = {}
    for d in (10, 20):
        stable, unstable, runs = studies.density_ratio_limit(lib, d, 0.0, t[d] / 4, t[d] * 4, iters=4)
        assert stable is not None and unstable is not None, runs
        assert unstable < stable
        lim[d] = stable
        assert 1.5 * t[d] <= stable <= 2.5 * t[d], (d, stable, t[d])
        for r in runs:
            if not r["stable"]:
                assert r["t_n_force"] is not None, r
                assert r["t_n_status"] is None or r["t_n_force"] <= r["t_n_status"], r
    assert 1.5 <= lim[10] / lim[20] <= 2.5


def test_virtual_mass_stable_far_below_the_mem_limit(lib):
    from paper_2103_10882_gb300 import studies
    r = studies.rising_sphere_run(lib, 10, 0.001, 0.5)
    assert r["stable"] and r["steps"] == 10000
    assert 0.8 < r["u_z_over_u_g"] < 1.4
    assert not studies.rising_sphere_run(lib, 10, 0.001, 0.0)["stable"]
