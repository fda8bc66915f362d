"""Pins of the oracle's flow-based refinement sensor (Sec. 4.2.2).

phi_c = |curl u| s^((r+1)/r), r = 2, s the cell size in finest-level units,
the block's value the largest over its cells; a block asks for one level
finer above sigma_c, one level coarser below c sigma_c.  Pinned by:
- a linear velocity field, whose finite-difference curl is exact: every
  block of every level reads |curl A| s^1.5, and a symmetric A (pure strain)
  reads zero, which catches a swapped derivative or sign;
- numpy's gradient (second-order central inside, first-order one-sided at
  the ends), applied block by block to the oracle's own velocities;
- hand-derived block forests for uniform shears across the thresholds:
  refinement one level per regrid up to the finest level, the hysteresis
  band [c sigma_c, sigma_c] that keeps a level, and coarsening one level per
  regrid;
- a localised shear with a refined box: the forest stays 2:1 balanced and
  complete, no region moves by more than one level, and regions coarsen only
  where every block of their octet read below c sigma_c.
"""
import numpy as np
import pytest

from lattice_ref import C

SIGMA, CF = 1e-3, 0.2


def curl_norm(A):
    A = np.asarray(A, dtype=float).reshape(3, 3)
    return np.sqrt((A[2, 1] - A[1, 2]) ** 2 + (A[0, 2] - A[2, 0]) ** 2 + (A[1, 0] - A[0, 1]) ** 2)


def level_of_positions(sim, levels):
    """Level covering each finest-block position ([z, y, x] array)."""
    nbs = [tuple(v // 16 for v in sim.level_shape(l)) for l in range(levels)]
    nbf = nbs[-1]
    level = -np.ones((nbf[2], nbf[1], nbf[0]), dtype=int)
    for l in range(levels):
        f = 1 << (levels - 1 - l)
        real = sim.block_map(l).reshape(nbs[l][2], nbs[l][1], nbs[l][0]) >= 0
        up = np.repeat(np.repeat(np.repeat(real, f, 0), f, 1), f, 2)
        assert not np.any(level[up] >= 0)
        level[up] = l
    assert np.all(level >= 0)
    return level


def block_velocities(sim, level):
    """Velocity u = sum_q g_q c_q of every real block, [nblocks, 3, 16, 16, 16] (z, y, x)."""
    _, g = sim.real_cells(level)
    u = g @ C.astype(float)                     # [n, 3]
    nb = u.shape[0] // 4096
    return u.reshape(nb, 16, 16, 16, 3).transpose(0, 4, 1, 2, 3)


def test_linear_field_reads_exact_curl_on_every_level(orc):
    levels = 3
    s = orc.RefinedSim((32, 32, 32), levels, tau=0.55)
    s.refine_box((40.0, 40.0, 40.0), (72.0, 72.0, 72.0))   # three levels present
    rng = np.random.default_rng(7)
    A = rng.uniform(-1e-4, 1e-4, size=(3, 3))
    s.init_linear(A, u0=(1e-3, -2e-3, 5e-4), x0=(64.0, 64.0, 64.0))
    want = curl_norm(A)
    seen = 0
    for l in range(levels):
        phi = s.block_sensor(l)
        seen += phi.size
        h = float(1 << (levels - 1 - l))
        np.testing.assert_allclose(phi, want * h ** 1.5, rtol=1e-9, atol=0)
    assert seen > 0
    # pure strain: no rotation anywhere
    S = 0.5 * (A + A.T)
    s.init_linear(S, x0=(64.0, 64.0, 64.0))
    for l in range(levels):
        assert np.all(s.block_sensor(l) < 1e-9 * want)


def test_sensor_matches_numpy_gradient_blockwise(orc):
    levels = 2
    s = orc.RefinedSim((64, 64, 64), levels, tau=0.6)
    s.add_sphere((45.0, 46.5, 50.2), 10.0, 0.5, cv=0.5)
    s.set_gravity((0.0, 0.0, 2e-5))
    s.init_equilibrium(shear=3e-3, shear_dir=1, shear_axis=0)
    s.step(3)
    for l in range(levels):
        h = float(1 << (levels - 1 - l))
        U = block_velocities(s, l)
        want = []
        for b in range(U.shape[0]):
            # np.gradient on [z, y, x] arrays: axis 2 is x, 1 is y, 0 is z
            d = [[np.gradient(U[b, comp], h, axis=2 - ax, edge_order=1) for ax in range(3)] for comp in range(3)]
            w = np.stack([d[2][1] - d[1][2], d[0][2] - d[2][0], d[1][0] - d[0][1]])
            want.append(np.sqrt((w ** 2).sum(axis=0)).max() * h ** 1.5)
        got = s.block_sensor(l)
        assert got.size == len(want) > 0
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-18)
        assert np.max(got) > 0


def _all_at(sim, levels, lvl):
    return bool(np.all(level_of_positions(sim, levels) == lvl))


def test_uniform_shear_refines_then_coarsens_one_level_per_regrid(orc):
    """u_x = a z: |curl u| = a, phi = a s^1.5 with s = 4, 2, 1 on levels 0, 1, 2."""
    levels = 3
    s = orc.RefinedSim((32, 32, 32), levels, tau=0.55)
    s.set_sensor(SIGMA, CF)
    assert _all_at(s, levels, 0)

    def shear(a):
        s.init_linear([[0, 0, a], [0, 0, 0], [0, 0, 0]], x0=(0.0, 0.0, 64.0))

    shear(0.5 * SIGMA)            # phi_0 = 4 sigma > sigma
    s.regrid()
    assert _all_at(s, levels, 1)
    shear(0.5 * SIGMA)            # phi_1 = 1.41 sigma > sigma
    s.regrid()
    assert _all_at(s, levels, 2)
    shear(0.5 * SIGMA)            # phi_2 = 0.5 sigma: inside the band, kept
    s.regrid()
    assert _all_at(s, levels, 2)
    shear(0.15 * SIGMA)           # phi_2 = 0.15 sigma < c sigma: one level coarser
    s.regrid()
    assert _all_at(s, levels, 1)
    shear(0.15 * SIGMA)           # phi_1 = 0.42 sigma: kept
    s.regrid()
    assert _all_at(s, levels, 1)
    shear(0.02 * SIGMA)           # phi_1 = 0.057 sigma: coarser
    s.regrid()
    assert _all_at(s, levels, 0)
    shear(0.02 * SIGMA)           # phi_0 = 0.16 sigma: level 0 stays level 0
    s.regrid()
    assert _all_at(s, levels, 0)


def test_sensor_off_and_invalid_factor(orc):
    levels = 2
    s = orc.RefinedSim((32, 32, 32), levels, tau=0.55)
    s.init_linear([[0, 0, 1e-2], [0, 0, 0], [0, 0, 0]])
    s.regrid()                    # sensor off: nothing asks for refinement
    assert _all_at(s, levels, 0)
    with pytest.raises(RuntimeError):
        s.set_sensor(SIGMA, 0.36)     # c must stay below 2^-1.5
    with pytest.raises(RuntimeError):
        s.set_sensor(SIGMA, 0.0)


def _neighbours(nb, p):
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dx or dy or dz:
                    yield ((p[0] + dx) % nb[0], (p[1] + dy) % nb[1], (p[2] + dz) % nb[2])


def _check_forest(level, levels):
    nbf = level.shape[::-1]
    for z in range(nbf[2]):
        for y in range(nbf[1]):
            for x in range(nbf[0]):
                for c in _neighbours(nbf, (x, y, z)):
                    assert abs(level[z, y, x] - level[c[2], c[1], c[0]]) <= 1
    for l in range(1, levels):
        f = 1 << (levels - 1 - l)
        nz, ny, nx = (v // f for v in level.shape)
        cov = (level >= l).reshape(nz, f, ny, f, nx, f).all(axis=(1, 3, 5))
        oct_ = cov.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2).sum(axis=(1, 3, 5))
        assert np.all((oct_ == 0) | (oct_ == 8))


def test_localised_shear_keeps_forest_balanced(orc):
    levels = 3
    s = orc.RefinedSim((32, 32, 64), levels, tau=0.55)
    s.refine_box((20.0, 20.0, 20.0), (40.0, 40.0, 40.0))
    s.set_sensor(SIGMA, CF)
    rng = np.random.default_rng(3)
    changed_total = 0
    for rnd in range(4):
        amp = [2e-2, 8e-3, 2e-3, 1e-4][rnd]
        s.init_equilibrium(shear=amp, shear_dir=int(rng.integers(0, 2)), shear_axis=2)
        before = level_of_positions(s, levels)
        # per finest-block position: the demand of the block covering it
        nbf = before.shape[::-1]
        ask = np.zeros_like(before)
        octet_low = np.zeros_like(before, dtype=bool)
        for l in range(levels):
            f = 1 << (levels - 1 - l)
            nb = tuple(v // 16 for v in s.level_shape(l))
            m = s.block_map(l).reshape(nb[2], nb[1], nb[0])
            phi = s.block_sensor(l)
            t = np.full(m.shape, -1)
            low = np.zeros(m.shape, dtype=bool)
            real = m >= 0
            t[real] = np.where(phi[m[real]] > SIGMA, min(l + 1, levels - 1),
                               np.where(phi[m[real]] < CF * SIGMA, max(l - 1, 0), l))
            low[real] = phi[m[real]] < CF * SIGMA
            # octet of level-l blocks all low (positions of the parent)
            if l > 0:
                lo8 = low.reshape(nb[2] // 2, 2, nb[1] // 2, 2, nb[0] // 2, 2).all(axis=(1, 3, 5))
                low = np.repeat(np.repeat(np.repeat(lo8, 2, 0), 2, 1), 2, 2)
            up = lambda a: np.repeat(np.repeat(np.repeat(a, f, 0), f, 1), f, 2)
            sel = up(real)
            ask[sel] = up(t)[sel]
            octet_low[sel] = up(low)[sel]
        s.regrid()
        after = level_of_positions(s, levels)
        _check_forest(after, levels)
        assert np.all(after >= ask)                       # every wish met
        assert np.all(after <= np.maximum(before + 1, ask))
        assert np.all(after >= before - 1)                # one level per regrid
        assert np.all(~(after < before) | octet_low)      # coarsen only where the octet agreed
        # the refined box stays finest
        for z in range(1, 3):
            for y in range(1, 3):
                for x in range(1, 3):
                    assert after[z, y, x] == levels - 1
        changed_total += int(np.sum(after != before))
    assert changed_total > 0
