"""Seeded synthetic inputs shared by the tests, the bench and the oracle runs.

Holds only random-number generation and the workload parameters (sizes,
diameters, density ratios, Galileo numbers); none of the method's
arithmetic lives here.  SplitMix64 follows its published definition
(Steele, Lea & Flood 2014): state += 0x9E3779B97F4A7C15, then the
xor-shift-multiply finaliser.
"""
import numpy as np

_MASK = (1 << 64) - 1


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n successive 64-bit outputs of SplitMix64 started at `seed`."""
    out = np.empty(n, dtype=np.uint64)
    s = seed & _MASK
    for i in range(n):
        s = (s + 0x9E3779B97F4A7C15) & _MASK
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        out[i] = z ^ (z >> 31)
    return out


def uniform01(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def sub_cell_offset(seed: int) -> np.ndarray:
    """Seeded uniform sub-cell offset in [0, 1)^3."""
    return uniform01(seed, 3)


# Workload parameters (lattice units).  "u_g = 0.01" is the paper's fixed
# gravitational velocity (Sec. 3.1 and Sec. 5.1); Ga and pi_p set g and nu.
SINGLE_SPHERE_32 = dict(shape=(32, 32, 32), diameter=8.0, density_ratio=0.5, cv=0.5, tau=0.6, magic=3.0 / 16.0,
                        ga=100.0, u_g=0.01, steps=200)

# Uniform stand-in for the rising-sphere runs used for bandwidth measurement:
# a periodic 512^3 box with one light sphere of 40 cells, like the finest
# level around the sphere in the large refined run.
ROOFLINE_512 = dict(shape=(512, 512, 512), diameter=40.0, density_ratio=0.5, cv=0.5, ga=200.0, u_g=0.01)

# Batched sweep: 64 independent cubic periodic boxes.
BATCH_EDGES = (32, 48, 64, 96)


def batch_sweep(seed: int = 0, count: int = 64):
    """Seeded (edge, diameter, density ratio, Ga, offset) for the batched sweep."""
    u = uniform01(seed, 6 * count).reshape(count, 6)
    sims = []
    for i in range(count):
        edge = BATCH_EDGES[min(int(u[i, 0] * len(BATCH_EDGES)), len(BATCH_EDGES) - 1)]
        sims.append(dict(edge=edge, diameter=float(round(edge / 6.0)), density_ratio=0.1 + 0.8 * u[i, 1],
                         ga=100.0 + 300.0 * u[i, 2], offset=u[i, 3:6].copy()))
    return sims


# Differentiation workload: periodic 64^3 box, sphere of 12 cells held fixed
# near the centre, fluid body force g_x = 1e-6, initial velocity from
# divergence-free Fourier modes |k| <= 4 of amplitude 1e-3, 500 steps with a
# checkpoint every 50.  tau is not fixed by the workload; 0.6 is used.
ADJOINT_64 = dict(shape=(64, 64, 64), diameter=12.0, tau=0.6, magic=3.0 / 16.0, body_force=1e-6, kmax=4,
                  amplitude=1e-3, steps=500, checkpoint=50)


def fourier_velocity_field(shape, kmax: float, amplitude: float, seed: int) -> np.ndarray:
    """Seeded divergence-free velocity field (3, nz, ny, nx) at the cell
    centres: a sum over the integer wave vectors 0 < |k| <= kmax (one of each
    +-k pair) of a_k cos(2 pi k.x / L) + b_k sin(2 pi k.x / L), with a_k and b_k
    uniform in [-1, 1]^3 projected normal to k / L, scaled so that the largest
    speed on the grid equals `amplitude`."""
    nx, ny, nz = (int(v) for v in shape)
    r = int(np.floor(kmax))
    modes = []
    for kx in range(-r, r + 1):
        for ky in range(-r, r + 1):
            for kz in range(-r, r + 1):
                k = (kx, ky, kz)
                if k == (0, 0, 0) or kx * kx + ky * ky + kz * kz > kmax * kmax:
                    continue
                first = next(v for v in k if v != 0)
                if first > 0:
                    modes.append(k)
    coef = 2.0 * uniform01(seed, 6 * len(modes)).reshape(len(modes), 2, 3) - 1.0
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    u = np.zeros((3, nz, ny, nx))
    for m, (kx, ky, kz) in enumerate(modes):
        kv = np.array([kx / nx, ky / ny, kz / nz])
        phase = 2.0 * np.pi * (kv[0] * x + kv[1] * y + kv[2] * z)
        c, s = np.cos(phase), np.sin(phase)
        for j, wave in ((0, c), (1, s)):
            a = coef[m, j] - (coef[m, j] @ kv) / (kv @ kv) * kv
            for d in range(3):
                u[d] += a[d] * wave
    speed = np.sqrt((u * u).sum(axis=0)).max()
    return u * (amplitude / speed)


# Stability-limit study (Sec. 3.2, Table 1): a rising sphere in a periodic
# box of (6.4, 6.4, 12.8) d_p, starting at (3.2, 3.2, 0.6) d_p, Ga = 100 at
# u_g = 0.01, run until t_n = t u_g / d_p = 10.
STABILITY = dict(box=(6.4, 6.4, 12.8), start=(3.2, 3.2, 0.6), ga=100.0, u_g=0.01, t_n=10.0,
                 diameters=(10, 15, 20, 30, 40))
# The rotating virtual-mass test (Sec. 3.4): a (12.8, 6.4, 4.8) d_p box with no-slip walls on z (the upper one
# moving with u_w in x, the fluid starting from the Couette profile), the sphere at the centre with its
# translation held and its rotation released after the flow around it has developed; Re_p = u_p d_p / nu
# with u_p = u_w / 2 the undisturbed velocity at the centre.
ROTATION = dict(box=(12.8, 6.4, 4.8), diameter=40, u_w=0.1, re_p=110.0, develop_tc=4.0, monitor_tc=8.0,
                density_ratios=(0.1, 1.1, 0.001))

