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
