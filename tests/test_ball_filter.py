"""The solid flag of a cell is defined by the FP64 ball predicate
((dx*dx)+(dy*dy))+(dz*dz) <= r*r with round-to-nearest operations (no
contraction).  The CUDA kernels first evaluate the squared distance in FP32
from X split as floor(X) + (1/2 - Xh) and decide every cell whose FP32 value
lies outside [r^2 - m, r^2 + m], m = 1e-5 (r^2 + 1); only the cells in
between take the FP64 expression.  This checks, with the same FP32
operations emulated in numpy (with and without a fused multiply-add for the
sum of squares), that the FP32 decision never contradicts the FP64
predicate, on cells packed around sphere surfaces of many radii and
centres, including periodic images."""
import numpy as np


def exact(p, X, r, n):
    d = (p + 0.5) - X
    d = np.where(d > 0.5 * n, d - n, np.where(d < -0.5 * n, d + n, d))
    return ((d[:, 0] * d[:, 0]) + (d[:, 1] * d[:, 1])) + (d[:, 2] * d[:, 2]) <= r * r


def fp32_estimate(p, X, n, fma):
    f32 = np.float32
    Xi = np.floor(X)
    Xh = (0.5 - (X - Xi)).astype(f32)
    v = (p - Xi.astype(np.int64))
    t = v.astype(f32) + Xh
    half = (0.5 * n).astype(f32)
    v = np.where(t > half, v - n, np.where(t < -half, v + n, v))
    t = v.astype(f32) + Xh
    if fma:   # fmaf(t, t, e): one rounding per step, emulated in FP64 then rounded
        e = f32(0)
        for a in range(3):
            e = (t[:, a].astype(np.float64) * t[:, a].astype(np.float64) + np.float64(e)).astype(f32)
    else:
        e = ((t[:, 0] * t[:, 0]) + (t[:, 1] * t[:, 1])) + (t[:, 2] * t[:, 2])
    return e


def test_fp32_pretest_never_contradicts_fp64_predicate():
    rng = np.random.default_rng(0)
    undecided = total = 0
    for trial in range(60):
        n = np.array(rng.choice([32, 64, 256, 1024, 4096], size=3), dtype=np.int64)
        r = float(rng.uniform(2.0, 0.35 * n.min()))
        X = rng.uniform(0, n)
        # cells within a few cells of the surface, some across the periodic boundary
        m = 20000
        dirs = rng.normal(size=(m, 3))
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        rad = r + rng.uniform(-1.5, 1.5, size=m)
        p = np.floor(X + dirs * rad[:, None]).astype(np.int64) % n
        ref = exact(p, X, r, n)
        rr = r * r
        mg = 1e-5 * (rr + 1.0)
        lo, hi = np.float32(rr - mg), np.float32(rr + mg)
        for fma in (False, True):
            e = fp32_estimate(p, X, n, fma)
            inside, outside = e < lo, e > hi
            assert not np.any(inside & ~ref), "FP32 said inside, FP64 outside"
            assert not np.any(outside & ref), "FP32 said outside, FP64 inside"
            undecided += int(np.sum(~inside & ~outside))
            total += m
    assert undecided < 1e-3 * total   # the FP64 path is rare


def test_fp32_pretest_adversarial_radii():
    """Radii chosen so that cell centres sit within 1e-8..1e-5 (relative) of
    the surface, where the FP32 estimate alone would be wrong: the margin
    sends them to the FP64 path."""
    rng = np.random.default_rng(1)
    n = np.array([512, 512, 2048], dtype=np.int64)
    bad_without_margin = 0
    for trial in range(200):
        X = rng.uniform(0, n)
        p = (np.floor(X).astype(np.int64) + rng.integers(-30, 30, size=3)) % n
        d = (p + 0.5) - X
        d = np.where(d > 0.5 * n, d - n, np.where(d < -0.5 * n, d + n, d))
        dist = float(np.sqrt(d @ d))
        for rel in (1e-9, 1e-8, -1e-8, 1e-7, -1e-7, 1e-6, -1e-6):
            r = dist * (1.0 + rel)
            pp = p[None, :]
            ref = exact(pp, X, r, n)
            rr = r * r
            mg = 1e-5 * (rr + 1.0)
            for fma in (False, True):
                e = fp32_estimate(pp, X, n, fma)
                if e[0] < np.float32(rr - mg):
                    assert ref[0]
                elif e[0] > np.float32(rr + mg):
                    assert not ref[0]
                bad_without_margin += int((e[0] <= np.float32(rr)) != ref[0])
    assert bad_without_margin > 0   # the cases do exercise the FP32 rounding


C18 = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1],
                [1, 0, -1], [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]])


def test_neighbour_pretest_never_contradicts_fp64_predicate():
    """The remap decides the neighbours of a cell from the cell's own FP32
    offset t as (t + c_q)^2 (one more FP32 rounding per component); the
    margin still covers it, including cells near half a period of small
    periodic boxes (spheres reaching within two cells of half a period take
    the FP64 path everywhere)."""
    rng = np.random.default_rng(2)
    f32 = np.float32
    checked = 0
    for trial in range(80):
        n = np.array(rng.choice([10, 16, 24, 64, 512], size=3), dtype=np.int64)
        r = float(rng.uniform(1.5, 0.45 * n.min()))
        if np.any(r > 0.4 * n) or np.any(r + 2.0 >= 0.5 * n):
            continue   # the kernels take the FP64 path for every cell here
        X = rng.uniform(0, n)
        m = 4000
        dirs = rng.normal(size=(m, 3))
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        rad = r + rng.uniform(-2.0, 2.0, size=m)
        p = np.floor(X + dirs * rad[:, None]).astype(np.int64) % n
        Xi = np.floor(X)
        Xh = (0.5 - (X - Xi)).astype(f32)
        v = p - Xi.astype(np.int64)
        t = v.astype(f32) + Xh
        half = (0.5 * n).astype(f32)
        v = np.where(t > half, v - n, np.where(t < -half, v + n, v))
        t = v.astype(f32) + Xh
        rr = r * r
        mg = 1e-5 * (rr + 1.0)
        lo, hi = f32(rr - mg), f32(rr + mg)
        for c in C18:
            a = t + c.astype(f32)
            e = ((a[:, 0] * a[:, 0]) + (a[:, 1] * a[:, 1])) + (a[:, 2] * a[:, 2])
            ref = exact((p + c) % n, X, r, n)
            assert not np.any((e < lo) & ~ref)
            assert not np.any((e > hi) & ref)
            checked += m
    assert checked > 0
