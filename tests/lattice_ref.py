"""Independent D3Q19 tables for the tests (typed from the textbook definition
of the velocity set, not imported from either implementation)."""
import numpy as np

C = np.array([[0, 0, 0],
              [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
              [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1],
              [1, 0, -1], [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]], dtype=np.int64)
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def opposite(q):
    return 0 if q == 0 else (q + 1 if q % 2 == 1 else q - 1)


def moments(g, shape):
    """rho and u from deviation populations g[19, ncells] (rho_0 = 1)."""
    rho = 1.0 + g.sum(axis=0)
    u = np.einsum("qa,qn->an", C.astype(np.float64), g)
    return rho, u


def cell_centres(shape):
    nx, ny, nz = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([i.ravel() + 0.5, j.ravel() + 0.5, k.ravel() + 0.5])
