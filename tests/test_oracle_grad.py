"""Pins of the Grad refill of uncovered cells (Sec. 2.3, Dorschner et al.'s
approach read as Grad's approximation from the local strain rate).

- Grad's post-collision non-equilibrium part, -3 w (1 - s+)/s+ Q:S, is the
  lattice Boltzmann method's own: in a converged plane Couette flow between
  moving CLI walls (exact linear profile) every bulk cell's stored
  post-collision populations equal f_eq(rho, u) plus that term for the
  exact shear rate, to O(gamma^2).  At tau = 0.9 the post-collision factor
  (1 - s+)/s+ = -0.1 differs in sign from the pre-collision 1/s+, so a
  wrong collision factor, sign or tensor fails;
- a moving sphere refilled either way follows nearly the same path: the
  refill differs by the Grad term, at most a fifth of the populations here.
"""
import numpy as np

from lattice_ref import C, W


def eq_dev(rho, u):
    cu = C @ u
    return W * ((rho - 1) + 3 * cu + 4.5 * cu ** 2 - 1.5 * u @ u)


def test_grad_term_is_the_couette_stress(orc):
    tau, U, lo, hi = 0.9, 1e-3, 1.3, 14.7
    s = orc.UniformSim((4, 16, 4), tau=tau)
    s.set_planes(1, lo, hi, (0, 0, 0), (U, 0, 0))
    s.init_equilibrium()
    s.step(8000)
    g = s.populations().reshape(19, 4, 16, 4)          # [q][z][y][x]
    gamma = U / (hi - lo)
    S = np.zeros((3, 3))
    S[0, 1] = S[1, 0] = 0.5 * gamma
    grad = orc.grad_noneq(tau, S)
    assert np.abs(grad).max() > 0
    worst = 0.0
    for y in range(4, 12):
        cell = g[:, 1, y, 2]
        rho = 1 + cell.sum()
        u = cell @ C.astype(float)
        assert abs(u[0] - gamma * (y + 0.5 - lo)) < 1e-9          # the exact linear profile
        worst = max(worst, np.abs(cell - eq_dev(rho, u) - grad).max())
    assert worst < 1e-3 * np.abs(grad).max(), worst
    # the pre-collision factor would be far off
    pre = -3 * W * tau * np.einsum("qa,qb,ab->q", C, C, S)
    assert np.abs(pre - grad).max() > 10 * worst


def test_grad_and_equilibrium_refill_of_a_moving_sphere(orc):
    out = {}
    for mode in ("equilibrium", "grad"):
        s = orc.UniformSim((24, 24, 24), tau=0.6, refill=mode)
        s.add_sphere((12.3, 11.8, 12.6), 8.0, 0.2, cv=0.5)
        s.set_gravity((0, 0, -2e-3))
        s.init_equilibrium()
        s.step(40)
        out[mode] = (s.populations(), s.flags(), s.history())
    (ge, fe, he), (gg, fg, hg) = out["equilibrium"], out["grad"]
    assert hg[-1, 8] - hg[0, 8] > 0.5                # the sphere moved across cell centres, so cells were refilled
    assert np.abs(hg - he).max() > 0                  # the refill reaches the coupling
    assert np.abs(hg[:, 6:9] - he[:, 6:9]).max() < 1e-2   # and changes the path only slightly
    both = (fe == 0) & (fg == 0)
    assert np.abs(gg[:, both] - ge[:, both]).max() < 0.2 * np.abs(ge).max()   # strain near a sphere at 0.02 lattice speed
