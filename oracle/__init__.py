"""Oracle for the coupled LBM-MEM method (arXiv 2103.10882).

TEST INFRASTRUCTURE ONLY.  A plain FP64 CPU restatement of the paper's
method (C++ in this folder, loaded through ctypes) against which the CUDA
library is checked.  It shares no code with the library.  Only tests/, the
smoke check in __graft_entry__ and the CPU-baseline leg of bench.py may use it.

Function-level citations are in uniform.cpp; every pin of this oracle is in
tests/test_oracle_*.py.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("periodic", ctypes.c_int * 3),
        ("tau", ctypes.c_double),
        ("magic", ctypes.c_double),
        ("body_force", ctypes.c_double * 3),
        ("boundary", ctypes.c_int),
        ("force_average", ctypes.c_int),
        ("plain_mem", ctypes.c_int),
        ("bulk", ctypes.c_double),
        ("refill", ctypes.c_int),
    ]


class OrcDragParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("tau", ctypes.c_double), ("magic", ctypes.c_double),
        ("body_force", ctypes.c_double * 3),
        ("boundary", ctypes.c_int),
        ("pos", ctypes.c_double * 3),
        ("diameter", ctypes.c_double),
    ]


class OrcAmrParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("levels", ctypes.c_int),
        ("periodic", ctypes.c_int * 3),
        ("tau", ctypes.c_double),
        ("magic", ctypes.c_double),
        ("boundary", ctypes.c_int),
        ("force_average", ctypes.c_int),
        ("plain_mem", ctypes.c_int),
        ("rescale", ctypes.c_int),
        ("bulk", ctypes.c_double),
        ("refill", ctypes.c_int),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
        L.orc_create.restype = vp
        L.orc_create.argtypes = [ctypes.POINTER(OrcParams)]
        L.orc_destroy.argtypes = [vp]
        L.orc_add_sphere.restype = ip
        L.orc_add_sphere.argtypes = [vp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ip]
        L.orc_set_particle_velocity.argtypes = [vp, dp, dp]
        L.orc_set_gravity.argtypes = [vp, dp]
        L.orc_set_planes.restype = ip
        L.orc_set_planes.argtypes = [vp, ip, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_init_equilibrium.argtypes = [vp, ctypes.c_double, dp, dp]
        L.orc_set_populations.argtypes = [vp, dp]
        L.orc_get_populations.argtypes = [vp, dp]
        L.orc_get_flags.argtypes = [vp, ctypes.POINTER(ctypes.c_uint8)]
        L.orc_moments.argtypes = [vp, dp, dp]
        L.orc_step.argtypes = [vp, ip]
        L.orc_get_links.restype = ctypes.c_int64
        L.orc_get_links.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32), dp,
                                    ctypes.c_int64]
        L.orc_get_particle.argtypes = [vp, dp]
        L.orc_get_history.restype = ctypes.c_int64
        L.orc_get_history.argtypes = [vp, dp, ctypes.c_int64]
        L.orc_get_plane_force.argtypes = [vp, dp]
        L.orc_particle_only_step.argtypes = [vp, dp, dp]
        L.orc_set_particle_fixed.restype = ip
        L.orc_set_particle_fixed.argtypes = [vp, ip]
        L.orc_set_wall_velocity.restype = ip
        L.orc_set_wall_velocity.argtypes = [vp, ip, ip, dp]
        L.orc_set_threads.restype = ip
        L.orc_set_threads.argtypes = [ip]
        L.orc_amr_create.restype = vp
        L.orc_amr_create.argtypes = [ctypes.POINTER(OrcAmrParams)]
        L.orc_amr_destroy.argtypes = [vp]
        L.orc_amr_refine_box.restype = ip
        L.orc_amr_refine_box.argtypes = [vp, dp, dp]
        L.orc_amr_add_sphere.restype = ip
        L.orc_amr_add_sphere.argtypes = [vp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, ip]
        L.orc_amr_set_gravity.argtypes = [vp, dp]
        L.orc_amr_set_particle_velocity.argtypes = [vp, dp, dp]
        L.orc_amr_regrid.restype = ip
        L.orc_amr_regrid.argtypes = [vp]
        L.orc_amr_init_equilibrium.argtypes = [vp, ctypes.c_double, dp, ctypes.c_double, ip, ip]
        L.orc_amr_set_sensor.restype = ip
        L.orc_amr_set_sensor.argtypes = [vp, ctypes.c_double, ctypes.c_double]
        L.orc_amr_block_sensor.restype = ctypes.c_int64
        L.orc_amr_block_sensor.argtypes = [vp, ip, dp, ctypes.c_int64]
        L.orc_amr_init_linear.argtypes = [vp, ctypes.c_double, dp, dp, dp]
        L.orc_amr_step.restype = ip
        L.orc_amr_step.argtypes = [vp, ip]
        L.orc_amr_error.restype = ip
        L.orc_amr_error.argtypes = [vp]
        L.orc_amr_level_shape.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_int)]
        L.orc_amr_block_map.restype = ctypes.c_int64
        L.orc_amr_block_map.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_int32), ctypes.c_int64]
        L.orc_amr_level_populations.argtypes = [vp, ip, dp]
        L.orc_amr_mass.argtypes = [vp, dp]
        L.orc_amr_real_cells.restype = ctypes.c_int64
        L.orc_amr_real_cells.argtypes = [vp, ip, ctypes.POINTER(ctypes.c_int32), dp, ctypes.c_int64]
        L.orc_amr_get_flags.restype = ctypes.c_int64
        L.orc_amr_get_flags.argtypes = [vp, ctypes.POINTER(ctypes.c_uint8), ctypes.c_int64]
        L.orc_amr_get_links.restype = ctypes.c_int64
        L.orc_amr_get_links.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32), dp,
                                        ctypes.c_int64]
        L.orc_amr_get_particle.argtypes = [vp, dp]
        L.orc_amr_get_history.restype = ctypes.c_int64
        L.orc_amr_get_history.argtypes = [vp, dp, ctypes.c_int64]
        L.orc_grad_noneq.argtypes = [ctypes.c_double, dp, dp]
        L.orc_drag_tangent.restype = ctypes.c_double
        L.orc_drag_tangent.argtypes = [ctypes.POINTER(OrcDragParams), dp, ip, ctypes.c_double, dp, dp, ip, dp, dp]
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def grad_noneq(tau, S):
    """Grad's post-collision non-equilibrium part (19 values) for a strain rate S (3x3)."""
    _, pS = _d(np.asarray(S, dtype=np.float64).reshape(9))
    out = np.empty(19)
    lib().orc_grad_noneq(float(tau), pS, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def _fixed_mode(fixed):
    if fixed == "translation":
        return 2
    if fixed is True or fixed is False:
        return int(fixed)
    return int(fixed)


def set_threads(n: int) -> int:
    return lib().orc_set_threads(int(n))


class UniformSim:
    """One uniform-grid simulation held by the C++ oracle."""

    def __init__(self, shape, tau, magic=3.0 / 16.0, periodic=(1, 1, 1), body_force=(0.0, 0.0, 0.0),
                 boundary="cli", force_average=True, plain_mem=False, bulk=1.0, refill="equilibrium"):
        L = lib()
        p = OrcParams()
        p.nx, p.ny, p.nz = (int(v) for v in shape)
        p.periodic = (ctypes.c_int * 3)(*[int(v) for v in periodic])
        p.tau = float(tau)
        p.magic = float(magic)
        p.body_force = (ctypes.c_double * 3)(*[float(v) for v in body_force])
        p.boundary = {"cli": 0, "sbb": 1}[boundary]
        p.force_average = int(bool(force_average))
        p.plain_mem = int(bool(plain_mem))
        p.bulk = float(bulk)
        p.refill = {"equilibrium": 0, "grad": 1}[refill]
        self.shape = tuple(int(v) for v in shape)
        self.ncells = self.shape[0] * self.shape[1] * self.shape[2]
        self._h = L.orc_create(ctypes.byref(p))
        if not self._h:
            raise ValueError("oracle rejected the parameters")
        self._L = L

    def close(self):
        if self._h:
            self._L.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_sphere(self, pos, diameter, density_ratio, cv=0.0, cv_omega=None, fixed=False):
        if cv_omega is None:
            cv_omega = cv
        a, pa = _d(pos)
        rc = self._L.orc_add_sphere(self._h, pa, float(diameter), float(density_ratio), float(cv),
                                    float(cv_omega), _fixed_mode(fixed))
        if rc != 0:
            raise ValueError("add_sphere rejected")

    def set_fixed(self, fixed):
        """Held degrees of freedom: False/0 none, True/1 all, 2 or "translation" translation only."""
        if self._L.orc_set_particle_fixed(self._h, _fixed_mode(fixed)) != 0:
            raise ValueError("set_fixed rejected")

    def set_wall_velocity(self, axis, side, u):
        """Velocity of the domain wall on the low (0) or high (1) face of a non-periodic axis."""
        a, pa = _d(u)
        if self._L.orc_set_wall_velocity(self._h, int(axis), int(side), pa) != 0:
            raise ValueError("set_wall_velocity rejected")

    def set_particle_velocity(self, u, w=(0.0, 0.0, 0.0)):
        a, pa = _d(u)
        b, pb = _d(w)
        self._L.orc_set_particle_velocity(self._h, pa, pb)

    def set_gravity(self, g):
        a, pa = _d(g)
        self._L.orc_set_gravity(self._h, pa)

    def set_planes(self, axis, lo, hi, v_lo=(0, 0, 0), v_hi=(0, 0, 0)):
        a, pa = _d(v_lo)
        b, pb = _d(v_hi)
        if self._L.orc_set_planes(self._h, int(axis), float(lo), float(hi), pa, pb) != 0:
            raise ValueError("set_planes rejected")

    def init_equilibrium(self, rho=1.0, u=(0.0, 0.0, 0.0), u_field=None):
        a, pa = _d(u)
        if u_field is not None:
            f, pf = _d(np.asarray(u_field).reshape(3, -1))
        else:
            f, pf = None, None
        self._L.orc_init_equilibrium(self._h, float(rho), pa, pf)

    def set_populations(self, g):
        a, pa = _d(np.asarray(g).reshape(19, -1))
        assert a.shape[1] == self.ncells
        self._L.orc_set_populations(self._h, pa)

    def populations(self):
        out = np.empty((19, self.ncells), dtype=np.float64)
        self._L.orc_get_populations(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return out

    def flags(self):
        out = np.empty(self.ncells, dtype=np.uint8)
        self._L.orc_get_flags(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
        return out

    def moments(self):
        rho = np.empty(self.ncells)
        u = np.empty((3, self.ncells))
        self._L.orc_moments(self._h, rho.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return rho, u

    def step(self, n=1):
        self._L.orc_step(self._h, int(n))

    def links(self):
        n = self._L.orc_get_links(self._h, None, None, None, 0)
        cell = np.empty(n, dtype=np.int64)
        q = np.empty(n, dtype=np.int32)
        delta = np.empty(n, dtype=np.float64)
        self._L.orc_get_links(self._h, cell.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                              q.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                              delta.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n)
        return cell, q, delta

    def particle(self):
        out = np.empty(24)
        self._L.orc_get_particle(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return out

    def history(self):
        n = self._L.orc_get_history(self._h, None, 0)
        out = np.empty((n, 15))
        self._L.orc_get_history(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n)
        return out

    def plane_force(self):
        out = np.empty(3)
        self._L.orc_get_plane_force(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return out

    def particle_only_step(self, F, T=(0.0, 0.0, 0.0)):
        a, pa = _d(F)
        b, pb = _d(T)
        self._L.orc_particle_only_step(self._h, pa, pb)


class RefinedSim:
    """Block-structured refined simulation held by the C++ oracle (refined.cpp)."""

    def __init__(self, shape, levels, tau, magic=3.0 / 16.0, periodic=(1, 1, 1), boundary="cli",
                 force_average=True, plain_mem=False, rescale=False, bulk=1.0, refill="equilibrium"):
        L = lib()
        p = OrcAmrParams()
        p.nx, p.ny, p.nz = (int(v) for v in shape)
        p.levels = int(levels)
        p.periodic = (ctypes.c_int * 3)(*[int(v) for v in periodic])
        p.tau = float(tau)
        p.magic = float(magic)
        p.boundary = {"cli": 0, "sbb": 1}[boundary]
        p.force_average = int(bool(force_average))
        p.plain_mem = int(bool(plain_mem))
        p.rescale = int(bool(rescale))
        p.bulk = float(bulk)
        p.refill = {"equilibrium": 0, "grad": 1}[refill]
        self._L = L
        self.levels = int(levels)
        self._h = L.orc_amr_create(ctypes.byref(p))
        if not self._h:
            raise ValueError("oracle rejected the parameters")

    def close(self):
        if self._h:
            self._L.orc_amr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _rc(self, rc):
        if rc != 0:
            raise RuntimeError("refined oracle error %d" % rc)

    def refine_box(self, lo, hi):
        a, pa = _d(lo)
        b, pb = _d(hi)
        self._rc(self._L.orc_amr_refine_box(self._h, pa, pb))

    def add_sphere(self, pos, diameter, density_ratio, cv=0.0, cv_omega=None, fixed=False):
        if cv_omega is None:
            cv_omega = cv
        a, pa = _d(pos)
        self._rc(self._L.orc_amr_add_sphere(self._h, pa, float(diameter), float(density_ratio), float(cv),
                                            float(cv_omega), _fixed_mode(fixed)))

    def set_gravity(self, g):
        a, pa = _d(g)
        self._L.orc_amr_set_gravity(self._h, pa)

    def set_particle_velocity(self, u, w=(0.0, 0.0, 0.0)):
        a, pa = _d(u)
        b, pb = _d(w)
        self._L.orc_amr_set_particle_velocity(self._h, pa, pb)

    def regrid(self):
        self._rc(self._L.orc_amr_regrid(self._h))

    def init_equilibrium(self, rho=1.0, u=(0.0, 0.0, 0.0), shear=0.0, shear_dir=0, shear_axis=2):
        a, pa = _d(u)
        self._L.orc_amr_init_equilibrium(self._h, float(rho), pa, float(shear), int(shear_dir), int(shear_axis))

    def set_sensor(self, sigma, c=0.2):
        """Flow sensor of Sec. 4.2.2 (sigma = 0 turns it off); consulted by regrid()."""
        self._rc(self._L.orc_amr_set_sensor(self._h, float(sigma), float(c)))

    def block_sensor(self, level):
        """Scaled curl (largest over the block's cells) of every real block of a level."""
        n = self._L.orc_amr_block_sensor(self._h, int(level), None, 0)
        out = np.empty(max(n, 0))
        self._L.orc_amr_block_sensor(self._h, int(level), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n)
        return out

    def init_linear(self, A, u0=(0.0, 0.0, 0.0), x0=(0.0, 0.0, 0.0), rho=1.0):
        """Equilibrium with the linear velocity u0 + A (x - x0) (finest-level units)."""
        _, pu = _d(u0)
        Am, pA = _d(np.asarray(A, dtype=np.float64).reshape(9))
        _, px = _d(x0)
        self._L.orc_amr_init_linear(self._h, float(rho), pu, pA, px)

    def step(self, n=1):
        self._rc(self._L.orc_amr_step(self._h, int(n)))

    def level_shape(self, level):
        out = (ctypes.c_int * 3)()
        self._L.orc_amr_level_shape(self._h, int(level), out)
        return tuple(out)

    def block_map(self, level):
        n = self._L.orc_amr_block_map(self._h, int(level), None, 0)
        out = np.empty(n, dtype=np.int32)
        self._L.orc_amr_block_map(self._h, int(level), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n)
        return out

    def level_populations(self, level):
        nx, ny, nz = self.level_shape(level)
        out = np.empty((19, nx * ny * nz))
        self._L.orc_amr_level_populations(self._h, int(level), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return out

    def real_cells(self, level):
        """(coords [n,3] int32, deviations [n,19]) of the real cells of a level."""
        n = self._L.orc_amr_real_cells(self._h, int(level), None, None, 0)
        xyz = np.empty((n, 3), dtype=np.int32)
        g = np.empty((n, 19))
        self._L.orc_amr_real_cells(self._h, int(level), xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                   g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n)
        return xyz, g

    def flags(self):
        """Finest-level flags in real_cells order: 1 solid, 2 fluid next to the sphere, 0 fluid."""
        n = self._L.orc_amr_get_flags(self._h, None, 0)
        out = np.empty(n, dtype=np.uint8)
        self._L.orc_amr_get_flags(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), n)
        return out

    def links(self):
        """Finest-level boundary links: (cell [n] int64, q [n] int32, delta [n])."""
        n = self._L.orc_amr_get_links(self._h, None, None, None, 0)
        cell = np.empty(n, dtype=np.int64)
        q = np.empty(n, dtype=np.int32)
        d = np.empty(n)
        self._L.orc_amr_get_links(self._h, cell.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  q.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                  d.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n)
        return cell, q, d

    def mass(self):
        out = np.empty(4)
        self._L.orc_amr_mass(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return out

    def particle(self):
        out = np.empty(24)
        self._L.orc_amr_get_particle(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return out

    def history(self):
        n = self._L.orc_amr_get_history(self._h, None, 0)
        out = np.empty((n, 15))
        self._L.orc_amr_get_history(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n)
        return out


def drag_tangent(shape, tau, pos, diameter, nsteps, u0=None, body_force=(0.0, 0.0, 0.0), magic=3.0 / 16.0,
                 boundary="cli", dtau=0.0, dforce=(0.0, 0.0, 0.0), du0=None, axis=0):
    """Mean drag J = (1/N) sum_n F_axis^n on a fixed sphere in a periodic box
    and its derivative along (dtau, dforce, du0), by the tangent-linear model
    of tangent.cpp.  u0, du0: arrays (3, nz, ny, nx) or None.  Returns
    (J, dJ, forces[nsteps, 3])."""
    L = lib()
    p = OrcDragParams()
    p.nx, p.ny, p.nz = (int(v) for v in shape)
    p.tau = float(tau)
    p.magic = float(magic)
    p.body_force = (ctypes.c_double * 3)(*[float(v) for v in body_force])
    p.boundary = {"cli": 0, "sbb": 1}[boundary]
    p.pos = (ctypes.c_double * 3)(*[float(v) for v in pos])
    p.diameter = float(diameter)
    n = p.nx * p.ny * p.nz
    keep = []

    def field(a):
        if a is None:
            return None
        arr, ptr = _d(np.asarray(a).reshape(3, n))
        keep.append(arr)
        return ptr

    df, pdf = _d(dforce)
    forces = np.zeros((int(nsteps), 3))
    dJ = ctypes.c_double(0.0)
    J = L.orc_drag_tangent(ctypes.byref(p), field(u0), int(nsteps), float(dtau), pdf, field(du0), int(axis),
                           ctypes.byref(dJ), forces.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return J, dJ.value, forces
