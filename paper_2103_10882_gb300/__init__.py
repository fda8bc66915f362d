"""GB300 library for the coupled lattice Boltzmann / momentum exchange method
with virtual-mass correction for light particles (Werner, Rettinger & Ruede,
arXiv 2103.10882).

The compute path is the CUDA library liblbmp.so (C ABI in include/lbmp.h).
This module only marshals arguments: the functions named lbmp_* mirror the C
entry points one to one, and `Simulation` wraps a handle for convenience.
PyTorch supplies device memory (its caching allocator) and the CUDA stream.
There is no CPU fallback: without the library or a GPU every call raises.
"""
import ctypes
import os

import numpy as np

from . import _native
from ._native import LbmpConfig

__all__ = ["LbmpError", "Simulation", "lbmp_config_default", "lbmp_create", "lbmp_destroy", "lbmp_add_sphere",
           "lbmp_set_particle_velocity", "lbmp_set_particle_fixed", "lbmp_set_wall_velocity", "lbmp_ga_parameters", "lbmp_set_ga",
           "lbmp_set_tau", "lbmp_set_gravity", "lbmp_set_body_force", "lbmp_init_fluid", "lbmp_set_populations",
           "lbmp_get_populations", "lbmp_gather_populations", "lbmp_step", "lbmp_step_async", "lbmp_check_status", "lbmp_synchronize",
           "lbmp_get_particle", "lbmp_get_history", "lbmp_get_flags", "lbmp_get_links", "lbmp_get_counters",
           "lbmp_profile", "lbmp_get_profile", "lbmp_boundary_cells_noalloc", "lbmp_last_error",
           "lbmp_init_fluid_wave", "lbmp_refine_box", "lbmp_regrid", "lbmp_save", "lbmp_load", "lbmp_set_refinement_sensor", "lbmp_get_block_sensor",
           "lbmp_level_shape", "lbmp_get_block_map",
           "lbmp_get_level_cells", "lbmp_get_level_flags", "lbmp_updates_per_step", "lbmp_batch_create", "lbmp_batch_autotune",
           "lbmp_batch_info", "lbmp_batch_get_populations", "BatchSimulation", "PRECISIONS", "lbmp_drag_forward",
           "lbmp_drag_backward", "mean_drag"]

PRECISIONS = {"fp64": 0, "fp32": 1, "fp16": 2}
BC = {"periodic": 0, "noslip": 1}
REFILL = {"equilibrium": 0, "grad": 1}
BOUNDARY = {"cli": 0, "sbb": 1}
STATUS = {0: "LBMP_OK", 1: "LBMP_ERR_INVALID_ARG", 2: "LBMP_ERR_OOM", 3: "LBMP_ERR_CUDA", 4: "LBMP_ERR_UNSTABLE",
          5: "LBMP_ERR_PARTICLE_NOT_FINEST", 6: "LBMP_ERR_TIMEOUT", 7: "LBMP_ERR_UNSUPPORTED"}


class LbmpError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status


def _lib():
    return _native.load()


def _dp(a):
    return a.ctypes.data_as(_native.c_double_p)


def _vec3(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(3))


def _check(h, rc):
    if rc != 0:
        msg = _lib().lbmp_last_error(h)
        raise LbmpError(rc, msg.decode() if msg else "")


# ------------------------------------------------------------- C ABI mirror
def lbmp_config_default():
    cfg = LbmpConfig()
    _check(None, _lib().lbmp_config_default(ctypes.byref(cfg)))
    return cfg


def lbmp_create(cfg):
    h = ctypes.c_void_p()
    _check(None, _lib().lbmp_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def lbmp_destroy(h):
    _check(h, _lib().lbmp_destroy(h))


def lbmp_add_sphere(h, pos, diameter, density_ratio, cv=0.0, cv_omega=None):
    p = _vec3(pos)
    pid = ctypes.c_int(-1)
    cvw = cv if cv_omega is None else cv_omega
    _check(h, _lib().lbmp_add_sphere(h, _dp(p), float(diameter), float(density_ratio), float(cv), float(cvw),
                                     ctypes.byref(pid)))
    return pid.value


def lbmp_set_particle_velocity(h, pid, u, omega=(0.0, 0.0, 0.0)):
    a, b = _vec3(u), _vec3(omega)
    _check(h, _lib().lbmp_set_particle_velocity(h, int(pid), _dp(a), _dp(b)))


def lbmp_set_particle_fixed(h, pid, fixed=True):
    """fixed: False/0 free, True/1 translation and rotation held, 2 or "translation" translation held."""
    mode = 2 if fixed == "translation" else int(fixed)
    _check(h, _lib().lbmp_set_particle_fixed(h, int(pid), mode))


def lbmp_set_wall_velocity(h, axis, side, u):
    a = np.ascontiguousarray(u, dtype=np.float64)
    _check(h, _lib().lbmp_set_wall_velocity(h, int(axis), int(side), _dp(a)))


def lbmp_ga_parameters(ga, u_g, diameter, density_ratio):
    nu, g, tau = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(None, _lib().lbmp_ga_parameters(float(ga), float(u_g), float(diameter), float(density_ratio),
                                           ctypes.byref(nu), ctypes.byref(g), ctypes.byref(tau)))
    return nu.value, g.value, tau.value


def lbmp_set_ga(h, ga, u_g, direction):
    d = _vec3(direction)
    _check(h, _lib().lbmp_set_ga(h, float(ga), float(u_g), _dp(d)))


def lbmp_set_tau(h, tau):
    _check(h, _lib().lbmp_set_tau(h, float(tau)))


def lbmp_set_gravity(h, g):
    a = _vec3(g)
    _check(h, _lib().lbmp_set_gravity(h, _dp(a)))


def lbmp_set_body_force(h, f):
    a = _vec3(f)
    _check(h, _lib().lbmp_set_body_force(h, _dp(a)))


def lbmp_init_fluid(h, rho=1.0, u=(0.0, 0.0, 0.0), u_field=None):
    """u_field: None, a host array [3, nz, ny, nx] (FP64), or a CUDA tensor of that shape (float64)."""
    a = _vec3(u)
    if u_field is None:
        _check(h, _lib().lbmp_init_fluid(h, float(rho), _dp(a), None, 0))
    elif hasattr(u_field, "is_cuda") and u_field.is_cuda:
        import torch
        t = u_field.to(torch.float64).contiguous()
        _check(h, _lib().lbmp_init_fluid(h, float(rho), _dp(a), ctypes.c_void_p(t.data_ptr()), 1))
    else:
        f = np.ascontiguousarray(np.asarray(u_field, dtype=np.float64))
        _check(h, _lib().lbmp_init_fluid(h, float(rho), _dp(a), f.ctypes.data_as(ctypes.c_void_p), 0))


def lbmp_set_populations(h, g):
    a = np.ascontiguousarray(np.asarray(g, dtype=np.float64)).reshape(-1)
    _check(h, _lib().lbmp_set_populations(h, _dp(a), a.size))


def lbmp_get_populations(h, ncells):
    out = np.empty(19 * int(ncells), dtype=np.float64)
    _check(h, _lib().lbmp_get_populations(h, _dp(out), out.size))
    return out.reshape(19, -1)


def lbmp_gather_populations(h, cells):
    c = np.ascontiguousarray(np.asarray(cells, dtype=np.int64).reshape(-1))
    out = np.empty((c.size, 19), dtype=np.float64)
    _check(h, _lib().lbmp_gather_populations(h, c.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), c.size,
                                             _dp(out)))
    return out


def lbmp_step(h, n=1):
    _check(h, _lib().lbmp_step(h, int(n)))


def lbmp_step_async(h, n=1):
    _check(h, _lib().lbmp_step_async(h, int(n)))


def lbmp_check_status(h):
    _check(h, _lib().lbmp_check_status(h))


def lbmp_synchronize(h):
    _check(h, _lib().lbmp_synchronize(h))


def lbmp_get_particle(h, pid=0):
    out = np.empty(24, dtype=np.float64)
    _check(h, _lib().lbmp_get_particle(h, int(pid), _dp(out)))
    return out


def lbmp_get_history(h, pid=0, max_steps=None):
    n = ctypes.c_int(0)
    _check(h, _lib().lbmp_get_history(h, int(pid), None, 0, ctypes.byref(n)))
    m = n.value if max_steps is None else min(n.value, int(max_steps))
    out = np.empty((max(m, 0), 15), dtype=np.float64)
    if m > 0:
        _check(h, _lib().lbmp_get_history(h, int(pid), _dp(out), m, ctypes.byref(n)))
    return out[: n.value]


def lbmp_get_flags(h, ncells):
    out = np.empty(int(ncells), dtype=np.uint8)
    _check(h, _lib().lbmp_get_flags(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), out.size))
    return out


def lbmp_get_links(h):
    n = ctypes.c_size_t(0)
    _check(h, _lib().lbmp_get_links(h, None, None, None, 0, ctypes.byref(n)))
    m = n.value
    cell = np.empty(m, dtype=np.int64)
    q = np.empty(m, dtype=np.int32)
    delta = np.empty(m, dtype=np.float64)
    if m:
        _check(h, _lib().lbmp_get_links(h, cell.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                        q.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dp(delta), m,
                                        ctypes.byref(n)))
    return cell, q, delta


def lbmp_get_counters(h):
    out = (ctypes.c_int64 * 5)()
    _check(h, _lib().lbmp_get_counters(h, out))
    return tuple(out)


def lbmp_profile(h, enable=True):
    _check(h, _lib().lbmp_profile(h, int(bool(enable))))


def lbmp_get_profile(h):
    out = np.zeros(6, dtype=np.float64)
    _check(h, _lib().lbmp_get_profile(h, _dp(out)))
    return out


def lbmp_boundary_cells_noalloc(flags_ptr, shape, periodic, center, diameter, list_ptr, capacity, count_ptr,
                                stream_ptr=0):
    """Boundary cells of one sphere without any allocation inside the call.
    flags_ptr, list_ptr, count_ptr are device addresses (e.g. tensor.data_ptr())."""
    per = (ctypes.c_int * 3)(*[int(bool(p)) for p in periodic])
    c = _vec3(center)
    nx, ny, nz = (int(v) for v in shape)
    _check(None, _lib().lbmp_boundary_cells_noalloc(ctypes.c_void_p(flags_ptr), nx, ny, nz, per, _dp(c),
                                                    float(diameter), ctypes.c_void_p(list_ptr), int(capacity),
                                                    ctypes.c_void_p(count_ptr), ctypes.c_void_p(stream_ptr)))


def lbmp_init_fluid_wave(h, rho=1.0, u=(0.0, 0.0, 0.0), amp=0.0, direction=0, axis=2):
    a = _vec3(u)
    _check(h, _lib().lbmp_init_fluid_wave(h, float(rho), _dp(a), float(amp), int(direction), int(axis)))


def lbmp_refine_box(h, lo, hi):
    a, b = _vec3(lo), _vec3(hi)
    _check(h, _lib().lbmp_refine_box(h, _dp(a), _dp(b)))


def lbmp_regrid(h):
    _check(h, _lib().lbmp_regrid(h))


def lbmp_level_shape(h, level):
    out = (ctypes.c_int * 3)()
    _check(h, _lib().lbmp_level_shape(h, int(level), out))
    return tuple(out)


def lbmp_save(h, path):
    _check(h, _lib().lbmp_save(h, os.fsencode(path)))


def lbmp_load(h, path):
    _check(h, _lib().lbmp_load(h, os.fsencode(path)))


def lbmp_set_refinement_sensor(h, sigma_c, c):
    _check(h, _lib().lbmp_set_refinement_sensor(h, float(sigma_c), float(c)))


def lbmp_get_block_sensor(h, level):
    n = ctypes.c_size_t(0)
    _check(h, _lib().lbmp_get_block_sensor(h, int(level), None, 0, ctypes.byref(n)))
    out = np.empty(n.value, dtype=np.float64)
    _check(h, _lib().lbmp_get_block_sensor(h, int(level), _dp(out), out.size, ctypes.byref(n)))
    return out


def lbmp_get_block_map(h, level):
    n = ctypes.c_size_t(0)
    _check(h, _lib().lbmp_get_block_map(h, int(level), None, 0, ctypes.byref(n)))
    out = np.empty(n.value, dtype=np.int32)
    _check(h, _lib().lbmp_get_block_map(h, int(level), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), out.size,
                                        ctypes.byref(n)))
    return out


def lbmp_get_level_cells(h, level):
    n = ctypes.c_size_t(0)
    _check(h, _lib().lbmp_get_level_cells(h, int(level), None, None, 0, ctypes.byref(n)))
    xyz = np.empty((n.value, 3), dtype=np.int32)
    g = np.empty((n.value, 19), dtype=np.float64)
    if n.value:
        _check(h, _lib().lbmp_get_level_cells(h, int(level), xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                              _dp(g), n.value, ctypes.byref(n)))
    return xyz, g


def lbmp_get_level_flags(h, level):
    n = ctypes.c_size_t(0)
    _check(h, _lib().lbmp_get_level_flags(h, int(level), None, 0, ctypes.byref(n)))
    out = np.empty(n.value, dtype=np.uint8)
    if n.value:
        _check(h, _lib().lbmp_get_level_flags(h, int(level), out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                              n.value, ctypes.byref(n)))
    return out


def lbmp_updates_per_step(h):
    u, l = ctypes.c_int64(0), ctypes.c_int32(0)
    _check(h, _lib().lbmp_updates_per_step(h, ctypes.byref(u), ctypes.byref(l)))
    return u.value, l.value


def lbmp_batch_create(cfg, sims):
    """sims: sequence of dicts with edge, pos, diameter, density_ratio, cv, cv_omega, tau, gravity."""
    arr = (_native.LbmpBatchSim * len(sims))()
    for i, d in enumerate(sims):
        arr[i].edge = int(d["edge"])
        arr[i].pos = (ctypes.c_double * 3)(*[float(v) for v in d["pos"]])
        arr[i].diameter = float(d["diameter"])
        arr[i].density_ratio = float(d["density_ratio"])
        arr[i].cv = float(d.get("cv", 0.0))
        arr[i].cv_omega = float(d.get("cv_omega", d.get("cv", 0.0)))
        arr[i].tau = float(d["tau"])
        arr[i].gravity = (ctypes.c_double * 3)(*[float(v) for v in d.get("gravity", (0.0, 0.0, 0.0))])
    h = ctypes.c_void_p()
    _check(None, _lib().lbmp_batch_create(ctypes.byref(cfg), arr, len(sims), ctypes.byref(h)))
    return h


def lbmp_batch_autotune(h, reps=5):
    _check(h, _lib().lbmp_batch_autotune(h, int(reps)))


def lbmp_batch_info(h):
    out = (ctypes.c_int64 * 8)()
    _check(h, _lib().lbmp_batch_info(h, out))
    return tuple(out)


def lbmp_batch_get_populations(h, sim, edge):
    out = np.empty(19 * int(edge) ** 3, dtype=np.float64)
    _check(h, _lib().lbmp_batch_get_populations(h, int(sim), _dp(out), out.size))
    return out.reshape(19, -1)


def lbmp_last_error(h=None):
    m = _lib().lbmp_last_error(h)
    return m.decode() if m else ""


def lbmp_drag_forward(h, u0_ptr, nsteps, checkpoint_interval, axis, J_ptr, forces_ptr=0):
    """Device pointers: u0 [3][nz][ny][nx] float64, J one float64, forces [nsteps][3] float64 (0: not wanted)."""
    _check(h, _lib().lbmp_drag_forward(h, ctypes.c_void_p(u0_ptr), int(nsteps), int(checkpoint_interval), int(axis),
                                       ctypes.c_void_p(J_ptr), ctypes.c_void_p(forces_ptr or None)))


def lbmp_drag_backward(h, dJ_ptr, grad_tau_ptr, grad_force_ptr, grad_u0_ptr):
    """Device pointers (the three outputs may be 0 for 'not wanted')."""
    _check(h, _lib().lbmp_drag_backward(h, ctypes.c_void_p(dJ_ptr), ctypes.c_void_p(grad_tau_ptr or None),
                                        ctypes.c_void_p(grad_force_ptr or None),
                                        ctypes.c_void_p(grad_u0_ptr or None)))


# ------------------------------------------------------------ convenience
class _TorchAllocator:
    """Routes the library's device allocations through PyTorch's caching allocator."""

    def __init__(self, device, stream):
        import torch
        self._torch = torch
        self.device = device
        self.stream = stream

        def _alloc(nbytes, ctx):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream))
            except Exception:
                return None

        def _free(ptr, nbytes, ctx):
            try:
                torch.cuda.caching_allocator_delete(ptr)
            except Exception:
                pass

        self.alloc = _native.ALLOC_FN(_alloc)
        self.free = _native.FREE_FN(_free)


class Simulation:
    """One coupled LBM-MEM simulation on the current CUDA device."""

    def __init__(self, shape, precision="fp32", tau=0.6, magic=3.0 / 16.0, bc=("periodic",) * 3, boundary="cli",
                 force_average=True, history_capacity=4096, fp16_scale_log2=11, stream=None,
                 torch_allocator=True, levels=1, rescale=False, regrid_interval=0, bulk=1.0,
                 refill="equilibrium"):
        import torch
        if not torch.cuda.is_available():
            raise LbmpError(3, "no CUDA device: this library has no CPU path")
        cfg = lbmp_config_default()
        cfg.nx, cfg.ny, cfg.nz = (int(v) for v in shape)
        cfg.levels = int(levels)
        cfg.rescale_noneq = int(bool(rescale))
        cfg.regrid_interval = int(regrid_interval)
        cfg.bc = (ctypes.c_int * 3)(*[BC[b] for b in bc])
        cfg.precision = PRECISIONS[precision]
        cfg.tau = float(tau)
        cfg.magic = float(magic)
        cfg.bulk_factor = float(bulk)
        cfg.refill = REFILL[refill]
        cfg.boundary = BOUNDARY[boundary]
        cfg.force_average = int(bool(force_average))
        cfg.history_capacity = int(history_capacity)
        cfg.fp16_scale_log2 = int(fp16_scale_log2)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        cfg.cuda_stream = ctypes.c_void_p(self.stream.cuda_stream)
        self._allocator = None
        if torch_allocator:
            self._allocator = _TorchAllocator(torch.cuda.current_device(), self.stream)
            cfg.alloc = self._allocator.alloc
            cfg.free = self._allocator.free
        self.shape = tuple(int(v) for v in shape)
        self.ncells = self.shape[0] * self.shape[1] * self.shape[2]
        self.precision = precision
        self.h = lbmp_create(cfg)

    def close(self):
        if getattr(self, "h", None):
            lbmp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_sphere(self, pos, diameter, density_ratio, cv=0.0, cv_omega=None):
        return lbmp_add_sphere(self.h, pos, diameter, density_ratio, cv, cv_omega)

    def set_particle_velocity(self, u, omega=(0.0, 0.0, 0.0)):
        lbmp_set_particle_velocity(self.h, 0, u, omega)

    def set_fixed(self, fixed=True):
        """True: translation and rotation held; "translation": translation held, rotation free."""
        lbmp_set_particle_fixed(self.h, 0, fixed)

    def set_wall_velocity(self, axis, side, u):
        """Velocity of the domain wall on the low (0) or high (1) face of a non-periodic axis."""
        lbmp_set_wall_velocity(self.h, axis, side, u)

    def mean_drag(self, tau, force, u0, nsteps, checkpoint_interval=50, axis=0):
        """Differentiable mean drag on the fixed sphere; see mean_drag()."""
        return mean_drag(self, tau, force, u0, nsteps, checkpoint_interval, axis)

    def set_ga(self, ga, u_g=0.01, direction=(0.0, 0.0, -1.0)):
        lbmp_set_ga(self.h, ga, u_g, direction)

    def set_tau(self, tau):
        lbmp_set_tau(self.h, tau)

    def set_gravity(self, g):
        lbmp_set_gravity(self.h, g)

    def set_body_force(self, f):
        lbmp_set_body_force(self.h, f)

    def init_fluid(self, rho=1.0, u=(0.0, 0.0, 0.0), u_field=None):
        lbmp_init_fluid(self.h, rho, u, u_field)

    def set_populations(self, g):
        lbmp_set_populations(self.h, g)

    def populations(self):
        return lbmp_get_populations(self.h, self.ncells)

    def gather(self, cells):
        """Populations of the given cells, shape [len(cells), 19]."""
        return lbmp_gather_populations(self.h, cells)

    def step(self, n=1):
        lbmp_step(self.h, n)

    def step_async(self, n=1):
        lbmp_step_async(self.h, n)

    def check(self):
        lbmp_check_status(self.h)

    def synchronize(self):
        lbmp_synchronize(self.h)

    def particle(self):
        return lbmp_get_particle(self.h, 0)

    def history(self, max_steps=None):
        return lbmp_get_history(self.h, 0, max_steps)

    def flags(self):
        return lbmp_get_flags(self.h, self.ncells)

    def links(self):
        return lbmp_get_links(self.h)

    def init_fluid_wave(self, rho=1.0, u=(0.0, 0.0, 0.0), amp=0.0, direction=0, axis=2):
        lbmp_init_fluid_wave(self.h, rho, u, amp, direction, axis)

    def refine_box(self, lo, hi):
        lbmp_refine_box(self.h, lo, hi)

    def regrid(self):
        lbmp_regrid(self.h)

    def save(self, path):
        """Checkpoint of the whole state into the file `path`."""
        lbmp_save(self.h, path)

    def load(self, path):
        """Restores a checkpoint written by save() on a handle of the same grid."""
        lbmp_load(self.h, path)

    def set_refinement_sensor(self, sigma_c=1e-3, c=0.2):
        """Flow-based refinement sensor of Sec. 4.2.2 (sigma_c = 0 turns it off)."""
        lbmp_set_refinement_sensor(self.h, sigma_c, c)

    def block_sensor(self, level):
        """Largest scaled curl of every real block of a level (block order)."""
        return lbmp_get_block_sensor(self.h, level)

    def level_shape(self, level):
        return lbmp_level_shape(self.h, level)

    def block_map(self, level):
        return lbmp_get_block_map(self.h, level)

    def level_cells(self, level):
        return lbmp_get_level_cells(self.h, level)

    def level_flags(self, level):
        """Flags of a level's real cells in level_cells order (finest level: 1 solid, 2 next to the sphere)."""
        return lbmp_get_level_flags(self.h, level)

    def updates_per_step(self):
        """(cell updates, kernel launches) of one level-0 step."""
        return lbmp_updates_per_step(self.h)

    def counters(self):
        """(steps, cell updates, kernel launches, h2d bytes, d2h bytes)."""
        return lbmp_get_counters(self.h)

    def profile(self, enable=True):
        lbmp_profile(self.h, enable)

    def profile_result(self):
        """(stream-collide ms, its launches, step ms, steps, algorithmic bytes, cell updates)."""
        return lbmp_get_profile(self.h)


class BatchSimulation:
    """Many independent uniform periodic simulations advanced together."""

    def __init__(self, sims, precision="fp32", magic=3.0 / 16.0, boundary="cli", force_average=True,
                 history_capacity=4096, stream=None, torch_allocator=True, bulk=1.0,
                 refill="equilibrium"):
        import torch
        if not torch.cuda.is_available():
            raise LbmpError(3, "no CUDA device: this library has no CPU path")
        cfg = lbmp_config_default()
        cfg.precision = PRECISIONS[precision]
        cfg.magic = float(magic)
        cfg.bulk_factor = float(bulk)
        cfg.refill = REFILL[refill]
        cfg.boundary = BOUNDARY[boundary]
        cfg.force_average = int(bool(force_average))
        cfg.history_capacity = int(history_capacity)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        cfg.cuda_stream = ctypes.c_void_p(self.stream.cuda_stream)
        self._allocator = None
        if torch_allocator:
            self._allocator = _TorchAllocator(torch.cuda.current_device(), self.stream)
            cfg.alloc = self._allocator.alloc
            cfg.free = self._allocator.free
        self.sims = [dict(d) for d in sims]
        self.h = lbmp_batch_create(cfg, self.sims)

    def close(self):
        if getattr(self, "h", None):
            lbmp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        lbmp_step(self.h, n)

    def step_async(self, n=1):
        lbmp_step_async(self.h, n)

    def check(self):
        lbmp_check_status(self.h)

    def autotune(self, reps=5):
        lbmp_batch_autotune(self.h, reps)

    def info(self):
        return lbmp_batch_info(self.h)

    def particle(self, i):
        return lbmp_get_particle(self.h, i)

    def history(self, i, max_steps=None):
        return lbmp_get_history(self.h, i, max_steps)

    def populations(self, i):
        return lbmp_batch_get_populations(self.h, i, self.sims[i]["edge"])

    def counters(self):
        return lbmp_get_counters(self.h)

    def profile(self, enable=True):
        lbmp_profile(self.h, enable)

    def profile_result(self):
        return lbmp_get_profile(self.h)


# ----------------------------------------------------------- differentiation
_MEAN_DRAG = None


def _mean_drag_function():
    global _MEAN_DRAG
    if _MEAN_DRAG is not None:
        return _MEAN_DRAG
    import torch

    class MeanDrag(torch.autograd.Function):
        """J = (1/N) sum_n F_axis^n on the fixed sphere of a Simulation; the
        backward pass is the library's adjoint (lbmp_drag_backward)."""

        @staticmethod
        def forward(ctx, tau, force, u0, sim, nsteps, interval, axis):
            sim.set_tau(float(tau))
            sim.set_body_force([float(v) for v in force.detach().cpu()])
            dev = torch.device("cuda", torch.cuda.current_device())
            u = u0.detach().to(device=dev, dtype=torch.float64).contiguous()
            if tuple(u.shape) != (3, sim.shape[2], sim.shape[1], sim.shape[0]):
                raise ValueError("u0 must have shape (3, nz, ny, nx)")
            J = torch.empty((), dtype=torch.float64, device=dev)
            sim.stream.wait_stream(torch.cuda.current_stream())
            lbmp_drag_forward(sim.h, u.data_ptr(), nsteps, interval, axis, J.data_ptr())
            torch.cuda.current_stream().wait_stream(sim.stream)
            u.record_stream(sim.stream)
            ctx.sim = sim
            ctx.meta = (tau.dtype, tau.device, force.dtype, force.device, u0.dtype, u0.device, tuple(u0.shape))
            return J

        @staticmethod
        def backward(ctx, gJ):
            sim = ctx.sim
            tdt, tdev, fdt, fdev, udt, udev, ushape = ctx.meta
            dev = torch.device("cuda", torch.cuda.current_device())
            g = gJ.detach().to(device=dev, dtype=torch.float64).contiguous()
            gt = torch.empty((), dtype=torch.float64, device=dev)
            gf = torch.empty(3, dtype=torch.float64, device=dev)
            gu = torch.empty(ushape, dtype=torch.float64, device=dev) if ctx.needs_input_grad[2] else None
            sim.stream.wait_stream(torch.cuda.current_stream())
            lbmp_drag_backward(sim.h, g.data_ptr(), gt.data_ptr(), gf.data_ptr(), gu.data_ptr() if gu is not None else 0)
            torch.cuda.current_stream().wait_stream(sim.stream)
            return (gt.to(dtype=tdt, device=tdev) if ctx.needs_input_grad[0] else None,
                    gf.to(dtype=fdt, device=fdev) if ctx.needs_input_grad[1] else None,
                    gu.to(dtype=udt, device=udev) if gu is not None else None, None, None, None, None)

    _MEAN_DRAG = MeanDrag
    return MeanDrag


def mean_drag(sim, tau, force, u0, nsteps, checkpoint_interval=50, axis=0):
    """Mean drag J = (1/nsteps) sum_n F_axis^n on the fixed sphere of `sim`
    (a uniform periodic Simulation, FP32 or FP64) from the equilibrium of u0,
    as a torch scalar that autograd differentiates with respect to tau (0-d
    tensor), the body force (3-tensor) and u0 (tensor (3, nz, ny, nx)) by the
    library's adjoint with checkpoints every `checkpoint_interval` steps."""
    return _mean_drag_function().apply(tau, force, u0, sim, int(nsteps), int(checkpoint_interval), int(axis))
