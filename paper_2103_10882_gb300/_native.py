"""ctypes declarations of the C ABI in include/lbmp.h (argument marshalling only)."""
import ctypes
import os

from . import build as _build

c_double_p = ctypes.POINTER(ctypes.c_double)

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class LbmpConfig(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("levels", ctypes.c_int),
        ("bc", ctypes.c_int * 3),
        ("precision", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("magic", ctypes.c_double),
        ("boundary", ctypes.c_int),
        ("force_average", ctypes.c_int),
        ("rescale_noneq", ctypes.c_int),
        ("regrid_interval", ctypes.c_int),
        ("history_capacity", ctypes.c_int),
        ("fp16_scale_log2", ctypes.c_int),
        ("cuda_stream", ctypes.c_void_p),
        ("alloc", ALLOC_FN),
        ("free", FREE_FN),
        ("alloc_ctx", ctypes.c_void_p),
        ("bulk_factor", ctypes.c_double),
        ("refill", ctypes.c_int),
    ]


class LbmpBatchSim(ctypes.Structure):
    _fields_ = [
        ("edge", ctypes.c_int),
        ("pos", ctypes.c_double * 3),
        ("diameter", ctypes.c_double),
        ("density_ratio", ctypes.c_double),
        ("cv", ctypes.c_double),
        ("cv_omega", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("gravity", ctypes.c_double * 3),
    ]


# name -> (restype, argtypes); every entry point declared in include/lbmp.h
SIGNATURES = {
    "lbmp_config_default": (ctypes.c_int, [ctypes.POINTER(LbmpConfig)]),
    "lbmp_create": (ctypes.c_int, [ctypes.POINTER(LbmpConfig), ctypes.POINTER(ctypes.c_void_p)]),
    "lbmp_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "lbmp_add_sphere": (ctypes.c_int, [ctypes.c_void_p, c_double_p, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]),
    "lbmp_set_particle_velocity": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_double_p, c_double_p]),
    "lbmp_set_particle_fixed": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "lbmp_set_wall_velocity": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, c_double_p]),
    "lbmp_ga_parameters": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          c_double_p, c_double_p, c_double_p]),
    "lbmp_set_ga": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, c_double_p]),
    "lbmp_set_tau": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "lbmp_set_gravity": (ctypes.c_int, [ctypes.c_void_p, c_double_p]),
    "lbmp_set_body_force": (ctypes.c_int, [ctypes.c_void_p, c_double_p]),
    "lbmp_init_fluid": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, c_double_p, ctypes.c_void_p,
                                       ctypes.c_int]),
    "lbmp_set_populations": (ctypes.c_int, [ctypes.c_void_p, c_double_p, ctypes.c_size_t]),
    "lbmp_get_populations": (ctypes.c_int, [ctypes.c_void_p, c_double_p, ctypes.c_size_t]),
    "lbmp_gather_populations": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_size_t,
                                               c_double_p]),
    "lbmp_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lbmp_step_async": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lbmp_check_status": (ctypes.c_int, [ctypes.c_void_p]),
    "lbmp_synchronize": (ctypes.c_int, [ctypes.c_void_p]),
    "lbmp_get_particle": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_double_p]),
    "lbmp_get_history": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_double_p, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int)]),
    "lbmp_get_flags": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint8), ctypes.c_size_t]),
    "lbmp_get_links": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_int32), c_double_p, ctypes.c_size_t,
                                      ctypes.POINTER(ctypes.c_size_t)]),
    "lbmp_get_counters": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "lbmp_profile": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lbmp_get_profile": (ctypes.c_int, [ctypes.c_void_p, c_double_p]),
    "lbmp_boundary_cells_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   ctypes.POINTER(ctypes.c_int), c_double_p, ctypes.c_double,
                                                   ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "lbmp_init_fluid_wave": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, c_double_p, ctypes.c_double,
                                            ctypes.c_int, ctypes.c_int]),
    "lbmp_refine_box": (ctypes.c_int, [ctypes.c_void_p, c_double_p, c_double_p]),
    "lbmp_regrid": (ctypes.c_int, [ctypes.c_void_p]),
    "lbmp_save": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "lbmp_load": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "lbmp_set_refinement_sensor": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double]),
    "lbmp_get_block_sensor": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_double_p, ctypes.c_size_t,
                                             ctypes.POINTER(ctypes.c_size_t)]),
    "lbmp_level_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "lbmp_get_block_map": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "lbmp_get_level_cells": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                                            c_double_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "lbmp_get_level_flags": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_uint8),
                                            ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "lbmp_updates_per_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                             ctypes.POINTER(ctypes.c_int32)]),
    "lbmp_batch_create": (ctypes.c_int, [ctypes.POINTER(LbmpConfig), ctypes.POINTER(LbmpBatchSim), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_void_p)]),
    "lbmp_batch_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "lbmp_batch_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "lbmp_batch_get_populations": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_double_p, ctypes.c_size_t]),
    "lbmp_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "lbmp_drag_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "lbmp_drag_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads liblbmp.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("liblbmp.so is not built; run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L
