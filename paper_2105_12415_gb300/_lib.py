"""ctypes binding of libmrdem.so: the C ABI of include/mrdem.h, same names.

Argument marshalling only.  Loading fails loudly when the library has not
been built; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import buildlib as _build

MRDEM_OK = 0
MRDEM_ERR_INVALID = -1
MRDEM_ERR_OOM = -2
MRDEM_ERR_CUDA = -3
MRDEM_ERR_CAPACITY = -4
MRDEM_ERR_NONFINITE = -5

MRDEM_PREC_FP32 = 0
MRDEM_PREC_FP64 = 1

MRDEM_STAT_LEVELS = 8
MRDEM_STAT_TESTS = 0
MRDEM_STAT_SURVIVORS = 8
MRDEM_STAT_TILES = 16
MRDEM_STAT_FINE_TESTS = 17
MRDEM_STAT_CANDIDATES = 18
MRDEM_STAT_UNCONVERGED = 19
MRDEM_STAT_CONTACTS = 20
MRDEM_STAT_FP64 = 21
MRDEM_STAT_SPHERE_TESTS = 22
MRDEM_STAT_FINE_SURROGATE = 23
MRDEM_STAT_LEVEL_SWEEPS = 24
MRDEM_STAT_NOALLOC_OVERFLOW = 25
MRDEM_STAT_NOALLOC_INVALID = 26
MRDEM_STAT_FINE_SWEEPS = 27
MRDEM_STAT_ITEMS_PT = 28
MRDEM_STAT_ITEMS_EE = 29
MRDEM_STAT_BOX_PRUNED = 30
MRDEM_STAT_COUNT = 32
MRDEM_STATUS_WORDS = 8


class mrdem_params(C.Structure):
    _fields_ = [
        ("n_iter", C.c_int32), ("rho_reg", C.c_float), ("rho_iter", C.c_float),
        ("conv_c", C.c_float), ("fanout", C.c_int32), ("leaf_max", C.c_int32),
        ("leaf_min", C.c_int32), ("kmeans_iters", C.c_int32), ("cap_level", C.c_int64),
        ("cap_tiles", C.c_int64), ("cap_candidates", C.c_int64), ("tile_warps", C.c_int32),
        ("sweep_warps", C.c_int32), ("level_warps", C.c_int32),
        ("exact_threads", C.c_int32), ("cap_sweep", C.c_int64), ("expand_items", C.c_int32),
        ("node_threads", C.c_int32), ("level_kernel", C.c_int32),
    ]


class mrdem_contacts(C.Structure):
    _fields_ = [
        ("capacity", C.c_int64), ("count", C.c_void_p), ("pair", C.c_void_p),
        ("tri_a", C.c_void_p), ("tri_b", C.c_void_p), ("dist", C.c_void_p),
        ("point_a", C.c_void_p), ("point_b", C.c_void_p),
    ]


class mrdem_active_set(C.Structure):
    _fields_ = [("capacity", C.c_int64), ("count", C.c_void_p), ("item", C.c_void_p)]


class mrdem_hier_info(C.Structure):
    _fields_ = [
        ("n_particles", C.c_int32), ("max_depth", C.c_int32), ("n_nodes", C.c_int64),
        ("n_tri", C.c_int64), ("n_tri_pad", C.c_int64), ("n_verts", C.c_int64),
    ]


# every symbol of include/mrdem.h with its ctypes signature
_P = C.c_void_p
_I = C.c_int32
_I64 = C.c_int64
_D = C.c_double
SIGNATURES = {
    "mrdem_default_params": (None, [C.POINTER(mrdem_params)]),
    "mrdem_status_string": (C.c_char_p, [C.c_int]),
    "mrdem_create": (C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(mrdem_params)]),
    "mrdem_destroy": (C.c_int, [_P]),
    "mrdem_get_params": (C.c_int, [_P, C.POINTER(mrdem_params)]),
    "mrdem_set_params": (C.c_int, [_P, C.POINTER(mrdem_params)]),
    "mrdem_reserve": (C.c_int, [_P, _I64, _I64, _I64, _I64]),
    "mrdem_build_hierarchy_host": (C.c_int, [C.POINTER(mrdem_params), _I, _P, _P, _P, _P,
                                             C.POINTER(_P)]),
    "mrdem_hier_upload": (C.c_int, [_P, _P]),
    "mrdem_build_hierarchy": (C.c_int, [_P, _I, _P, _P, _P, _P, C.POINTER(_P)]),
    "mrdem_hier_destroy": (C.c_int, [_P]),
    "mrdem_hier_get_info": (C.c_int, [_P, C.POINTER(mrdem_hier_info)]),
    "mrdem_hier_export": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "mrdem_hier_export_boxes": (C.c_int, [_P, _P]),
    "mrdem_detect": (C.c_int, [_P, _P, _I64, _P, _P, _P, _I, C.POINTER(mrdem_contacts), _P, _P]),
    "mrdem_check": (C.c_int, [_P, _P, _P]),
    "mrdem_contact_forces": (C.c_int, [_P, _P, _I64, _P, _P, _P, C.POINTER(mrdem_contacts), _P,
                                       _P, _D, _P, _P, _P]),
    "mrdem_contact_grad": (C.c_int, [_P, _P, _I64, _P, _P, _P, C.POINTER(mrdem_contacts), _P, _D,
                                     _D, _P, _P, _P, _P]),
    "mrdem_merge_contacts": (C.c_int, [_P, _I64, _P, C.POINTER(mrdem_contacts),
                                       C.POINTER(mrdem_contacts), _P, _P]),
    "mrdem_contact_hessian": (C.c_int, [_P, _P, _I64, _P, _P, _P, C.POINTER(mrdem_contacts), _P,
                                        _D, _P, _P, _P]),
    "mrdem_newton_residual": (C.c_int, [_P, _I, _P, _P, _P, _P, _P, _P, _D, _P, _P, _P]),
    "mrdem_newton_solve": (C.c_int, [_P, _I, _I64, _P, _P, _P, _P, _D, _P, _P, _I, _D, _I, _P,
                                     _P]),
    "mrdem_vel_axpy": (C.c_int, [_P, _I64, _D, _P, _P, _P, _P]),
    "mrdem_refine_contacts": (C.c_int, [_P, _P, _I64, _P, _P, _P, C.POINTER(mrdem_contacts),
                                        C.POINTER(mrdem_contacts), _P]),
    "mrdem_motion_bound": (C.c_int, [_P, _I, _P, _P, _P, _P, _P]),
    "mrdem_status_async": (C.c_int, [_P, _P, _P]),
    "mrdem_status_decode": (C.c_int, [_P, _P]),
    "mrdem_active_set_init": (C.c_int, [_P, _P, _I64, _P, C.POINTER(mrdem_active_set), _P]),
    "mrdem_active_set_step": (C.c_int, [_P, _P, _I64, _P, _P, _P, _I,
                                        C.POINTER(mrdem_active_set),
                                        C.POINTER(mrdem_active_set), C.POINTER(mrdem_contacts),
                                        C.POINTER(mrdem_contacts), _P, _P]),
    "mrdem_surrogate_forces": (C.c_int, [_P, _P, _I64, _P, _P, _P, C.POINTER(mrdem_contacts),
                                         _P, _P, _D, _D, _P, _P, _P]),
    "mrdem_broad_phase": (C.c_int, [_P, _I, _P, _P, _P, _D, _P, _P, _I64, _P, _P]),
    "mrdem_move_poses": (C.c_int, [_P, _I, _P, _P, _D, _P, _P]),
    "mrdem_picard_update": (C.c_int, [_P, _I, _P, _P, _P, _P, _P, _D, _P, _P, _P]),
    "mrdem_detect_plain_fp64": (C.c_int, [_P, _P, _I64, _P, _P, _P, C.POINTER(mrdem_contacts),
                                          _P]),
    "mrdem_triangle_distance": (C.c_int, [_P, _I64, _P, _P, _P, _I, _P, _P, _P, _P, _P, _P, _P,
                                          _P]),
    "mrdem_detect_noalloc": (C.c_int, [_P, _I64, _P, _P, _P, _I, C.POINTER(mrdem_contacts), _P,
                                       _P]),
    "mrdem_autotune": (C.c_int, [_P, _P, _I64, _P, _P, _P, _I, C.POINTER(mrdem_contacts), _I,
                                 _P, _P]),
    "mrdem_build_hierarchy_device": (C.c_int, [_P, _I, _P, _P, _P, _P, C.POINTER(_P), _P]),
    "mrdem_twist_grad": (C.c_int, [_P, _I, _P, _P, _P, _P]),
    "mrdem_profile": (C.c_int, [_P, _I]),
    "mrdem_profile_read": (C.c_int, [_P, _I, C.POINTER(C.c_char_p), _P, _P, C.POINTER(_I)]),
}

_lock = threading.Lock()
_lib = None


class MrdemError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} ({status})")


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmrdem.so (building it first if missing and allowed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"libmrdem.so not built ({path}); run build()")
            _build.build()
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def status_string(status: int) -> str:
    return load().mrdem_status_string(status).decode()


def check(status: int, what: str):
    if status != MRDEM_OK:
        raise MrdemError(status, what)


def default_params() -> mrdem_params:
    p = mrdem_params()
    load().mrdem_default_params(C.byref(p))
    return p
