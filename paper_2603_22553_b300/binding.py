"""ctypes binding of the C ABI declared in ``include/lpc3d.h``.

Argument marshalling only: every step of the lattice update runs in the CUDA
library ``liblpc3d.so``.  The functions keep the C names.  Loading fails
loudly when the library is missing; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblpc3d.so")

LPC_OK, LPC_ERR_INVALID, LPC_ERR_OOM, LPC_ERR_CUDA, LPC_ERR_TIMEOUT, LPC_ERR_STATE = range(6)
LPC_WEIGHTS_F32, LPC_WEIGHTS_BF16 = 0, 1
LPC_INIT_UNIFORM, LPC_INIT_BOLTZMANN = 0, 1
LPC_KERNEL_AUTO, LPC_KERNEL_STEP1, LPC_KERNEL_TB = 0, 1, 2
LPC_STATIC_AUTO, LPC_STATIC_GATHER, LPC_STATIC_LINK = 0, 1, 2
LPC_PLANE_FIRST, LPC_PLANE_LAST, LPC_PLANE_HALO_BELOW, LPC_PLANE_HALO_ABOVE = 0, 1, 2, 3

STATUS_NAMES = {0: "LPC_OK", 1: "LPC_ERR_INVALID", 2: "LPC_ERR_OOM", 3: "LPC_ERR_CUDA",
                4: "LPC_ERR_TIMEOUT", 5: "LPC_ERR_STATE"}


class lpc_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("periodic", ctypes.c_int32 * 3), ("alpha", ctypes.c_double),
                ("dt", ctypes.c_double), ("kT", ctypes.c_double),
                ("weight_dtype", ctypes.c_int32), ("msd_axes", ctypes.c_int32),
                ("init", ctypes.c_int32), ("ghost", ctypes.c_int32)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class lpc_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


class lpc_reservoir(ctypes.Structure):
    _fields_ = [("enabled", ctypes.c_int32), ("reserved", ctypes.c_int32), ("F", ctypes.c_double),
                ("rho", ctypes.c_double), ("m_re", ctypes.c_double), ("m_im", ctypes.c_double)]


LPC_MAX_REGIONS = 4


class lpc_options(ctypes.Structure):
    _fields_ = [("alpha_links", ctypes.POINTER(ctypes.c_double)), ("reservoir", lpc_reservoir * 6),
                ("region", ctypes.POINTER(ctypes.c_uint8)), ("n_regions", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class lpc_plane_set(ctypes.Structure):
    _fields_ = [("plane", ctypes.c_void_p * 5), ("bytes", ctypes.c_int64 * 5)]


class lpc_info(ctypes.Structure):
    _fields_ = [("n_sites", ctypes.c_int64), ("n_padded", ctypes.c_int64),
                ("ghost", ctypes.c_int32), ("pitch_x", ctypes.c_int32),
                ("pitch_y", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("block_steps", ctypes.c_int32), ("static_form", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("bytes_per_site_update", ctypes.c_int64),
                ("tile_rows", ctypes.c_int32), ("items_per_cta", ctypes.c_int32)]


_H = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_FP = ctypes.POINTER(ctypes.c_float)
_U8P = ctypes.POINTER(ctypes.c_uint8)
_I64P = ctypes.POINTER(ctypes.c_int64)

# name -> (restype, argtypes); the same list is the symbol table the CPU tests
# check against include/lpc3d.h.
SIGNATURES = {
    "lattice_create": (ctypes.c_int, [ctypes.POINTER(lpc_params), _DP, _DP, _U8P, _DP,
                                      ctypes.POINTER(lpc_allocator), ctypes.c_void_p,
                                      ctypes.POINTER(_H)]),
    "lattice_create_links": (ctypes.c_int, [ctypes.POINTER(lpc_params), _DP, _DP, _U8P, _DP, _DP,
                                            ctypes.POINTER(lpc_allocator), ctypes.c_void_p,
                                            ctypes.POINTER(_H)]),
    "lattice_create_ex": (ctypes.c_int, [ctypes.POINTER(lpc_params), ctypes.POINTER(lpc_options), _DP, _DP,
                                         _U8P, _DP, ctypes.POINTER(lpc_allocator), ctypes.c_void_p,
                                         ctypes.POINTER(_H)]),
    "lattice_create_slab": (ctypes.c_int, [ctypes.POINTER(lpc_params), ctypes.c_int32, ctypes.POINTER(lpc_options),
                                           _DP, _DP, _U8P, _DP, ctypes.POINTER(lpc_allocator), ctypes.c_void_p,
                                           ctypes.POINTER(_H)]),
    "lattice_slab_planes": (ctypes.c_int, [_H, ctypes.c_int32, ctypes.POINTER(lpc_plane_set)]),
    "lattice_destroy": (ctypes.c_int, [_H]),
    "lattice_footprint": (ctypes.c_int, [ctypes.POINTER(lpc_params), ctypes.c_int64, _I64P]),
    "lattice_step_n": (ctypes.c_int, [_H, ctypes.c_int64]),
    "lattice_step_many": (ctypes.c_int, [ctypes.POINTER(_H), _I64P, ctypes.c_int32]),
    "lattice_set_schedule": (ctypes.c_int, [_H, ctypes.c_int32, ctypes.c_int32]),
    "lattice_set_static_form": (ctypes.c_int, [_H, ctypes.c_int32]),
    "lattice_set_tiling": (ctypes.c_int, [_H, ctypes.c_int32, ctypes.c_int32]),
    "lattice_sync": (ctypes.c_int, [_H]),
    "lattice_autotune": (ctypes.c_int, [_H, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int32), _DP]),
    "lattice_steps_done": (ctypes.c_int, [_H, _I64P]),
    "lattice_info": (ctypes.c_int, [_H, ctypes.POINTER(lpc_info)]),
    "lattice_fid": (ctypes.c_int, [_H, ctypes.c_int64, ctypes.c_int64, _DP]),
    "lattice_population": (ctypes.c_int, [_H, ctypes.c_int64, ctypes.c_int64, _DP]),
    "lattice_msd": (ctypes.c_int, [_H, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _DP]),
    "lattice_dmsd": (ctypes.c_int, [_H, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _DP]),
    "lattice_fid_region": (ctypes.c_int, [_H, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _DP]),
    "lattice_population_region": (ctypes.c_int, [_H, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _DP]),
    "lattice_msd_region": (ctypes.c_int, [_H, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                          _DP]),
    "lattice_density": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_int32]),
    "lattice_magnetization": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_int32]),
    "lattice_moment": (ctypes.c_int, [_H, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32]),
    "lattice_weights": (ctypes.c_int, [_H, _FP]),
    "lattice_rotation": (ctypes.c_int, [_H, _FP]),
    "lattice_solid": (ctypes.c_int, [_H, _U8P]),
    "lattice_state_size": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_size_t)]),
    "lattice_get_state": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_size_t]),
    "lattice_set_state": (ctypes.c_int, [_H, ctypes.c_void_p, ctypes.c_size_t]),
    "lattice_equilibrate": (ctypes.c_int, [_H, ctypes.c_double, ctypes.c_int64, ctypes.c_int32,
                                           _I64P, _DP]),
    "lpc_step_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_int32)] + [ctypes.c_void_p] * 8),
    "lpc_wait_selftest": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p]),
    "lpc_last_error": (ctypes.c_char_p, []),
    "lpc_version": (ctypes.c_char_p, []),
}

_lib = None


class LPCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


def load(path=None):
    """Load ``liblpc3d.so`` (raises if it is missing: no fallback)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError("liblpc3d.so not built (%s); run paper_2603_22553_b300.build" % p)
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def check(status, lib=None):
    if status != LPC_OK:
        lib = lib or load()
        raise LPCError(status, lib.lpc_last_error().decode(errors="replace"))
    return status
