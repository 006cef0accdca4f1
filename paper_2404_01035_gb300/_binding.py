"""ctypes binding of the C ABI in include/microsim_gb.h (argument marshalling only).

Every step of the method runs in the CUDA library; this module only converts
Python/NumPy/torch arguments into the C structs and pointers the ABI takes.
There is no fallback: if the compiled library is missing, importing
`lib()` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

MS_OK = 0
STATUS_NAMES = {0: "MS_OK", 1: "MS_ERR_ARG", 2: "MS_ERR_CUDA", 3: "MS_ERR_OOM",
                4: "MS_ERR_DT_UNSTABLE", 5: "MS_ERR_NONFINITE", 6: "MS_ERR_TIMEOUT",
                7: "MS_ERR_BOUNDS", 8: "MS_ERR_STATE", 9: "MS_ERR_UNSUPPORTED"}
MS_F32, MS_F64 = 0, 1
MS_BC_HALO = 16

# Every function the header declares (checked by the CPU test-suite).
EXPORTS = [
    "ms_create", "ms_check_params", "ms_destroy", "ms_last_error", "ms_update_params", "ms_set_fields",
    "ms_get_fields", "ms_fields", "ms_step", "ms_diag", "ms_set_diag_every", "ms_sync",
    "ms_time", "ms_checkpoint_bytes", "ms_checkpoint", "ms_restore", "ms_set_launch",
    "ms_tile_count", "ms_tile_shape", "ms_tile_split", "ms_get_launch", "ms_tune",
    "ms_shift", "ms_front", "ms_diag_noalloc",
    "ms_enable_checkpoints", "ms_grad_param_count", "ms_grad",
    "ms_batch_create", "ms_batch_destroy", "ms_batch_last_error", "ms_batch_set_fields",
    "ms_batch_get_fields", "ms_batch_step", "ms_batch_sync", "ms_batch_cells",
    "ms_halo_exchange", "ms_halo_mirror", "ms_selftest_timeout", "ms_peak_fp32",
    "ms_halo_plane_bytes", "ms_halo_pack", "ms_halo_unpack",
    "ms_batch_set_tile", "ms_batch_tile", "ms_batch_tune",
    "ms_ggs_create", "ms_ggs_destroy", "ms_ggs_last_error", "ms_ggs_set_fields", "ms_ggs_get_fields",
    "ms_ggs_step", "ms_ggs_sync", "ms_ggs_stats",
]


class MSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("dx", ctypes.c_double), ("bc", ctypes.c_int * 3),
                ("z_origin", ctypes.c_int)]


class Params(ctypes.Structure):
    _fields_ = [
        ("dtype", ctypes.c_int), ("potential", ctypes.c_int), ("eps", ctypes.c_double),
        ("tau", ctypes.c_double), ("dt", ctypes.c_double),
        ("gamma", ctypes.c_void_p), ("delta", ctypes.c_void_p), ("rot", ctypes.c_void_p),
        ("gamma3", ctypes.c_void_p), ("D", ctypes.c_void_p), ("A", ctypes.c_void_p),
        ("ceq", ctypes.c_void_p), ("slopes", ctypes.c_void_p), ("f0", ctypes.c_void_p),
        ("T_ref", ctypes.c_double), ("T0", ctypes.c_double), ("G", ctypes.c_double),
        ("z0", ctypes.c_double), ("V", ctypes.c_double), ("t0", ctypes.c_double),
        ("noise_amp", ctypes.c_double), ("noise_seed", ctypes.c_ulonglong),
        ("anti_trapping", ctypes.c_int), ("grain_growth", ctypes.c_int),
        ("elastic_C", ctypes.c_void_p), ("eigenstrain", ctypes.c_void_p),
    ]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("release", FREE_FN), ("user", ctypes.c_void_p)]


_lock = threading.Lock()
_lib = None


def lib(build_if_missing: bool = True):
    """Load libmicrosim_gb.so (building it first when allowed); raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise ImportError(f"CUDA library not built: {path}")
        L = ctypes.CDLL(path)
        vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        L.ms_create.argtypes = [ctypes.POINTER(Grid), ctypes.c_int, ctypes.c_int,
                                ctypes.POINTER(Params), vp, ctypes.POINTER(Allocator),
                                ctypes.POINTER(vp)]
        L.ms_check_params.argtypes = [ctypes.POINTER(Grid), ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(Params), dp]
        L.ms_destroy.argtypes = [vp]
        L.ms_destroy.restype = None
        L.ms_last_error.argtypes = [vp]
        L.ms_last_error.restype = ctypes.c_char_p
        L.ms_update_params.argtypes = [vp, ctypes.POINTER(Params)]
        L.ms_set_fields.argtypes = [vp, vp, vp, ctypes.c_int]
        L.ms_get_fields.argtypes = [vp, vp, vp, ctypes.c_int]
        L.ms_fields.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i64)]
        L.ms_step.argtypes = [vp, i64]
        L.ms_diag.argtypes = [vp, dp]
        L.ms_set_diag_every.argtypes = [vp, i64]
        L.ms_sync.argtypes = [vp]
        L.ms_time.argtypes = [vp, ctypes.POINTER(i64), dp]
        L.ms_checkpoint_bytes.argtypes = [vp]
        L.ms_checkpoint_bytes.restype = ctypes.c_size_t
        L.ms_checkpoint.argtypes = [vp, vp, ctypes.c_size_t]
        L.ms_restore.argtypes = [vp, vp, ctypes.c_size_t]
        L.ms_set_launch.argtypes = [vp, ctypes.c_int, ctypes.c_int]
        L.ms_tile_count.argtypes = [vp]
        L.ms_tile_shape.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int)]
        L.ms_shift.argtypes = [vp, ctypes.c_int, dp]
        L.ms_front.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        L.ms_tile_split.argtypes = [vp, ctypes.c_int]
        L.ms_get_launch.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.ms_tune.argtypes = [vp, ctypes.c_char_p, ctypes.c_int, dp]
        L.ms_batch_create.argtypes = [ctypes.c_int, ctypes.POINTER(Grid), ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(Params), vp, ctypes.POINTER(Allocator),
                                      ctypes.POINTER(vp)]
        L.ms_batch_destroy.argtypes = [vp]
        L.ms_batch_destroy.restype = None
        L.ms_batch_last_error.argtypes = [vp]
        L.ms_batch_last_error.restype = ctypes.c_char_p
        L.ms_batch_set_fields.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_int]
        L.ms_batch_get_fields.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_int]
        L.ms_batch_step.argtypes = [vp, i64]
        L.ms_batch_sync.argtypes = [vp]
        L.ms_batch_cells.argtypes = [vp]
        L.ms_batch_cells.restype = ctypes.c_int64
        L.ms_batch_set_tile.argtypes = [vp, ctypes.c_int]
        L.ms_batch_tile.argtypes = [vp]
        L.ms_batch_tune.argtypes = [vp, ctypes.c_int, dp]
        L.ms_ggs_create.argtypes = [ctypes.POINTER(Grid), ctypes.c_int, ctypes.POINTER(Params), vp,
                                    ctypes.POINTER(Allocator), ctypes.POINTER(vp)]
        L.ms_ggs_destroy.argtypes = [vp]
        L.ms_ggs_destroy.restype = None
        L.ms_ggs_last_error.argtypes = [vp]
        L.ms_ggs_last_error.restype = ctypes.c_char_p
        L.ms_ggs_set_fields.argtypes = [vp, vp, ctypes.c_int]
        L.ms_ggs_get_fields.argtypes = [vp, vp, ctypes.c_int]
        L.ms_ggs_step.argtypes = [vp, i64]
        L.ms_ggs_sync.argtypes = [vp]
        L.ms_ggs_stats.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.ms_halo_exchange.argtypes = [vp, vp]
        L.ms_halo_mirror.argtypes = [vp, ctypes.c_int]
        L.ms_halo_plane_bytes.argtypes = [vp]
        L.ms_halo_plane_bytes.restype = ctypes.c_size_t
        L.ms_halo_pack.argtypes = [vp, ctypes.c_int, vp]
        L.ms_halo_unpack.argtypes = [vp, ctypes.c_int, vp]
        L.ms_selftest_timeout.argtypes = [vp, i64]
        L.ms_peak_fp32.argtypes = [vp, ctypes.c_int, dp]
        L.ms_enable_checkpoints.argtypes = [vp, ctypes.c_int]
        L.ms_grad_param_count.argtypes = [vp]
        L.ms_grad.argtypes = [vp, vp, vp, dp, vp, vp]
        L.ms_diag_noalloc.argtypes = [ctypes.POINTER(Grid), ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(Params), ctypes.c_double, vp, vp, vp, vp]
        for name in EXPORTS:
            if name not in ("ms_destroy", "ms_last_error", "ms_checkpoint_bytes", "ms_batch_destroy",
                            "ms_batch_last_error", "ms_batch_cells", "ms_halo_plane_bytes",
                            "ms_ggs_destroy", "ms_ggs_last_error"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
        return _lib


def _check(status, ctx=None):
    if status != MS_OK:
        msg = lib().ms_last_error(ctx).decode(errors="replace")
        raise MSError(status, msg)


def _dev_ptr(x):
    """Device pointer of a torch tensor / __cuda_array_interface__ object, else None."""
    if hasattr(x, "data_ptr") and getattr(x, "is_cuda", False):
        return x.data_ptr()
    cai = getattr(x, "__cuda_array_interface__", None)
    if cai is not None:
        return cai["data"][0]
    return None


class _DeviceView:
    """Minimal __cuda_array_interface__ wrapper over a borrowed device pointer."""

    def __init__(self, ptr, shape, strides_elems, typestr, itemsize, owner):
        self.__cuda_array_interface__ = {
            "data": (ptr, False), "shape": tuple(shape), "typestr": typestr,
            "strides": tuple(s * itemsize for s in strides_elems), "version": 3,
        }
        self._owner = owner


class TorchAllocator:
    """Routes the library's device allocations through torch's caching allocator."""

    def __init__(self):
        import torch
        self._torch = torch
        self._live = {}
        self._alloc = ALLOC_FN(self._do_alloc)
        self._free = FREE_FN(self._do_free)
        self.struct = Allocator(self._alloc, self._free, None)

    def _do_alloc(self, nbytes, user):
        try:
            t = self._torch.empty(int(nbytes), dtype=self._torch.uint8, device="cuda")
        except Exception:
            return None
        self._live[t.data_ptr()] = t
        return t.data_ptr()

    def _do_free(self, ptr, user):
        self._live.pop(ptr, None)
