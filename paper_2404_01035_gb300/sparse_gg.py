"""Python front end of the sparse grain-growth C ABI (ms_ggs_*): argument
marshalling only.  A problem is any object with the fields of
workloads.Problem (grid, gamma, gamma3, eps, tau, dt); the grains' fields are
dense [N][z][y][x] arrays at the boundary, sparse inside the library."""
from __future__ import annotations

import ctypes

import numpy as np

from ._binding import MSError, TorchAllocator, _dev_ptr, lib
from .simulation import make_grid, make_params


class SparseGrainGrowth:
    """Isotropic grain growth with few grains stored per cell (ms_ggs_*)."""

    def __init__(self, prob, dtype: str = "f32", stream=None, torch_alloc: bool = True):
        import torch
        self._torch = torch
        self.prob = prob
        self.dtype = "f64" if dtype in ("f64", "float64", "double") else "f32"
        self.np_dtype = np.float64 if self.dtype == "f64" else np.float32
        self.N = int(prob.n_phases)
        self.shape = (int(prob.nz) if prob.dim == 3 else 1, int(prob.ny), int(prob.nx))
        keep = []
        params = make_params(prob, self.dtype, keep)
        grid = make_grid(prob)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self._alloc = TorchAllocator() if torch_alloc else None
        h = ctypes.c_void_p()
        rc = lib().ms_ggs_create(ctypes.byref(grid), self.N, ctypes.byref(params),
                                 ctypes.c_void_p(stream.cuda_stream),
                                 ctypes.byref(self._alloc.struct) if self._alloc else None, ctypes.byref(h))
        if rc != 0:
            raise MSError(rc, lib().ms_ggs_last_error(None).decode(errors="replace"))
        self.h = h

    def _c(self, rc):
        if rc != 0:
            raise MSError(rc, lib().ms_ggs_last_error(self.h).decode(errors="replace"))

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().ms_ggs_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fields(self, phi):
        ptr = _dev_ptr(phi)
        if ptr is not None:
            self._c(lib().ms_ggs_set_fields(self.h, ctypes.c_void_p(ptr), 1))
        else:
            a = np.ascontiguousarray(np.asarray(phi, dtype=self.np_dtype).reshape((self.N,) + self.shape))
            self._c(lib().ms_ggs_set_fields(self.h, a.ctypes.data_as(ctypes.c_void_p), 0))

    def get_fields(self):
        out = np.empty((self.N,) + self.shape, dtype=self.np_dtype)
        self._c(lib().ms_ggs_get_fields(self.h, out.ctypes.data_as(ctypes.c_void_p), 0))
        return out

    def step(self, n: int = 1):
        self._c(lib().ms_ggs_step(self.h, int(n)))

    def sync(self):
        self._c(lib().ms_ggs_sync(self.h))

    def stats(self):
        """(cells listed by the last step, step count)."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        self._c(lib().ms_ggs_stats(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value
