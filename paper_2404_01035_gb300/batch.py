"""Python front end of the batched C ABI (ms_batch_*): argument marshalling only."""
from __future__ import annotations

import ctypes

import numpy as np

from ._binding import Grid, MSError, Params, TorchAllocator, lib
from .simulation import make_grid, make_params


class Batch:
    """Many independent 2-D simulations advanced by one persistent launch."""

    def __init__(self, probs, stream=None, torch_alloc: bool = True):
        import torch
        self._torch = torch
        L = lib()
        self.probs = list(probs)
        n = len(self.probs)
        self._keep = []
        grids = (Grid * n)(*[make_grid(p) for p in self.probs])
        params = (Params * n)(*[make_params(p, "f32", self._keep) for p in self.probs])
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self._alloc = TorchAllocator() if torch_alloc else None
        h = ctypes.c_void_p()
        p0 = self.probs[0]
        rc = L.ms_batch_create(n, grids, p0.n_phases, p0.n_components, params,
                               ctypes.c_void_p(stream.cuda_stream),
                               ctypes.byref(self._alloc.struct) if self._alloc else None, ctypes.byref(h))
        if rc != 0:
            raise MSError(rc, L.ms_last_error(None).decode())
        self.h = h
        self._keep = []

    def _c(self, rc):
        if rc != 0:
            raise MSError(rc, lib().ms_batch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().ms_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_fields(self, sim, phi, mu):
        p = self.probs[sim]
        phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float32))
        mu = np.ascontiguousarray(np.asarray(mu, dtype=np.float32))
        self._c(lib().ms_batch_set_fields(self.h, sim, phi.ctypes.data_as(ctypes.c_void_p),
                                          mu.ctypes.data_as(ctypes.c_void_p), 0))

    def get_fields(self, sim):
        p = self.probs[sim]
        shape = (1, p.ny, p.nx)
        phi = np.empty((p.n_phases,) + shape, dtype=np.float32)
        mu = np.empty((p.n_components - 1,) + shape, dtype=np.float32)
        self._c(lib().ms_batch_get_fields(self.h, sim, phi.ctypes.data_as(ctypes.c_void_p),
                                          mu.ctypes.data_as(ctypes.c_void_p), 0))
        return phi, mu

    def step(self, n: int):
        self._c(lib().ms_batch_step(self.h, int(n)))

    def sync(self):
        self._c(lib().ms_batch_sync(self.h))

    @property
    def cells(self) -> int:
        return lib().ms_batch_cells(self.h)

    def set_tile(self, tile_height: int):
        """Tile height of the work list (4, 8 or 16 rows of 32 cells)."""
        self._c(lib().ms_batch_set_tile(self.h, int(tile_height)))

    def tile_height(self) -> int:
        return lib().ms_batch_tile(self.h)

    def tune(self, steps_per_trial: int = 50) -> float:
        """Time every compiled tile height on the current states (restored
        afterwards) and keep the fastest; returns its ms per step."""
        out = ctypes.c_double(0.0)
        self._c(lib().ms_batch_tune(self.h, int(steps_per_trial), ctypes.byref(out)))
        return out.value
