"""Python front end of the C ABI: one simulation context.

`Simulation` mirrors ms_create / ms_set_fields / ms_step / ms_fields /
ms_diag / ms_checkpoint; it only marshals arguments.  Problems are described
by any object carrying the fields of `workloads.Problem` (grid, boundary
codes and the paper's raw model inputs).
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._binding import (MS_F32, MS_F64, Grid, MSError, Params, TorchAllocator, _check,
                       _DeviceView, _dev_ptr, lib)


def _arr(keep, x, shape):
    if x is None:
        return None
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(shape))
    keep.append(a)
    return a.ctypes.data


def make_params(prob, dtype: str, keep: list, **override) -> Params:
    g = lambda k: override.get(k, getattr(prob, k))
    N = int(g("n_phases"))
    NM = int(g("n_components")) - 1
    p = Params()
    p.dtype = MS_F64 if dtype in ("f64", "float64", "double") else MS_F32
    p.potential = 1 if g("potential") == "obstacle" else 2
    p.eps, p.tau, p.dt = float(g("eps")), float(g("tau")), float(g("dt"))
    p.gamma = _arr(keep, g("gamma"), (N, N))
    p.delta = _arr(keep, g("delta"), (N, N))
    p.rot = _arr(keep, g("rot"), (N, N, 3, 3))
    p.gamma3 = _arr(keep, g("gamma3"), (N, N, N))
    p.D = _arr(keep, g("D"), (N, NM, NM))
    p.A = _arr(keep, g("A"), (N, NM, NM))
    p.ceq = _arr(keep, g("ceq"), (N, NM))
    p.slopes = _arr(keep, g("slopes"), (N, NM))
    p.f0 = _arr(keep, g("f0"), (N,))
    p.T_ref, p.T0, p.G = float(g("T_ref")), float(g("T0")), float(g("G"))
    p.z0, p.V = float(g("z0")), float(g("V"))
    p.t0 = float(override.get("t0", 0.0))
    p.noise_amp = float(override.get("noise_amp", getattr(prob, "noise_amp", 0.0)))
    p.noise_seed = int(override.get("noise_seed", getattr(prob, "noise_seed", 0))) & 0xFFFFFFFFFFFFFFFF
    p.anti_trapping = int(bool(override.get("anti_trapping", getattr(prob, "anti_trapping", 0))))
    p.grain_growth = int(bool(override.get("grain_growth", getattr(prob, "grain_growth", 0))))
    C = override.get("elastic_C", getattr(prob, "elastic_C", None))
    if C is not None:
        p.elastic_C = _arr(keep, C, (6, 6))
        p.eigenstrain = _arr(keep, override.get("eigenstrain", getattr(prob, "eigenstrain", None)), (N, 3, 3))
    return p


def make_grid(prob) -> Grid:
    gr = Grid()
    gr.dim, gr.nx, gr.ny = int(prob.dim), int(prob.nx), int(prob.ny)
    gr.nz = int(prob.nz) if prob.dim == 3 else 1
    gr.dx = float(prob.dx)
    bc = list(prob.bc) + [3, 3, 3]
    gr.bc = (ctypes.c_int * 3)(*bc[:3])
    gr.z_origin = int(getattr(prob, "meta", {}).get("z_origin", 0))
    return gr


def check_params(prob, dtype: str = "f32", **override) -> float:
    """The library's checks of ms_create, without a device (ms_check_params).
    Returns the explicit stability bound on dt.  A failed check raises MSError,
    with the bound (when it was reached) as its `dt_bound` attribute."""
    keep = []
    params = make_params(prob, dtype, keep, **override)
    grid = make_grid(prob)
    bound = ctypes.c_double(0.0)
    rc = lib().ms_check_params(ctypes.byref(grid), int(prob.n_phases), int(prob.n_components),
                               ctypes.byref(params), ctypes.byref(bound))
    if rc != 0:
        err = MSError(rc, lib().ms_last_error(None).decode(errors="replace"))
        err.dt_bound = bound.value or None
        raise err
    return bound.value


class Simulation:
    """One grand-potential simulation living on the GPU."""

    def __init__(self, prob, dtype: str = "f32", stream=None, torch_alloc: bool = True,
                 allocator=None, **override):
        import torch
        self._torch = torch
        L = lib()
        self.prob = prob
        self.dtype = "f64" if dtype in ("f64", "float64", "double") else "f32"
        self.np_dtype = np.float64 if self.dtype == "f64" else np.float32
        self.torch_dtype = torch.float64 if self.dtype == "f64" else torch.float32
        self.N = int(prob.n_phases)
        self.NM = int(prob.n_components) - 1
        self.shape = (int(prob.nz) if prob.dim == 3 else 1, int(prob.ny), int(prob.nx))
        self._keep = []
        params = make_params(prob, self.dtype, self._keep, **override)
        grid = make_grid(prob)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        # allocator: any object with a ctypes `struct` (an ms_allocator), e.g. a
        # TorchAllocator subclass; default torch's caching allocator
        self._alloc = allocator if allocator is not None else (TorchAllocator() if torch_alloc else None)
        h = ctypes.c_void_p()
        _check(L.ms_create(ctypes.byref(grid), self.N, int(prob.n_components),
                                ctypes.byref(params), ctypes.c_void_p(stream.cuda_stream),
                                ctypes.byref(self._alloc.struct) if self._alloc else None,
                                ctypes.byref(h)))
        self.h = h
        self._keep = []

    # -------------------------------------------------------------- lifecycle
    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().ms_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _c(self, status):
        _check(status, self.h)

    # ----------------------------------------------------------------- fields
    def set_fields(self, phi, mu):
        dp, dm = _dev_ptr(phi), _dev_ptr(mu)
        if dp is not None and dm is not None:
            assert phi.dtype == self.torch_dtype and mu.dtype == self.torch_dtype
            assert phi.is_contiguous() and mu.is_contiguous()
            self._c(lib().ms_set_fields(self.h, ctypes.c_void_p(dp), ctypes.c_void_p(dm), 1))
            return
        phi = np.ascontiguousarray(np.asarray(phi, dtype=self.np_dtype).reshape((self.N,) + self.shape))
        mu = np.ascontiguousarray(np.asarray(mu, dtype=self.np_dtype).reshape((self.NM,) + self.shape))
        self._c(lib().ms_set_fields(self.h, phi.ctypes.data_as(ctypes.c_void_p),
                                    mu.ctypes.data_as(ctypes.c_void_p), 0))
        self._host_keep = (phi, mu)
        self.sync_stream()

    def get_fields(self):
        phi = np.empty((self.N,) + self.shape, dtype=self.np_dtype)
        mu = np.empty((self.NM,) + self.shape, dtype=self.np_dtype)
        self._c(lib().ms_get_fields(self.h, phi.ctypes.data_as(ctypes.c_void_p),
                                    mu.ctypes.data_as(ctypes.c_void_p), 0))
        return phi, mu

    def get_fields_into(self, phi, mu, on_device: bool):
        """Copy the state into caller buffers (torch tensors or numpy arrays)."""
        if on_device:
            self._c(lib().ms_get_fields(self.h, ctypes.c_void_p(_dev_ptr(phi)),
                                        ctypes.c_void_p(_dev_ptr(mu)), 1))
        else:
            pp = phi.data_ptr() if hasattr(phi, "data_ptr") else phi.ctypes.data
            mp = mu.data_ptr() if hasattr(mu, "data_ptr") else mu.ctypes.data
            self._c(lib().ms_get_fields(self.h, ctypes.c_void_p(pp), ctypes.c_void_p(mp), 0))

    def set_fields_from(self, phi, mu, on_device: bool):
        if on_device:
            self._c(lib().ms_set_fields(self.h, ctypes.c_void_p(_dev_ptr(phi)),
                                        ctypes.c_void_p(_dev_ptr(mu)), 1))
        else:
            pp = phi.data_ptr() if hasattr(phi, "data_ptr") else phi.ctypes.data
            mp = mu.data_ptr() if hasattr(mu, "data_ptr") else mu.ctypes.data
            self._c(lib().ms_set_fields(self.h, ctypes.c_void_p(pp), ctypes.c_void_p(mp), 0))

    def fields(self):
        """Zero-copy torch views (phi[N,nz,ny,nx], mu[K-1,nz,ny,nx]) of the current state."""
        torch = self._torch
        pp, mp = ctypes.c_void_p(), ctypes.c_void_p()
        strides = (ctypes.c_int64 * 4)()
        self._c(lib().ms_fields(self.h, ctypes.byref(pp), ctypes.byref(mp), strides))
        it = 8 if self.dtype == "f64" else 4
        ts = "<f8" if self.dtype == "f64" else "<f4"
        st = list(strides)
        vp = _DeviceView(pp.value, (self.N,) + self.shape, st, ts, it, self)
        vm = _DeviceView(mp.value, (self.NM,) + self.shape, st, ts, it, self)
        return torch.as_tensor(vp, device="cuda"), torch.as_tensor(vm, device="cuda")

    # --------------------------------------------------------------- stepping
    def step(self, n: int = 1):
        self._c(lib().ms_step(self.h, int(n)))

    def selftest_timeout(self, limit_ns: int = 1_000_000):
        """Enqueue the bounded-wait self-test (include/microsim_gb.h)."""
        self._c(lib().ms_selftest_timeout(self.h, int(limit_ns)))

    def sync(self):
        self._c(lib().ms_sync(self.h))

    def sync_stream(self):
        self.stream.synchronize()

    def diag(self):
        out = np.zeros(self.NM + 7)
        self._c(lib().ms_diag(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return {"mass": out[:self.NM].copy(), "sum_err": out[self.NM], "phi_min": out[self.NM + 1],
                "phi_max": out[self.NM + 2], "nonfinite": out[self.NM + 3],
                "mu_diffusion_number": out[self.NM + 4], "step": int(out[self.NM + 5]),
                "t": out[self.NM + 6]}

    def set_diag_every(self, k: int):
        self._c(lib().ms_set_diag_every(self.h, int(k)))

    def time(self):
        s, t = ctypes.c_int64(), ctypes.c_double()
        self._c(lib().ms_time(self.h, ctypes.byref(s), ctypes.byref(t)))
        return s.value, t.value

    def update_params(self, **override):
        keep = []
        params = make_params(self.prob, self.dtype, keep, **override)
        self._c(lib().ms_update_params(self.h, ctypes.byref(params)))

    # --------------------------------------------------------------- adjoint
    def enable_checkpoints(self, every: int):
        self._c(lib().ms_enable_checkpoints(self.h, int(every)))

    def param_count(self) -> int:
        return lib().ms_grad_param_count(self.h)

    def grad(self, dphi_T, dmu_T=None, want_fields: bool = True):
        """Reverse pass; dphi_T / dmu_T are torch CUDA tensors shaped like the fields.

        Returns (dparams [numpy, FP64], dphi0, dmu0 [torch tensors or None]).
        dparams = [dL/d delta_ab for pairs a < b..., dL/d(1/tau), dL/dD^a_ij ...].
        """
        torch = self._torch
        dphi_T = dphi_T.to(self.torch_dtype).contiguous()
        dmu_T = None if dmu_T is None else dmu_T.to(self.torch_dtype).contiguous()
        out = np.zeros(self.param_count())
        dphi0 = torch.empty_like(dphi_T) if want_fields else None
        dmu0 = (torch.empty((self.NM,) + self.shape, dtype=self.torch_dtype, device="cuda")
                if want_fields else None)
        self._c(lib().ms_grad(self.h, ctypes.c_void_p(dphi_T.data_ptr()),
                              ctypes.c_void_p(dmu_T.data_ptr()) if dmu_T is not None else None,
                              out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                              ctypes.c_void_p(dphi0.data_ptr()) if dphi0 is not None else None,
                              ctypes.c_void_p(dmu0.data_ptr()) if dmu0 is not None else None))
        return out, dphi0, dmu0

    # ------------------------------------------------------------ checkpoints
    def checkpoint(self) -> bytes:
        n = lib().ms_checkpoint_bytes(self.h)
        buf = ctypes.create_string_buffer(n)
        self._c(lib().ms_checkpoint(self.h, buf, n))
        return buf.raw

    def restore(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        self._c(lib().ms_restore(self.h, buf, len(blob)))

    # ------------------------------------------------------------ moving frame
    def shift(self, planes: int, mu_fill):
        """Moving frame: drop `planes` cells at the start of the last axis, fill
        the far end with pure liquid at chemical potentials mu_fill (K-1
        values), advance the lab origin (ms_shift)."""
        mf = np.ascontiguousarray(np.atleast_1d(np.asarray(mu_fill, dtype=np.float64)))
        self._c(lib().ms_shift(self.h, int(planes), mf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def front(self) -> int:
        """Highest index along the last axis with a cell that is not pure liquid (-1 if none)."""
        v = ctypes.c_int()
        self._c(lib().ms_front(self.h, ctypes.byref(v)))
        return v.value

    def step_moving_frame(self, n: int, keep: int, mu_fill, check_every: int = 100):
        """n steps in a frame that follows the growth front: every check_every
        steps, when the front has passed index `keep`, shift it back to `keep`."""
        done = 0
        while done < n:
            k = min(check_every, n - done)
            self.step(k)
            done += k
            f = self.front()
            if f > keep:
                self.shift(f - keep, mu_fill)

    # ----------------------------------------------------------- launch shape
    def tiles(self):
        """Compiled launch variants: (tx, ty, split) per tile index."""
        n = lib().ms_tile_count(self.h)
        out = []
        for i in range(n):
            tx, ty = ctypes.c_int(), ctypes.c_int()
            lib().ms_tile_shape(self.h, i, ctypes.byref(tx), ctypes.byref(ty))
            out.append((tx.value, ty.value, int(lib().ms_tile_split(self.h, i))))
        return out

    def launch(self):
        """Current launch: (tile index, z-chunk)."""
        t, z = ctypes.c_int(), ctypes.c_int()
        self._c(lib().ms_get_launch(self.h, ctypes.byref(t), ctypes.byref(z)))
        return t.value, z.value

    def set_launch(self, tile: int, zchunk: int = 0):
        self._c(lib().ms_set_launch(self.h, int(tile), int(zchunk)))

    def tune(self, cache_path: str = None, steps_per_trial: int = 20):
        best = ctypes.c_double()
        self._c(lib().ms_tune(self.h, cache_path.encode() if cache_path else None,
                              int(steps_per_trial), ctypes.byref(best)))
        return best.value


def peak_fp32(paired: bool = False, stream=None) -> float:
    """Measured FP32 FMA throughput of the current device in TFLOP/s
    (ms_peak_fp32: scalar or paired f32x2 fused multiply-adds)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    out = ctypes.c_double(0.0)
    _check(lib().ms_peak_fp32(ctypes.c_void_p(st.cuda_stream), int(bool(paired)), ctypes.byref(out)))
    return out.value
