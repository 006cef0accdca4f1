"""GPU test of ms_diag_noalloc, the allocation-free diagnostics entry point.

Callers that cannot allocate device memory while they run (a fixed memory
budget, a stream being captured into a CUDA graph, a latency-bound loop) use
ms_diag_noalloc on fields they hold; it must agree with ms_diag, which works
on a library context.  Two calls in a row check that the shared scratch array
left over from one call does not leak into the next.  This file is collected
after the rest of the GPU suite (only the input-deck driver's test follows
it), so that a run stopping at its first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,rtol", [("f64", 1e-12), ("f32", 1e-9)])
def test_noalloc_diagnostics_match_context_diagnostics(dtype, rtol):
    import torch
    from paper_2404_01035_gb300 import Simulation, lib
    from paper_2404_01035_gb300._binding import _check
    from paper_2404_01035_gb300.simulation import make_grid, make_params

    p = W.small_multiphase(n=20, dim=3, N=3, NM=2, nx=45, ny=22, nz=19, rotate=True)
    K = p.n_components
    sim = Simulation(p, dtype=dtype)
    sim.set_fields(p.phi0, p.mu0)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    out = torch.full((K + 4,), float("nan"), dtype=torch.float64, device="cuda")
    keep = []
    params = make_params(p, dtype, keep)
    grid = make_grid(p)
    stream = torch.cuda.current_stream()
    for call in range(2):
        sim.step(25 + 10 * call)
        ref = sim.diag()
        phi, mu = sim.get_fields()
        dphi = torch.tensor(phi, dtype=tdt, device="cuda")
        dmu = torch.tensor(mu, dtype=tdt, device="cuda")
        torch.cuda.synchronize()
        _check(lib().ms_diag_noalloc(ctypes.byref(grid), p.n_phases, K, ctypes.byref(params),
                                     ctypes.c_double(ref["t"]), ctypes.c_void_p(dphi.data_ptr()),
                                     ctypes.c_void_p(dmu.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                     ctypes.c_void_p(stream.cuda_stream)))
        stream.synchronize()
        got = out.cpu().numpy()
        NM = K - 1
        np.testing.assert_allclose(got[:NM], ref["mass"], rtol=rtol)
        assert got[NM] == pytest.approx(ref["sum_err"], rel=1e-12, abs=1e-15)
        assert got[NM + 1] == ref["phi_min"] and got[NM + 2] == ref["phi_max"]
        assert got[NM + 3] == ref["nonfinite"] == 0
        assert got[NM + 4] == pytest.approx(ref["mu_diffusion_number"], rel=1e-12)
    sim.close()


def test_noalloc_rejects_grids_beyond_its_limit():
    import torch
    from paper_2404_01035_gb300 import lib
    from paper_2404_01035_gb300.simulation import make_grid, make_params

    p = W.eutectic_3d(n=8)
    big = p.copy(nx=1024, ny=1024, nz=512)   # 536,870,912 cells > 268,435,456
    keep = []
    params = make_params(big, "f32", keep)
    grid = make_grid(big)
    dummy = torch.zeros(16, device="cuda")
    rc = lib().ms_diag_noalloc(ctypes.byref(grid), big.n_phases, big.n_components,
                               ctypes.byref(params), ctypes.c_double(0.0),
                               ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()),
                               ctypes.c_void_p(dummy.data_ptr()), None)
    assert rc == 7
    assert b"exceeds the allocation-free diagnostics limit" in lib().ms_last_error(None)
