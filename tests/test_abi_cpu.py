"""C-ABI checks that need no GPU: the library builds, loads, exports every
function include/microsim_gb.h declares, and rejects bad inputs with the
documented status codes before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W
from paper_2404_01035_gb300 import _binding as B
from paper_2404_01035_gb300.simulation import make_grid, make_params

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ms_[a-z0-9_]+)\s*\(", src))
    return names - {"ms_status"}


def test_library_loads_and_exports_every_declared_symbol():
    L = B.lib()
    decl = declared_functions()
    assert len(decl) >= 19
    missing = [n for n in sorted(decl) if not hasattr(L, n)]
    assert not missing, missing
    assert set(B.EXPORTS) <= decl


def test_binding_lists_every_declared_function():
    assert declared_functions() <= set(B.EXPORTS) | {"MS_DIAG_LEN"}


def _create(prob, dtype="f32", **override):
    L = B.lib()
    keep = []
    params = make_params(prob, dtype, keep, **override)
    grid = make_grid(prob)
    h = ctypes.c_void_p()
    rc = L.ms_create(ctypes.byref(grid), prob.n_phases, prob.n_components, ctypes.byref(params),
                     None, None, ctypes.byref(h))
    return rc, h, L.ms_last_error(None).decode()


def test_create_rejects_unstable_dt():
    p = W.dendrite_2d()
    rc, h, msg = _create(p, dt=10.0)
    assert rc == 4 and "stability" in msg and not h.value


def test_create_rejects_bad_dimension_and_sizes():
    p = W.dendrite_2d()
    bad = p.copy(dim=4)
    assert _create(bad)[0] == 1
    assert _create(p.copy(nx=0))[0] == 1
    many = W.small_multiphase(n=4, dim=2, N=9, NM=1)
    assert _create(many)[0] == 1


def test_create_rejects_bad_boundary_and_potential():
    p = W.dendrite_2d()
    assert _create(p.copy(bc=[2, 3, 3]))[0] == 1
    assert _create(p, eps=-1.0)[0] == 1


def test_create_reports_uncompiled_combination():
    # 3-D with 5 phases is not compiled into the library
    p = W.small_multiphase(n=8, dim=3, N=5, NM=1)
    rc, h, msg = _create(p)
    assert rc == 9 and "no compiled step kernel" in msg


def test_null_handles_are_rejected():
    L = B.lib()
    assert L.ms_step(None, 1) == 1
    assert L.ms_sync(None) == 1
    assert L.ms_checkpoint_bytes(None) == 0
    L.ms_destroy(None)


def test_batch_create_rejects_unsupported_combinations():
    L = B.lib()
    p = W.small_multiphase(n=8, dim=3, N=3, NM=2)
    keep = []
    grids = (B.Grid * 1)(make_grid(p))
    params = (B.Params * 1)(make_params(p, "f32", keep))
    h = ctypes.c_void_p()
    rc = L.ms_batch_create(1, grids, p.n_phases, p.n_components, params, None, None, ctypes.byref(h))
    assert rc == 9 and not h.value
    assert L.ms_batch_create(0, grids, 2, 2, params, None, None, ctypes.byref(h)) == 1


def test_params_struct_layout_matches_the_header(tmp_path):
    # the ctypes mirror of ms_params / ms_grid against the C compiler's layout
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    fields = [f for f, _ in B.Params._fields_]
    src = tmp_path / "layout.c"
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "microsim_gb.h"', "int main(void) {",
             '  printf("%zu\\n", sizeof(ms_params));']
    lines += [f'  printf("%zu\\n", offsetof(ms_params, {f}));' for f in fields]
    lines += ['  printf("%zu\\n", sizeof(ms_grid));', "  return 0;", "}"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert out[0] == ctypes.sizeof(B.Params)
    assert out[1:1 + len(fields)] == [getattr(B.Params, f).offset for f in fields]
    assert out[-1] == ctypes.sizeof(B.Grid)


def test_create_rejects_inconsistent_options():
    p = W.dendrite_2d()
    C = np.eye(6) * 100.0
    eig = np.zeros((2, 3, 3))
    # a stiffness without eigenstrains
    assert _create(p, elastic_C=C, eigenstrain=None)[0] == 1
    # the FFT equilibrium needs periodic boundaries; not with grain growth
    assert _create(p.copy(bc=[3, 1, 1]), elastic_C=C, eigenstrain=eig)[0] == 9
    assert _create(p, elastic_C=C, eigenstrain=eig, grain_growth=1)[0] == 9
    # grain growth holds mu, so the anti-trapping current cannot apply
    assert _create(p, anti_trapping=1, grain_growth=1)[0] == 1
    # a slab with halo faces cannot take the anti-trapping current
    q = W.small_multiphase(n=8, dim=3, N=3, NM=2, bc=[3, 3, 16])
    rc, h, msg = _create(q, anti_trapping=1)
    assert rc == 9 and "anti-trapping" in msg


def test_create_refuses_grids_beyond_the_fft_plans():
    # the elasticity's batched FFT plans take the cell count as an int: a
    # 2048 x 1024 x 1024 grid (2^31 cells) is refused before any allocation
    q = W.small_multiphase(n=8, dim=3, N=3, NM=2, bc=[3, 3, 3]).copy(nx=2048, ny=1024, nz=1024)
    rc, h, msg = _create(q, elastic_C=np.eye(6) * 100.0, eigenstrain=np.zeros((3, 3, 3)))
    assert rc == 9 and "too large" in msg and not h.value


@pytest.mark.parametrize("spec", ["step:3", "step:-1,code:6", "step:2,code:0", "step:2,code:42",
                                  "step:2,code:6,extra", "bogus"])
def test_create_rejects_a_malformed_fault_spec(monkeypatch, spec):
    # MS_FAULT is parsed before any device work, so a bad spec fails on CPU
    monkeypatch.setenv("MS_FAULT", spec)
    rc, h, msg = _create(W.dendrite_2d())
    assert rc == 1 and "MS_FAULT" in msg and not h.value


def test_check_params_reports_the_stability_bound():
    """ms_check_params runs ms_create's checks without a device and returns the
    explicit bound: for the 2-D dendrite (gamma = 1, delta = 0, tau = 1, D = 1,
    dx = 1) it is (1 / 4) min(1, 1)."""
    from paper_2404_01035_gb300.simulation import check_params
    p = W.dendrite_2d()
    assert check_params(p, "f64") == pytest.approx(0.25, rel=1e-12)
    with pytest.raises(B.MSError) as ex:
        check_params(p, "f64", dt=10.0)
    assert ex.value.status == 4 and ex.value.dt_bound == pytest.approx(0.25, rel=1e-12)
    q = W.small_multiphase(n=8, dim=2, N=4, NM=1)          # (2-D, N=4, K=2) is not compiled
    with pytest.raises(B.MSError) as ex:
        check_params(q, "f32")
    assert ex.value.status == 9
