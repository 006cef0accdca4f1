"""Host-side helpers of bench.py (no GPU): the pure-stencil classification
the ALU roof uses, against a per-cell brute force."""
import numpy as np
import pytest

import bench


@pytest.mark.parametrize("bc", [[3, 3, 3], [3, 1, 1], [1, 3, 1]])
def test_pure_stencil_mask_matches_brute_force(bc):
    rng = np.random.default_rng(3)
    nz, ny, nx = 5, 6, 7
    lab = rng.integers(0, 3, size=(nz, ny, nx))
    lab[1:4, 1:5, 1:6] = 2                      # a pure block with interior cells
    phi = np.stack([(lab == a).astype(float) for a in range(3)])
    phi[0, 0, 0, 0], phi[2, 0, 0, 0] = 0.5, 0.5  # one mixed cell
    got = bench.pure_stencil_mask(phi, bc)

    def m(i, n, b):
        if 0 <= i < n:
            return i
        return i % n if b == 3 else min(max(i, 0), n - 1)

    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                vals = set()
                for dz in (-1, 0, 1):
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            if abs(dz) + abs(dy) + abs(dx) == 3:
                                continue
                            c = (m(z + dz, nz, bc[2]), m(y + dy, ny, bc[1]), m(x + dx, nx, bc[0]))
                            vals.add(tuple(phi[:, c[0], c[1], c[2]]))
                want = len(vals) == 1 and max(next(iter(vals))) == 1.0
                assert got[z, y, x] == want, (z, y, x)
    assert got.any() and not got.all()


def test_kernel_digest_follows_the_step_kernels_sources(tmp_path, monkeypatch):
    # the digest that ties a committed ncu traffic figure to a kernel version
    # covers the step kernels' translation unit and the headers it includes:
    # editing one of those changes it, editing another unit does not
    import os
    import shutil
    src = os.path.join(bench.ROOT, "paper_2404_01035_gb300", "csrc")
    dst = tmp_path / "paper_2404_01035_gb300" / "csrc"
    shutil.copytree(src, dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d0 = bench.kernel_digest()
    with open(dst / "ms_adjoint.cu", "a") as fh:
        fh.write("\n// unrelated edit\n")
    assert bench.kernel_digest() == d0
    with open(dst / "ms_split.cuh", "a") as fh:
        fh.write("\n// step kernel edit\n")
    d1 = bench.kernel_digest()
    assert d1 != d0
    with open(dst / "ms_device.cuh", "a") as fh:   # reached through the includes
        fh.write("\n// header edit\n")
    assert bench.kernel_digest() != d1
