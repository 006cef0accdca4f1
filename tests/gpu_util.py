"""Helpers for the GPU parity tests (imported by test modules only)."""
import numpy as np

import oracle

BC_PERIODIC = 3


def _axis_index(c, n, bc, r):
    idx = np.arange(c - r, c + r + 1)
    if bc == BC_PERIODIC:
        return idx % n
    return np.clip(idx, 0, n - 1)   # mirror ghost = adjacent interior cell


def windowed_one_step(prob, phi, mu, cells, t0=0.0, r=2):
    """Oracle outputs of ONE step at the given (z, y, x) cells of a full grid.

    One step of a cell depends on its 19-point (3-D) / 9-point (2-D)
    neighbourhood only, so each sampled cell is advanced on a (2r+1)^d window
    cut out of the full input with the grid's boundary mapping; the window's
    own periodic wrap never reaches the centre's stencil.  The temperature is
    kept right at the centre by shifting z0 with the window origin.
    """
    phi = np.asarray(phi, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    dim = prob.dim
    nz, ny, nx = phi.shape[1:]
    out_phi = np.zeros((len(cells), phi.shape[0]))
    out_mu = np.zeros((len(cells), mu.shape[0]))
    w = 2 * r + 1
    for n, (z, y, x) in enumerate(cells):
        ix = _axis_index(x, nx, prob.bc[0], r)
        iy = _axis_index(y, ny, prob.bc[1], r)
        if dim == 3:
            iz = _axis_index(z, nz, prob.bc[2], r)
        else:
            iz = np.array([0])
        wp = phi[:, iz][:, :, iy][:, :, :, ix]
        wm = mu[:, iz][:, :, iy][:, :, :, ix]
        last = z if dim == 3 else y
        wprob = prob.copy(nx=w, ny=w, nz=(w if dim == 3 else 1), bc=[BC_PERIODIC] * 3,
                          z0=prob.z0 - (last - r) * prob.dx)
        op, om = oracle.run(wprob, wp, wm, 1, t0=t0)
        cz = r if dim == 3 else 0
        out_phi[n] = op[:, cz, r, r]
        out_mu[n] = om[:, cz, r, r]
    return out_phi, out_mu


def pick_cells(phi, rng, n_random=48, n_interface=96):
    """Random cells, cells inside interfaces (0 < phi < 1) and the grid corners."""
    nz, ny, nx = phi.shape[1:]
    cells = set()
    for _ in range(n_random):
        cells.add((int(rng.integers(nz)), int(rng.integers(ny)), int(rng.integers(nx))))
    inter = np.argwhere(((phi > 0) & (phi < 1)).any(axis=0))
    if len(inter):
        sel = rng.choice(len(inter), size=min(n_interface, len(inter)), replace=False)
        for k in sel:
            cells.add(tuple(int(v) for v in inter[k]))
    for z in (0, nz - 1):
        for y in (0, ny - 1):
            for x in (0, nx - 1):
                cells.add((z, y, x))
    return sorted(cells)
