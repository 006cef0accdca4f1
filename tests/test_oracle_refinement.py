"""Grid-refinement pin of the oracle's full multiphase trajectory: a smooth
2-D state of three anisotropic phases (rotated pairs, two solutes, well
potential, a pulled temperature gradient) advanced to a fixed physical time
on grids of spacing dx, dx/2 and dx/4 with dt proportional to dx^2 (explicit
Euler is first order in dt, so the whole scheme is second order in dx).

The change over the run, u(T) - u(0), is compared between successive
resolutions after restriction to the coarse grid by cell averages (the
initial sampling then cancels); the differences must shrink by about 4 per
halving: every term
of the discrete step has to scale correctly with dx (gradients 1/dx, the
divergences and Laplacians 1/dx^2, positions (k + 1/2) dx), which no test at
dx = 1 can see."""
import math

import numpy as np

import oracle
import workloads as W


def _smooth_state(p, n, L):
    """phi: a softmax of smooth periodic functions (every phase in (0, 1),
    interfaces several coarse cells wide); mu: a smooth perturbation."""
    dx = L / n
    x = (np.arange(n) + 0.5) * dx
    X, Y = np.meshgrid(x, x, indexing="xy")
    k = 2 * math.pi / L
    f = np.stack([1.6 * np.cos(k * X + 0.3) + 0.8 * np.sin(k * Y),
                  1.4 * np.sin(k * (X + Y) + 1.1),
                  1.2 * np.cos(k * Y - 0.7) - 0.6 * np.cos(2 * k * X)])
    e = np.exp(f - f.max(axis=0))
    phi = (e / e.sum(axis=0))[:, None]
    mu = np.stack([0.05 * np.cos(k * X + 0.5 * i) for i in range(p.n_components - 1)])[:, None]
    mu = mu + p.mu0.mean(axis=(1, 2, 3))[:, None, None, None]
    return phi, mu


def _restrict(a, f):
    F, Z, ny, nx = a.shape
    return a.reshape(F, Z, ny // f, f, nx // f, f).mean(axis=(3, 5))


def test_second_order_convergence_under_refinement():
    L, n0 = 24.0, 24
    base = W.small_multiphase(n=n0, dim=2, N=3, NM=2, potential="well", rotate=True,
                              bc=[W.BC_PERIODIC, W.BC_PERIODIC, W.BC_PERIODIC])
    dt0 = 0.25 * base.dt
    steps0 = 20
    change = []   # phi(T) - phi(0), mu(T) - mu(0), restricted to the coarse grid
    for f in (1, 2, 4):
        n = n0 * f
        p = base.copy(nx=n, ny=n, dx=L / n, dt=dt0 / f ** 2, eps=4.0)
        phi0, mu0 = _smooth_state(p, n, L)
        phi, mu = oracle.run(p, phi0, mu0, steps0 * f ** 2)
        change.append((_restrict(phi - phi0, f), _restrict(mu - mu0, f)))
    for q in (0, 1):   # phi, mu
        e1 = np.abs(change[0][q] - change[1][q]).max()
        e2 = np.abs(change[1][q] - change[2][q]).max()
        assert e1 < 0.05 * np.abs(change[2][q]).max()   # resolved: differences well below the change
        assert 3.5 < e1 / e2 < 4.6, (q, e1, e2)


def _front_state(p, nx, ny, Lx, Ly):
    """A solid-liquid front across x, modulated along y (so the normals have
    both components and are defined wherever the rate is not negligible)."""
    dx = Lx / nx
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dx
    X, Y = np.meshgrid(x, y, indexing="xy")
    xf = 0.5 * Lx + 1.5 * np.cos(2 * math.pi * Y / Ly)
    s = 0.5 * (1 + np.tanh(1.5 * (xf - X) / p.eps))
    phi = np.stack([s, 1 - s])[:, None]
    mu = (p.mu0.mean(axis=(1, 2, 3))[:, None, None] + 0.02 * np.cos(2 * math.pi * Y / Ly))[:, None]
    return phi, mu


def test_anti_trapping_current_converges_at_second_order():
    # the current's face normals, face rates and divergence scale with dx as
    # well: a moving front with the current on, no-flux across it (the liquid
    # fraction is monotone along x, so its normal never flips)
    Lx, Ly, n0 = 24.0, 12.0, 12
    base = W.binary_problem("atref", 24, delta=0.02, Delta=0.2, R=5.0, potential="well", ny=12,
                            bc=[W.BC_NOFLUX, W.BC_PERIODIC, W.BC_PERIODIC])
    dt0 = 0.25 * base.dt
    change = []
    for f in (1, 2, 4):
        nx, ny = 2 * n0 * f, n0 * f
        p = base.copy(nx=nx, ny=ny, dx=Lx / nx, dt=dt0 / f ** 2, eps=3.0, anti_trapping=1)
        phi0, mu0 = _front_state(p, nx, ny, Lx, Ly)
        phi, mu = oracle.run(p, phi0, mu0, 40 * f ** 2)
        change.append((_restrict(phi - phi0, f), _restrict(mu - mu0, f)))
    for q in (0, 1):
        e1 = np.abs(change[0][q] - change[1][q]).max()
        e2 = np.abs(change[1][q] - change[2][q]).max()
        assert e1 < 0.1 * np.abs(change[2][q]).max()
        assert 3.5 < e1 / e2 < 5.0, (q, e1, e2)
