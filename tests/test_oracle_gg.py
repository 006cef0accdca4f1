"""Pins of the oracle's grain-growth mode (GRAINGROWTH = 1, read as the phi
equation without the chemical driving force and with mu held), on the CPU.

The rate is pinned by the sharp-interface limit of curvature-driven motion:
for two phases the simplex projection averages the two phases' rates, so the
gradient terms act as gamma eps Lap(phi) and a boundary moves with
v = -gamma kappa / tau; an isolated circular grain therefore loses area at the
constant rate dA/dt = -2 pi gamma / tau whatever its radius (von Neumann -
Mullins).  Planar boundaries (kappa = 0) stay put even where the chemical
driving force of the ordinary model would move them, and mu never changes.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W


@pytest.mark.parametrize("dx", [1.0, 0.5])
def test_circular_grain_loses_area_at_the_curvature_rate(dx):
    """The same physical grain (radius 20, eps 4 on a 64-long box) on grids of
    spacing 1 and 1/2 (dt scaled with dx^2): the same area loss rate."""
    m = int(round(64 / dx))
    p = W.binary_problem("gg_circle", m, dim=2, R=20.0, Delta=0.3)
    ps = W.circular_seed(m, m, 20.0 / dx, p.eps, p.potential, dx=dx)
    p = p.copy(dx=dx, dt=p.dt * dx * dx, phi0=np.stack([ps, 1.0 - ps])[:, None])
    p.grain_growth = 1
    phi, mu = p.phi0, p.mu0
    areas = [phi[0].sum() * dx * dx]
    n = int(round(300 / (dx * dx)))
    for k in range(3):
        phi, mu_k = oracle.run(p, phi, mu, n, t0=k * n * p.dt)
        assert np.array_equal(mu_k, mu)          # mu held
        areas.append(phi[0].sum() * dx * dx)
    rates = np.diff(areas) / (n * p.dt)
    expect = -2.0 * math.pi * p.gamma[0, 1] / p.tau
    np.testing.assert_allclose(rates, expect, rtol=0.03)
    # a constant rate while the radius falls from 20 to ~17.5
    assert abs(rates[0] - rates[-1]) <= 0.01 * abs(expect)


def test_driving_force_is_off():
    # the same disc without grain growth and with a strong undercooling grows
    p = W.binary_problem("gg_drive", 64, dim=2, R=20.0, Delta=0.5)
    grow = oracle.run(p, p.phi0, p.mu0, 200)[0][0].sum() - p.phi0[0].sum()
    p.grain_growth = 1
    gg = oracle.run(p, p.phi0, p.mu0, 200)[0][0].sum() - p.phi0[0].sum()
    assert grow > 0 > gg


def test_planar_boundaries_stay_put():
    # a periodic bicrystal slab with the obstacle equilibrium profile at both
    # boundaries, under a driving force that would move them in the ordinary
    # model: with grain growth the grain's area and boundary positions hold
    p = W.binary_problem("gg_planar", 64, dim=2, ny=4, R=1.0, Delta=0.4, bc=[3, 3, 3])
    x = (np.arange(64) + 0.5)[None, :]
    u = np.minimum(x - 16.0, 48.0 - x) / p.eps
    s = W.seed_profile(u, "obstacle")
    phi = np.zeros((2, 1, 4, 64))
    phi[0, 0] = np.repeat(s, 4, axis=0)
    phi[1] = 1.0 - phi[0]
    mu = np.full((1, 1, 4, 64), 1.634)
    moved = oracle.run(p, phi, mu, 300)[0][0].sum() - phi[0].sum()
    q = p.copy(grain_growth=1)
    out = oracle.run(q, phi, mu, 300)
    assert abs(moved) > 1.0
    assert abs(out[0][0].sum() - phi[0].sum()) < 1e-9
    # the half-value points stay at x = 16 and 48 (profile relaxes in place)
    row = out[0][0, 0, 0]
    for x0 in (16, 48):
        i = x0 - 1                       # cells at x = x0 - 1/2 and x0 + 1/2
        xc = (i + 0.5) + (0.5 - row[i]) / (row[i + 1] - row[i])
        assert abs(xc - x0) < 0.05
