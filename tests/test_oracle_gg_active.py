"""Pins of the locally-active projection option of the oracle (the Lagrange
multiplier over the phases present at the cell or its face neighbours; every
other phase stays 0), used by the sparse grain-growth path, and of the third
("ghost") phases that the projection over all phases produces at two-grain
boundaries of the multi-obstacle potential.

Ghost phases, derived for the relaxed planar profile phi_a = (1 + s)/2,
s = sin(4x / (pi eps)), of two isotropic grains with equal gamma: both grains
then move with the common rate R = -(24 gamma / (pi^2 eps^2)) (1 - s^2) / tau
(per unit dt), while a third grain c absent from the neighbourhood has
r_c = -(16 gamma / pi^2 + Gamma phi_a phi_b) / (eps^2 tau).  The projection
gives c a positive value where r_c > R, i.e. for Gamma = 0 where s^2 < 1/3
(mid-interface), and nowhere once Gamma >= 96 gamma / pi^2.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def _planar(n_phases, eps=4.0, nx=64, ny=4, gamma3=0.0):
    """Two grains (phases 0 and 1) meeting in a relaxed planar boundary; the
    other phases absent."""
    p = W.grain_growth(n=nx, dim=2, grains=n_phases, ny=ny)
    x = np.arange(nx) + 0.5
    lim = math.pi ** 2 / 8.0
    u = np.clip((x - nx / 4.0) / eps, -lim, lim)
    w = np.clip((3 * nx / 4.0 - x) / eps, -lim, lim)
    s1 = 0.5 * (1 + np.sin(4 * u / math.pi))
    s2 = 0.5 * (1 + np.sin(4 * w / math.pi))
    a = np.minimum(s1, s2)          # grain 0 in the middle, grain 1 outside
    phi = np.zeros((n_phases, 1, ny, nx))
    phi[0] = np.broadcast_to(a, (1, ny, nx))
    phi[1] = 1.0 - phi[0]
    G = None
    if gamma3:
        G = np.full((n_phases,) * 3, gamma3)
        for k in range(n_phases):
            G[k, k, :] = 0.0
            G[k, :, k] = 0.0
            G[:, k, k] = 0.0
    return p.copy(phi0=phi, gamma3=G)


def test_two_grains_are_the_same_under_both_projections():
    p = W.grain_growth(n=48, dim=2, grains=2)
    a = oracle.run(p, p.phi0, p.mu0, 40)
    b = oracle.run(p, p.phi0, p.mu0, 40, active_set=1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_ghost_phase_at_a_two_grain_boundary_and_its_suppression():
    # projection over all phases, Gamma = 0: the third grain appears in the
    # middle of the boundary (s^2 < 1/3) and nowhere near the edges
    p = _planar(3)
    phi, _ = oracle.run(p, p.phi0, p.mu0, 1)
    s = 2 * p.phi0[0, 0, 0] - 1
    ghost = phi[2, 0, 0] > 0
    assert ghost[np.abs(s) < 0.45].all() and not ghost[np.abs(s) > 0.7].any()
    # Gamma above 96 gamma / pi^2 suppresses it everywhere
    q = _planar(3, gamma3=2.0 * 96.0 / math.pi ** 2)
    phi, _ = oracle.run(q, q.phi0, q.mu0, 1)
    assert (phi[2] == 0).all()
    # and the locally-active projection never lets an absent grain in
    phi, _ = oracle.run(p, p.phi0, p.mu0, 1, active_set=1)
    assert (phi[2] == 0).all()


def test_locally_active_phases_stay_local_and_the_simplex_holds():
    p = W.grain_growth(n=64, dim=2, grains=12)
    N = p.n_phases
    G = np.full((N, N, N), 15.0)
    for k in range(N):
        G[k, k, :] = 0.0
        G[k, :, k] = 0.0
        G[:, k, k] = 0.0
    p = p.copy(gamma3=G)
    phi = p.phi0
    for _ in range(6):
        nxt, _ = oracle.run(p, phi, p.mu0, 1, active_set=1)
        # a grain can only appear where it is non-zero at the cell or a face neighbour
        present = phi > 0
        near = present.copy()
        for ax in (2, 3):
            near |= np.roll(present, 1, axis=ax) | np.roll(present, -1, axis=ax)
        assert not (nxt > 0)[~near].any()
        assert np.abs(nxt.sum(axis=0) - 1).max() < 1e-14 and nxt.min() >= 0.0
        phi = nxt
