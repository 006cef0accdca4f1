"""Pins of the oracle's anti-trapping current (Eq. jatr and the two forms of
j^{at,alpha} below it), on the CPU.

The face flux is pinned by closed-form values at a planar binary face (the
obstacle coefficient at phi0 = 1/2 and 1/5, the constant well coefficient),
by the direction the paper's physics fixes (a growing solid poorer in solute
than the liquid expels solute into the liquid), by exact inertness where the
current must vanish (phases of equal composition, no liquid present, AT off),
by the conservation its flux form implies (the change it makes to chi dmu sums
to zero over a closed domain), and by the mirror and axis-permutation
symmetry of the whole step.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def _planar(potential, phi_l=0.25, phi_r=0.75, dphi=1e-3, ceq=None):
    # 2-D 4 x 1 binary strip, solid (phase 0) rising along +x; the face between
    # cells 1 and 2 has phi_0 = (phi_l + phi_r) / 2 and no tangential gradient
    p = W.binary_problem("at_planar", 4, dim=2, ny=1, potential=potential, Delta=0.0)
    if ceq is not None:
        p.ceq = np.asarray(ceq, dtype=np.float64)
    s = np.array([0.0, phi_l, phi_r, 1.0])
    phi = np.zeros((2, 1, 1, 4))
    phi[0, 0, 0] = s
    phi[1] = 1.0 - phi[0]
    phin = phi.copy()
    phin[0, 0, 0, 1:3] += dphi
    phin[1] = 1.0 - phin[0]
    mu = np.full((1, 1, 1, 4), 1.7)
    return p, phi, phin, mu


def _delta_c(p, mu_face):
    T = p.T0 + p.G * (0.5 * p.dx - p.z0)   # both cells of the strip sit at y = 0 (the last axis)
    cs = oracle.thermo(p, 0, np.array([mu_face]), T)[0][0]
    cl = oracle.thermo(p, 1, np.array([mu_face]), T)[0][0]
    return cs - cl


@pytest.mark.parametrize("potential,phi_l,phi_r,coef", [
    # obstacle at phi0 = 1/2: pi eps (1/2)(1 - 1/2) / (4 (1/2)) = pi eps / 8
    ("obstacle", 0.25, 0.75, lambda eps: math.pi * eps / 8.0),
    # obstacle at phi0 = 1/5: h = 0.04 * 2.6 = 0.104, sqrt(0.16) = 0.4:
    # pi eps 0.2 * 0.896 / 1.6 = 0.112 pi eps
    ("obstacle", 0.1, 0.3, lambda eps: 0.112 * math.pi * eps),
    # well: eps / (2 sqrt 2), independent of phi
    ("well", 0.1, 0.3, lambda eps: eps / (2.0 * math.sqrt(2.0))),
])
def test_planar_face_flux_closed_form(potential, phi_l, phi_r, coef):
    dphi = 1e-3
    p, phi, phin, mu = _planar(potential, phi_l, phi_r, dphi)
    J = oracle.at_face_flux(p, phi, phin, mu, 1, 0, 0, 0)
    # unit normals +x (solid) and -x (liquid): -n_s . n_l = 1, n_s,x = 1
    expect = coef(p.eps) * _delta_c(p, 1.7) * (dphi / p.dt)
    np.testing.assert_allclose(J[0], expect, rtol=1e-12)
    # the same face seen along y has no normal component
    assert oracle.at_face_flux(p, phi, phin, mu, 1, 0, 0, 1)[0] == 0.0


@pytest.mark.parametrize("rich_solid", [False, True])
def test_growing_solid_expels_or_absorbs_solute(rich_solid):
    # solid on the LEFT (phi_0 falls along +x) and growing: a solid poorer in
    # solute than the liquid pushes solute into the liquid (flux along +x); a
    # richer one draws it in (flux along -x)
    ceq = [[0.95], [0.817]] if rich_solid else [[0.60], [0.817]]
    p, phi, phin, mu = _planar("obstacle", 0.75, 0.25, 1e-3, ceq=ceq)
    phi[0, 0, 0, 0], phi[0, 0, 0, 3] = 1.0, 0.0
    phi[1] = 1.0 - phi[0]
    phin[0, 0, 0] = phi[0, 0, 0] + np.array([0.0, 1e-3, 1e-3, 0.0])
    phin[1] = 1.0 - phin[0]
    J = oracle.at_face_flux(p, phi, phin, mu, 1, 0, 0, 0)[0]
    assert (J < 0) if rich_solid else (J > 0)
    # a melting solid reverses it
    Jm = oracle.at_face_flux(p, phi, 2 * phi - phin, mu, 1, 0, 0, 0)[0]
    assert Jm == pytest.approx(-J, rel=1e-12)


def test_inert_for_equal_compositions_and_without_liquid():
    p = W.small_multiphase(n=12, dim=3, N=3, NM=2, nx=14, ny=11, nz=10)
    # every phase with the same parabolic free energy: c^alpha = c^liq
    q = p.copy()
    q.A = np.repeat(p.A[-1:], 3, axis=0)
    q.ceq = np.repeat(p.ceq[-1:], 3, axis=0)
    q.slopes = np.repeat(p.slopes[-1:], 3, axis=0)
    a = oracle.run(q, q.phi0, q.mu0, 3)
    b = oracle.run(q, q.phi0, q.mu0, 3, anti_trapping=1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # no liquid anywhere in phi^n (solid-solid boundaries only): the liquid has
    # no normal (one step: the liquid may reappear in phi^{n+1})
    phi = p.phi0.copy()
    phi[0] += phi[2]
    phi[2] = 0.0
    a = oracle.run(p, phi, p.mu0, 1)
    b = oracle.run(p, phi, p.mu0, 1, anti_trapping=1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # but with the liquid present it acts
    a = oracle.run(p, p.phi0, p.mu0, 1)
    b = oracle.run(p, p.phi0, p.mu0, 1, anti_trapping=1)
    assert np.array_equal(a[0], b[0]) and np.abs(a[1] - b[1]).max() > 1e-6


@pytest.mark.parametrize("bc", [[3, 3, 3], [3, 1, 1]])
def test_flux_form_conserves_solute(bc):
    # one step with and without j_at from the same state: phi^{n+1} agrees, and
    # chi(h(phi^{n+1})) (mu_at - mu) = -dt div j_at sums to zero over the grid
    p = W.small_multiphase(n=12, dim=3, N=3, NM=2, nx=14, ny=11, nz=10, bc=bc)
    a = oracle.run(p, p.phi0, p.mu0, 1)
    b = oracle.run(p, p.phi0, p.mu0, 1, anti_trapping=1)
    assert np.array_equal(a[0], b[0])
    chis = [oracle.thermo(p, k, p.mu0[:, 0, 0, 0], 0.0)[2] for k in range(3)]
    tot = np.zeros(2)
    mag = 0.0
    N = 3
    flat_phi = a[0].reshape(N, -1)
    dmu = (b[1] - a[1]).reshape(2, -1)
    for c in range(flat_phi.shape[1]):
        h, _ = oracle.interp(flat_phi[:, c])
        chi = sum(h[k] * chis[k] for k in range(N))
        v = chi @ dmu[:, c]
        tot += v
        mag += np.abs(v).sum()
    assert mag > 1e-6
    assert np.abs(tot).max() <= 1e-12 * mag


def test_mirror_and_axis_permutation_symmetry():
    p = W.small_multiphase(n=12, dim=3, N=3, NM=2, nx=12, ny=12, nz=9, bc=[3, 3, 1])
    ref = oracle.run(p, p.phi0, p.mu0, 2, anti_trapping=1)
    # mirror along x
    m = oracle.run(p, p.phi0[..., ::-1].copy(), p.mu0[..., ::-1].copy(), 2, anti_trapping=1)
    assert max(np.abs(m[0][..., ::-1] - ref[0]).max(), np.abs(m[1][..., ::-1] - ref[1]).max()) < 1e-12
    # swap x and y (same boundary codes, cubic anisotropy without rotation)
    sw = lambda f: np.ascontiguousarray(np.swapaxes(f, 2, 3))
    s = oracle.run(p, sw(p.phi0), sw(p.mu0), 2, anti_trapping=1)
    assert max(np.abs(sw(s[0]) - ref[0]).max(), np.abs(sw(s[1]) - ref[1]).max()) < 1e-12
    # and the current matters on this state
    off = oracle.run(p, p.phi0, p.mu0, 2)
    assert np.abs(off[1] - ref[1]).max() > 1e-6


def test_current_moves_solute_from_a_growing_poor_solid_into_the_liquid():
    # one step with and without the current on a planar binary front (solid
    # poorer in solute, growing): across the face the current carries solute
    # out of the solid cell into the liquid cell, so chi dmu (the solute
    # change) falls on the solid side and rises on the liquid side
    p = W.binary_problem("at_sign", 16, dim=2, ny=1, Delta=0.4, bc=[1, 1, 1])
    p.ceq = np.array([[0.60], [0.817]])
    x = (np.arange(16) + 0.5)
    s = W.seed_profile((8.0 - x) / p.eps, "obstacle")        # solid on the left
    phi = np.zeros((2, 1, 1, 16))
    phi[0, 0, 0] = s
    phi[1] = 1.0 - phi[0]
    mu = np.full((1, 1, 1, 16), 1.634)
    a = oracle.run(p, phi, mu, 1)
    b = oracle.run(p, phi, mu, 1, anti_trapping=1)
    grow = a[0][0, 0, 0] - phi[0, 0, 0]
    assert grow[7] > 0 and grow[8] > 0                      # the solid grows
    d = (b[1] - a[1])[0, 0, 0]
    # the two cells of the central face (x = 7.5 | 8.5); chi > 0
    assert d[7] < 0 < d[8]
