"""Pins of the chemical mobility across interfaces (Eq. Mass_conservation:
M = sum_a h_a(phi) D^a chi^a, face value the mean of the two cells, evaluated
with phi^n) in the oracle's mu update (Eq. Mu_explicit_temperature).

The single-phase Fourier and Gaussian pins have h = phi = 1, mass
conservation holds for any M, and the interface pins freeze mu, so none of
them sees how M is interpolated inside a diffuse interface.  Here the two
phases share their thermodynamics (same A, same c_eq, no drive), so
psi^s(mu) = psi^l(mu) for every mu and chi^s = chi^l = chi: the phase update
does not depend on mu, the composition term sum_a c^a (h_a^{n+1} - h_a^n)
vanishes with sum_a h_a = 1, chi(h) = chi, and only the diffusivities differ
(D^s != D^l).  A mu mode cos(2 pi k x / n) on a state whose phi varies along
y only is then an eigenvector of one step: each row y scales it by the exact
factor

    I - 4 dt sin^2(pi k / n) chi^-1 M(y),   M(y) = sum_a h_a(phi^n(y)) D^a chi

(for one solute simply 1 - 4 dt sin^2(pi k / n) sum_a h_a D^a), which the
tests compare with the oracle to round-off.  Mistakes this catches (each
planted in a copy of the oracle): phi in place of h(phi) in M, phi^{n+1} in
place of phi^n in M, D^a chi^a multiplied in the wrong order.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def _h2(phi_s):
    """Two-phase restriction of Eq. (hphi): h_s = phi_s^2 (3 - 2 phi_s)."""
    return phi_s * phi_s * (3.0 - 2.0 * phi_s)


def _twin_phase_problem(nx, ny, D_s, D_l, NM=1, A=None, tau=1.0, potential="obstacle"):
    """Two phases with identical parabolic free energies, different D."""
    p = W.binary_problem("twin", nx, ny=ny, Delta=0.0, R=0.0, potential=potential, tau=tau)
    N = 2
    if A is None:
        A = np.eye(NM)
    p = p.copy(n_components=NM + 1,
               A=np.stack([A, A]),
               ceq=np.tile(np.linspace(0.3, 0.6, NM), (N, 1)),
               slopes=np.zeros((N, NM)),
               f0=np.zeros(N),
               D=np.stack([np.asarray(D_s, float).reshape(NM, NM), np.asarray(D_l, float).reshape(NM, NM)]),
               G=0.0, V=0.0)
    return p


def _ramp_profile(nx, ny, lo=0.04, hi=0.96):
    """phi_s varying along y only: a linear ramp (not the relaxed profile, so
    phi moves during the step) with many distinct interface values."""
    s = np.linspace(lo, hi, ny)
    ps = np.broadcast_to(s[None, :, None], (1, ny, nx)).copy()
    return np.stack([ps, 1.0 - ps])


def test_two_phase_interpolation_matches_closed_form():
    """oracle interp for N = 2 is phi_s^2 (3 - 2 phi_s) (the closed form the
    mobility pins below use)."""
    for s in np.linspace(0.0, 1.0, 11):
        h, _ = oracle.interp(np.array([s, 1.0 - s]))
        assert abs(h[0] - _h2(s)) < 1e-15 and abs(h[1] - _h2(1.0 - s)) < 1e-15


@pytest.mark.parametrize("potential", ["obstacle", "well"])
def test_mode_decay_across_a_moving_interface_one_step(potential):
    """One step: row y scales the x-mode by 1 - 4 dt s^2 sum_a h_a(phi^n(y)) D^a."""
    nx, ny, k = 16, 24, 3
    D_s, D_l = 0.25, 1.0
    p = _twin_phase_problem(nx, ny, D_s, D_l, potential=potential)
    p.dt = 0.1
    phi0 = _ramp_profile(nx, ny)
    x = np.arange(nx) + 0.5
    amp, mubar = 0.02, 0.7
    mode = np.cos(2 * np.pi * k * x / nx)
    mu0 = np.broadcast_to((mubar + amp * mode)[None, None, None, :], (1, 1, ny, nx)).copy()
    phi1, mu1 = oracle.run(p, phi0, mu0, 1)
    # the phase update ignores mu (identical thermodynamics) and moves phi
    assert np.abs(phi1 - phi1[:, :, :, :1]).max() < 1e-15
    moved = np.abs(_h2(phi1[0, 0, :, 0]) - _h2(phi0[0, 0, :, 0]))
    assert moved.max() > 2e-3
    s2 = math.sin(math.pi * k / nx) ** 2
    hs = _h2(phi0[0, 0, :, 0])
    Mrow = hs * D_s + (1.0 - hs) * D_l
    expect = mubar + amp * (1.0 - 4.0 * p.dt * s2 * Mrow)[:, None] * mode[None, :]
    np.testing.assert_allclose(mu1[0, 0], expect, rtol=0, atol=2e-15)


def test_mode_decay_frozen_mixed_state_many_steps():
    """phi frozen (tau huge) in a uniform mixed state phi_s = s: the mode of
    mu decays by (1 - 4 dt sum_d sin^2(pi k_d/n) (h_s D^s + h_l D^l))^n."""
    nx, ny, steps = 16, 12, 30
    D_s, D_l = 0.3, 0.9
    k = (2, 1)
    x = np.arange(nx) + 0.5
    y = np.arange(ny) + 0.5
    arg = 2 * np.pi * (k[0] * x[None, :] / nx + k[1] * y[:, None] / ny)
    amp, mubar = 0.01, 0.5
    mu0 = (mubar + amp * np.cos(arg))[None, None]
    for s in (0.2, 0.35, 0.8):
        p = _twin_phase_problem(nx, ny, D_s, D_l, tau=1e30)
        p.dt = 0.1
        phi0 = np.stack([np.full((1, ny, nx), s), np.full((1, ny, nx), 1.0 - s)])
        phi, mu = oracle.run(p, phi0, mu0, steps)
        assert np.abs(phi - phi0).max() < 1e-15
        hs = _h2(s)
        M = hs * D_s + (1.0 - hs) * D_l
        lam = 1.0 - 4.0 * p.dt * M * (math.sin(math.pi * k[0] / nx) ** 2 + math.sin(math.pi * k[1] / ny) ** 2)
        np.testing.assert_allclose(mu[0, 0] - mubar, amp * lam ** steps * np.cos(arg), rtol=0, atol=1e-15)


def test_matrix_mobility_order_two_solutes():
    """Two solutes: one step maps the mode's amplitude vector a to
    (I - 4 dt s^2 chi^-1 M) a with M = (sum_a h_a D^a) chi, chi = A-hat^-1
    (A-hat_ii = 2 A_ii, A-hat_ij = A_ij), per row, for non-commuting D^a and chi."""
    nx, ny, k = 16, 20, 2
    A = np.array([[1.0, 0.6], [0.0, 1.5]])      # i <= j used: A-hat = [[2, .6], [.6, 3]]
    D_s = np.array([[0.2, 0.05], [-0.03, 0.1]])
    D_l = np.array([[0.9, 0.2], [0.1, 0.6]])
    p = _twin_phase_problem(nx, ny, D_s, D_l, NM=2, A=A)
    p.dt = 0.05
    phi0 = _ramp_profile(nx, ny)
    x = np.arange(nx) + 0.5
    mode = np.cos(2 * np.pi * k * x / nx)
    a0 = np.array([0.013, -0.021])
    mubar = np.array([0.9, 1.2])
    mu0 = np.zeros((2, 1, ny, nx))
    for i in range(2):
        mu0[i, 0] = mubar[i] + a0[i] * mode[None, :]
    phi1, mu1 = oracle.run(p, phi0, mu0, 1)
    assert np.abs(phi1 - phi1[:, :, :, :1]).max() < 1e-15
    Ahat = np.array([[2 * A[0, 0], A[0, 1]], [A[0, 1], 2 * A[1, 1]]])
    chi = np.linalg.inv(Ahat)
    _, _, chi_or = oracle.thermo(p, 0, mubar, 0.0)
    np.testing.assert_allclose(chi_or, chi, rtol=0, atol=1e-15)
    s2 = math.sin(math.pi * k / nx) ** 2
    for y in range(ny):
        hs = _h2(phi0[0, 0, y, 0])
        M = (hs * D_s + (1.0 - hs) * D_l) @ chi
        a1 = (np.eye(2) - 4.0 * p.dt * s2 * np.linalg.solve(chi, M)) @ a0
        for i in range(2):
            np.testing.assert_allclose(mu1[i, 0, y], mubar[i] + a1[i] * mode, rtol=0, atol=3e-15)
