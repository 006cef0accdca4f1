"""Pins of the oracle's phase-field step against the free-energy functional it descends.

At a uniform chemical potential mu and temperature T, the phase-field
equation of Sec. 2 is the Allen-Cahn gradient flow of the grand-potential
functional

    F[phi] = sum over cells dx^dim [ eps * sum_{a<b} gamma_ab |q_ab|^2 + w(phi) / eps
                                     + sum_b psi_b(mu, T) h_b(phi) ],
    q_ab   = phi_a grad(phi_b) - phi_b grad(phi_a),

relaxed with mobility 1/(tau eps) and projected onto sum_a phi_a = 1.  For
the well potential the projection is onto the hyperplane: it subtracts the
mean over the phases.  For the obstacle potential it is onto the simplex.
That projection is the same as the hyperplane one wherever every phase stays
positive, which holds at every cell of the smooth states used here (each
phase exceeds 1e-3 and one step of dt = 1e-3 moves it by far less).  One
explicit Euler step therefore moves every cell by

    (phi^{n+1} - phi^n) / dt = -1/(tau eps) * Proj[ dF/dphi_a / dx^dim ].

Here dF/dphi is taken by central differences of F itself.  The gradient
energy is evaluated with spectral derivatives of the periodic field.  The
multi-well or obstacle energy w comes from the oracle's pointwise potential, and only its value
is used, never its derivative.  The same holds for the driving term: h comes
from the oracle's interpolation and psi from its thermodynamics, values only.
Curvature-driven motion (grain growth) drops that term.  The oracle's step assembles the same
derivative from face fluxes and centre terms.  The two therefore agree only
up to the flux scheme's second-order truncation error.  A dropped or
sign-flipped term breaks the agreement by O(1): the centre term, the sign of
q, a pair index, or eps placed on the wrong term.  The check needs three or
more phases: with two phases the centre terms of the two phases are equal and
cancel in the projection.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

L = 32.0


def _state(dim, n, N):
    """A smooth periodic N-phase field on [0, L)^dim with every pair in contact,
    sampled at x = i dx (so that cell i of a grid is cell 2i of the grid twice as fine)."""
    x = np.arange(n) * (L / n)
    g = np.meshgrid(*([x] * dim), indexing="ij")      # g[0] is the slowest axis
    k = 2 * math.pi / L
    f = []
    for a in range(N):
        s = 0.0
        for d in range(dim):
            s = s + (1.2 - 0.2 * a) * math.cos(0.7 * a + 1.3 * d) * \
                np.cos(k * (1 + (a + d) % 2) * g[d] + 0.4 * a + d)
        f.append(s)
    f = np.stack(f)
    e = np.exp(f - f.max(axis=0))
    phi = e / e.sum(axis=0)
    return phi if dim == 3 else phi[:, None]


MU = 0.37          # the uniform chemical potential of the driven cases
T_UNIFORM = 0.15   # and their uniform temperature


def _problem(dim, n, N, g3=0.0, drive=False, pot="well"):
    p = W.small_multiphase(n=n, dim=dim, N=N, NM=1, aniso=False, potential=pot,
                           bc=[W.BC_PERIODIC] * 3, gamma3=g3)
    p.dx = L / n
    p.tau = 1.3
    p.eps = 4.0
    p.dt = 1e-3
    if drive:
        # no temperature gradient, distinct phase free energies: psi_b(mu, T) differ
        p.G, p.V, p.T0 = 0.0, 0.0, T_UNIFORM
        p.f0 = np.array([0.05 * (b % 3) - 0.04 * b for b in range(N)])
    else:
        p.grain_growth = 1
    return p


class _Functional:
    """F[phi] on the periodic grid: spectral gradients, pointwise well energy and,
    when driven, the pointwise term sum_b psi_b h_b(phi)."""

    def __init__(self, p, dim, n, drive=False):
        self.p, self.dim, self.n = p, dim, n
        self.psi = None
        if drive:
            self.psi = np.array([oracle.thermo(p, b, np.array([MU]), T_UNIFORM)[1]
                                 for b in range(p.n_phases)])
        self.axes = tuple(range(3 - dim, 3))          # the grid axes of one [nz][ny][nx] field
        self.k = 2 * math.pi * np.fft.fftfreq(n, d=L / n)
        self.vol = (L / n) ** dim

    def _grad(self, f):
        F = np.fft.fftn(f, axes=self.axes)
        out = []
        for ax in self.axes:
            sh = [1, 1, 1]
            sh[ax] = self.n
            out.append(np.real(np.fft.ifftn(1j * self.k.reshape(sh) * F, axes=self.axes)))
        return out

    def gradient_energy(self, phi):
        p, N = self.p, phi.shape[0]
        g = [self._grad(phi[a]) for a in range(N)]
        E = 0.0
        for a in range(N):
            for b in range(a + 1, N):
                for d in range(self.dim):
                    q = phi[a] * g[b][d] - phi[b] * g[a][d]
                    E += p.gamma[a, b] * float((q * q).sum())
        return E * self.vol

    def derivative(self, phi, a, cell, h=1e-5):
        """dF/dphi_a at one cell, divided by the cell volume (central differences)."""
        p = self.p
        pp, pm = phi.copy(), phi.copy()
        pp[(a,) + cell] += h
        pm[(a,) + cell] -= h
        dEg = (self.gradient_energy(pp) - self.gradient_energy(pm)) / (2 * h * self.vol)
        wp, _ = oracle.potential(p, pp[(slice(None),) + cell])
        wm, _ = oracle.potential(p, pm[(slice(None),) + cell])
        dw = (wp - wm) / (2 * h)
        dpsi = 0.0
        if self.psi is not None:
            hp, _ = oracle.interp(pp[(slice(None),) + cell])
            hm, _ = oracle.interp(pm[(slice(None),) + cell])
            dpsi = float(self.psi @ (hp - hm)) / (2 * h)
        return p.eps * dEg + dw / p.eps + dpsi


def _cells(dim, n, count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        z, y, x = (int(v) for v in rng.integers(0, n, 3))
        out.append((z if dim == 3 else 0, y, x))
    return out


def _step_error(dim, n, N, cells=6, refine=1, g3=0.0, drive=False, pot="well"):
    """max over sampled cells and phases of |oracle step rate - projected gradient flow|,
    and the largest |rate| there (the scale).  The cells are drawn on the grid of n
    cells; `refine` runs the same points on a grid `refine` times as fine."""
    m = n * refine
    p = _problem(dim, m, N, g3, drive, pot)
    phi = _state(dim, m, N)
    assert phi.min() > 1e-3      # interior of the simplex: both projections agree
    mu = np.full((1,) + phi.shape[1:], MU)
    phi1, _ = oracle.run(p, phi, mu, 1)
    rate = (phi1 - phi) / p.dt
    F = _Functional(p, dim, m, drive)
    err = scale = 0.0
    for c0 in _cells(dim, n, cells, seed=n + 10 * N):
        c = (c0[0] * refine if dim == 3 else 0, c0[1] * refine, c0[2] * refine)
        dF = np.array([F.derivative(phi, a, c) for a in range(N)])
        expect = -(dF - dF.mean()) / (p.tau * p.eps)
        got = rate[(slice(None),) + c]
        err = max(err, float(np.abs(got - expect).max()))
        scale = max(scale, float(np.abs(expect).max()))
    return err, scale


@pytest.mark.parametrize("N,g3,drive,pot", [(3, 0.0, False, "well"), (4, 0.0, False, "well"),
                                            (3, 6.0, False, "well"), (3, 0.0, True, "well"),
                                            (4, 6.0, True, "well"), (3, 0.0, False, "obstacle"),
                                            (4, 6.0, True, "obstacle")])
def test_step_is_the_projected_gradient_flow_of_the_functional_2d(N, g3, drive, pot):
    """2-D, three and four phases, the multi-well or the obstacle potential, with
    and without the triple-junction term Gamma_abc phi_a phi_b phi_c,
    curvature-driven or with the chemical driving force: the step rate converges
    to -Proj dF/dphi / (tau eps) at second order as dx halves on a fixed domain
    (error ratio about 4)."""
    e1, s1 = _step_error(2, 32, N, g3=g3, drive=drive, pot=pot)
    e2, s2 = _step_error(2, 32, N, refine=2, g3=g3, drive=drive, pot=pot)
    assert e1 < 0.08 * s1, (e1, s1)
    assert 3.5 < e1 / e2 < 4.6, (e1, e2)


def test_step_is_the_projected_gradient_flow_of_the_functional_3d():
    """3-D, three phases, one resolution: the step rate and the functional's derivative
    agree to the flux scheme's truncation error."""
    e, s = _step_error(3, 24, 3, cells=4)
    assert e < 0.06 * s, (e, s)


def test_the_centre_term_carries_the_multiphase_signal():
    """The state is one on which the pins above can see the centre term.  After the
    projection, the oracle's centre term is more than 20% of the whole gradient part
    there.  A dropped or sign-flipped centre term would therefore miss the 8%
    tolerance by a wide margin."""
    n, N = 32, 3
    p = _problem(2, n, N)
    phi = _state(2, n, N)
    mu = np.zeros((1,) + phi.shape[1:])
    divJ, Gc, _, _ = oracle.rate_parts(p, phi, mu)
    Gp = Gc - Gc.mean(axis=0, keepdims=True)          # what survives the projection
    gp = (divJ - Gc) - (divJ - Gc).mean(axis=0, keepdims=True)
    assert np.abs(Gp).max() > 0.2 * np.abs(gp).max()


# ----------------------------------------------------------- anisotropic pairs
def _aniso_energy(p, phi, n, dim):
    """F[phi] with the rotated four-fold anisotropy of Eq. aniso_eqn,
    a_c(R q) = 1 - delta (3 - 4 sum_i (R q)_i^4 / |q|^4), spectral gradients,
    plus the well energy 9 gamma phi_a^2 phi_b^2 written out."""
    N = phi.shape[0]
    k = 2 * math.pi * np.fft.fftfreq(n, d=L / n)
    axes = (2, 1, 0)[:dim]                      # x, y (, z) of a [z][y][x] field
    spatial = tuple(range(3 - dim, 3))

    def grad(f):
        F = np.fft.fftn(f, axes=spatial)
        out = []
        for ax in axes:
            sh = [1, 1, 1]
            sh[ax] = n
            out.append(np.real(np.fft.ifftn(1j * k.reshape(sh) * F, axes=spatial)))
        return out

    g = [grad(phi[a]) for a in range(N)]
    E = 0.0
    w = 0.0
    for a in range(N):
        for b in range(a + 1, N):
            q = [phi[a] * g[b][d] - phi[b] * g[a][d] for d in range(dim)]
            Q = sum(c * c for c in q)
            R = p.rot[a, b]
            qr = [sum(R[i, j] * q[j] for j in range(dim)) for i in range(dim)]
            ac = 1.0 - p.delta[a, b] * (3.0 - 4.0 * sum(c ** 4 for c in qr) / np.maximum(Q * Q, 1e-300))
            E += p.gamma[a, b] * float((ac * ac * Q).sum())
            w += 9.0 * p.gamma[a, b] * float((phi[a] ** 2 * phi[b] ** 2).sum())
    return (p.eps * E + w / p.eps) * (L / n) ** dim


def _dissipation_error(n, N, dim=2):
    p = W.small_multiphase(n=n, dim=dim, N=N, NM=1, aniso=True, rotate=True, potential="well",
                           bc=[W.BC_PERIODIC] * 3)
    p.dx, p.grain_growth, p.tau, p.eps, p.dt = L / n, 1, 1.3, 4.0, 1e-4
    phi = _state(dim, n, N)
    phi1, _ = oracle.run(p, phi, np.zeros((1,) + phi.shape[1:]), 1)
    r = (phi1 - phi) / p.dt
    h = 1e-3
    dF = (_aniso_energy(p, phi + h * r, n, dim) - _aniso_energy(p, phi - h * r, n, dim)) / (2 * h)
    expect = -p.tau * p.eps * float((r * r).sum()) * (L / n) ** dim
    return abs(dF - expect) / abs(expect)


@pytest.mark.parametrize("N,dim,sizes,bound", [(3, 2, (32, 64, 128), 5e-3), (4, 2, (32, 64, 128), 5e-3),
                                               (3, 3, (16, 32, 64), 1.5e-2)])
def test_anisotropic_step_dissipates_the_functional_at_its_rate(N, dim, sizes, bound):
    """Rotated anisotropic pairs (2-D in-plane and 3-D rotations), three and four
    phases, curvature-driven.  For a projected gradient flow
    r = -Proj dF/dphi / (tau eps), the functional changes along r at the rate
    dF[r] = -tau eps |r|^2 (the projection is orthogonal).  dF[r] is the
    directional derivative of F itself, taken by central differences of the
    spectral F along the oracle's step rate.  The anisotropic energy has kinks
    where q_ab = 0.  They spoil a cell-by-cell comparison, but over the whole
    grid the identity converges at second order as dx halves."""
    e = [_dissipation_error(n, N, dim) for n in sizes]
    assert e[1] < bound, e
    assert 3.2 < e[0] / e[1] < 4.6 and 3.2 < e[1] / e[2] < 4.6, e
