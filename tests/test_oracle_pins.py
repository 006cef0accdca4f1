"""Pins for the FP64 oracle against facts the paper and mathematics fix.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand, a wrong constant) fails it:
closed forms (four-fold a_c, Laplacian identity, equilibrium profiles,
Fourier-mode decay), brute force (projection by support enumeration,
finite differences of energies), invariants (sum phi = 1, exact mass
conservation, equal-mu equilibrium, symmetry) and the sign of curvature-
driven motion (Gibbs-Thomson).
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W


def planar_problem(nx, eps, potential, *, delta=0.0, ny=1, dt=None, ceq_s=0.817,
                   D_l=1.0, f0_s=0.0, steps=0):
    """Two-phase binary 2-D strip (ny rows), periodic, solid slab in the middle."""
    p = W.binary_problem("planar", nx, ny=ny, delta=delta, Delta=-f0_s, R=0.0,
                         potential=potential, eps=eps, steps=steps)
    p.ceq = np.array([[ceq_s], [0.817]])
    p.D = np.array([[[0.0]], [[D_l]]])
    if dt is None:
        dt = 0.2 * 0.5 / (1.0 * (1 + 15 * delta))   # 1-D bound dx^2/2 with ny = 1
    p.dt = dt
    x = (np.arange(nx) + 0.5)
    # start from a deliberately wrong (linear-ramp) profile of the solid slab
    c1, c2 = nx / 4.0, 3 * nx / 4.0
    w = 3.0 * eps
    s = np.clip(0.5 + (x - c1) / w, 0, 1) * np.clip(0.5 + (c2 - x) / w, 0, 1)
    ps = np.broadcast_to(s[None, None, :], (1, ny, nx)).copy()
    p.phi0 = np.stack([ps, 1.0 - ps])
    p.mu0 = np.full((1, 1, ny, nx), 2.0 * 0.817)
    return p


def crossing_slope(phi_row, dx=1.0):
    """Slope of phi at its first rising 0.5 crossing (linear interpolation)."""
    for i in range(len(phi_row) - 1):
        a, b = phi_row[i], phi_row[i + 1]
        if a < 0.5 <= b:
            return (b - a) / dx, i + (0.5 - a) / (b - a)
    raise AssertionError("no crossing")


# ----------------------------------------------------------------- anisotropy
def test_ac_fourfold_closed_form_2d():
    p = W.small_multiphase(n=4, dim=2, N=2, NM=1)
    rng = np.random.default_rng(1)
    for _ in range(50):
        d = rng.uniform(0.0, 0.06)
        th = rng.uniform(0, 2 * math.pi)
        r = rng.uniform(0.1, 2.0)
        gam = p.gamma[0, 1]
        delta = np.array([[0, d], [d, 0]])
        q = r * np.array([math.cos(th), math.sin(th)])
        A = oracle.pair_energy(p, 0, 1, q, delta=delta)
        assert A == pytest.approx(gam * (1 + d * math.cos(4 * th)) ** 2 * r * r, rel=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_pair_energy_grad_matches_finite_difference(dim):
    rng = np.random.default_rng(2 + dim)
    p = W.small_multiphase(n=4, dim=dim, N=3, NM=1, rotate=True)
    for _ in range(30):
        q = rng.normal(size=dim)
        for (a, b) in [(0, 1), (0, 2), (1, 2)]:
            g = oracle.pair_energy_grad(p, a, b, q)
            h = 1e-6
            fd = np.zeros(dim)
            for i in range(dim):
                e = np.zeros(dim)
                e[i] = h
                fd[i] = (oracle.pair_energy(p, a, b, q + e) - oracle.pair_energy(p, a, b, q - e)) / (2 * h)
            np.testing.assert_allclose(g, fd, rtol=1e-7, atol=1e-9)


def test_rotation_identity_and_quarter_turn_invariance():
    rng = np.random.default_rng(5)
    p = W.small_multiphase(n=4, dim=3, N=2, NM=1)
    d = np.array([[0, 0.04], [0.04, 0]])
    eye = np.tile(np.eye(3), (2, 2, 1, 1))
    Rz = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    rz = np.tile(Rz, (2, 2, 1, 1))
    for _ in range(20):
        q = rng.normal(size=3)
        a0 = oracle.pair_energy(p, 0, 1, q, delta=d, rot=eye)
        a1 = oracle.pair_energy(p, 0, 1, q, delta=d, rot=rz)
        assert a1 == pytest.approx(a0, rel=1e-13)
        # a generic rotation changes the energy of a generic q
    R = W.shoemake_rotation(W.PCG32(3))
    q = np.array([1.0, 0.2, -0.3])
    assert abs(oracle.pair_energy(p, 0, 1, q, delta=d, rot=np.tile(R, (2, 2, 1, 1))) -
               oracle.pair_energy(p, 0, 1, q, delta=d, rot=eye)) > 1e-4


def test_isotropic_pair_gradient_is_exactly_two_gamma_q():
    p = W.small_multiphase(n=4, dim=3, N=3, NM=1, aniso=False)
    q = np.array([1e-8, -2e-7, 0.3])
    g = oracle.pair_energy_grad(p, 0, 2, q)
    np.testing.assert_array_equal(g, 2.0 * p.gamma[0, 2] * q)


# ------------------------------------------------------ interpolation, potential
@pytest.mark.parametrize("N", [2, 3, 5, 8])
def test_interpolation_partition_of_unity_and_derivative(N):
    rng = np.random.default_rng(N)
    for _ in range(20):
        phi = rng.dirichlet(np.ones(N))
        h, dh = oracle.interp(phi)
        assert h.sum() == pytest.approx(1.0, abs=1e-14)
        eps = 1e-6
        for a in range(N):
            e = np.zeros(N)
            e[a] = eps
            fd = (oracle.interp(phi + e)[0] - oracle.interp(phi - e)[0]) / (2 * eps)
            np.testing.assert_allclose(dh[:, a], fd, rtol=1e-7, atol=1e-9)
    for a in range(N):   # vertices map to themselves
        h, _ = oracle.interp(np.eye(N)[a])
        np.testing.assert_array_equal(h, np.eye(N)[a])


@pytest.mark.parametrize("pot", ["obstacle", "well"])
def test_potential_derivative_matches_finite_difference(pot):
    p = W.small_multiphase(n=4, dim=3, N=4, NM=1, potential=pot, gamma3=0.7)
    rng = np.random.default_rng(9)
    for _ in range(20):
        phi = rng.dirichlet(np.ones(4))
        w, dw = oracle.potential(p, phi)
        eps = 1e-6
        for a in range(4):
            e = np.zeros(4)
            e[a] = eps
            fd = (oracle.potential(p, phi + e)[0] - oracle.potential(p, phi - e)[0]) / (2 * eps)
            assert dw[a] == pytest.approx(fd, rel=1e-7, abs=1e-9)


def test_obstacle_two_phase_energy_integrates_to_gamma():
    """1-D interface energy of the sine profile equals gamma (Eq. Obstacle scaling)."""
    p = W.binary_problem("e", 8, potential="obstacle")
    eps, gam = p.eps, 1.0
    lim = math.pi ** 2 * eps / 8
    x = np.linspace(-lim, lim, 200001)
    phi = 0.5 * (1 + np.sin(4 * x / (math.pi * eps)))
    dphi = np.gradient(phi, x)
    w = np.array([oracle.potential(p, np.array([f, 1 - f]))[0] for f in phi[::100]])
    grad_e = eps * np.array([oracle.pair_energy(p, 0, 1, np.array([-d, 0.0])) for d in dphi[::100]])
    sigma = np.trapezoid(grad_e + w / eps, x[::100])
    assert sigma == pytest.approx(gam, rel=2e-4)


# ------------------------------------------------------------------ projection
def brute_simplex(v):
    N = len(v)
    best, bx = np.inf, None
    for mask in range(1, 1 << N):
        S = [i for i in range(N) if mask >> i & 1]
        x = np.zeros(N)
        x[S] = v[S] - (v[S].sum() - 1.0) / len(S)
        if (x >= -1e-15).all():
            d = ((x - v) ** 2).sum()
            if d < best:
                best, bx = d, x
    return np.maximum(bx, 0.0)


@pytest.mark.parametrize("N", [2, 3, 4])
def test_simplex_projection_matches_brute_force(N):
    rng = np.random.default_rng(10 + N)
    for _ in range(200):
        v = rng.normal(scale=0.7, size=N) + 1.0 / N
        np.testing.assert_allclose(oracle.project(v, "obstacle"), brute_simplex(v), atol=1e-13)
    x = rng.dirichlet(np.ones(N))   # points on the simplex are fixed
    np.testing.assert_allclose(oracle.project(x, "obstacle"), x, atol=1e-15)


def test_hyperplane_projection_closed_form():
    rng = np.random.default_rng(3)
    for N in (2, 3, 8):
        v = rng.normal(size=N)
        out = oracle.project(v, "well")
        np.testing.assert_allclose(out, v - v.mean() + 1.0 / N, atol=1e-14)


# ------------------------------------------------------------- thermodynamics
def test_parabolic_thermodynamics_meets_equilibrium_conditions():
    """Coeff_B / Coeff_C reproduce equal mu and equal psi at c_eq (Sec. 3)."""
    from scipy.optimize import brentq, fsolve
    p = W.small_multiphase(n=4, dim=3, N=3, NM=2)   # off-diagonal A, slopes on liquid
    L = p.n_phases - 1
    for T in (0.0, 0.7):
        cl = p.ceq[L] + p.slopes[L] * (T - p.T_ref)
        mu_eq = fsolve(lambda m: oracle.thermo(p, L, m, T)[0] - cl, np.zeros(2), xtol=1e-14)
        psi_l = oracle.thermo(p, L, mu_eq, T)[1] - p.f0[L]
        for a in range(L):
            c, psi, chi = oracle.thermo(p, a, mu_eq, T)
            ca = p.ceq[a] + p.slopes[a] * (T - p.T_ref)
            np.testing.assert_allclose(c, ca, atol=1e-12)
            assert psi - p.f0[a] == pytest.approx(psi_l, abs=1e-12)
    # psi is the Legendre transform: d psi/d mu = -c and d c/d mu = chi
    mu = np.array([0.3, 0.9])
    for a in range(p.n_phases):
        c, psi, chi = oracle.thermo(p, a, mu, 0.2)
        h = 1e-6
        for j in range(2):
            e = np.zeros(2)
            e[j] = h
            cp, pp, _ = oracle.thermo(p, a, mu + e, 0.2)
            cm, pm, _ = oracle.thermo(p, a, mu - e, 0.2)
            assert (pp - pm) / (2 * h) == pytest.approx(-c[j], rel=1e-7, abs=1e-9)
            np.testing.assert_allclose((cp - cm) / (2 * h), chi[:, j], rtol=1e-7, atol=1e-9)


# --------------------------------------------------------- discrete identities
@pytest.mark.parametrize("dim", [2, 3])
def test_isotropic_two_phase_gradient_terms_are_a_laplacian(dim):
    """div J_1 - G_1 - (div J_2 - G_2) = 2 gamma Lap(phi_1) to round-off."""
    n = 12
    p = W.small_multiphase(n=n, dim=dim, N=2, NM=1, aniso=False,
                           bc=[W.BC_PERIODIC] * 3)
    rng = np.random.default_rng(4)
    shape = (p.nz, p.ny, p.nx)
    f = 0.5 + 0.4 * np.sin(2 * np.pi * rng.integers(1, 3) * (np.indices(shape)[2] + 0.3) / n) * \
        np.cos(2 * np.pi * (np.indices(shape)[1] + np.indices(shape)[0]) / n)
    phi = np.stack([f, 1 - f])
    divJ, Gc, Wd, P = oracle.rate_parts(p, phi, p.mu0)
    lhs = (divJ[0] - Gc[0]) - (divJ[1] - Gc[1])
    axes = (3, 2, 1)[:dim]
    lap = sum(np.roll(phi[0:1], 1, ax) + np.roll(phi[0:1], -1, ax) - 2 * phi[0:1] for ax in axes)[0]
    np.testing.assert_allclose(lhs, 2.0 * p.gamma[0, 1] * lap, atol=1e-13)


@pytest.mark.parametrize("pot,expected", [
    ("obstacle", lambda x, e: 0.5 * (1 + np.sin(np.clip(4 * x / (math.pi * e), -math.pi / 2, math.pi / 2)))),
    ("well", lambda x, e: 0.5 * (1 + np.tanh(3 * x / (2 * e)))),
])
def test_planar_equilibrium_profile_second_order(pot, expected):
    """Relaxed planar interface vs the 1-D sine / tanh profile; error ~ dx^2/eps^2."""
    errs = []
    for eps in (4.0, 8.0):
        nx = int(32 * eps)
        p = planar_problem(nx, eps, pot)
        steps = int(60 * eps * eps / p.dt)
        phi, mu = oracle.run(p, p.phi0, p.mu0, steps)
        row = phi[0, 0, 0]
        _, x0 = crossing_slope(row)
        x = np.arange(nx) - x0
        sel = np.abs(x) < (math.pi ** 2 * eps / 8 if pot == "obstacle" else 2 * eps)
        errs.append(np.abs(row[sel] - expected(x[sel], eps)).max())
    assert errs[0] < 0.02
    assert 3.0 < errs[0] / errs[1] < 5.5, errs


@pytest.mark.parametrize("angle", [0, 45])
def test_anisotropic_planar_width(angle):
    """Four-fold anisotropy scales the profile width by (1+delta) at 0 deg, (1-delta) at 45 deg."""
    eps, d = 4.0, 0.05
    if angle == 0:
        nx = 128
        p = planar_problem(nx, eps, "obstacle", delta=d)
        phi, _ = oracle.run(p, p.phi0, p.mu0, int(60 * eps * eps / p.dt))
        slope, _ = crossing_slope(phi[0, 0, 0])
    else:
        n = 64
        p = planar_problem(n, eps, "obstacle", delta=d, ny=n, dt=0.2 * 0.25 / (1 + 15 * d))
        ii, jj = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5)
        s = (ii + jj) % n   # slab in the diagonal coordinate, periodic
        w = 3 * eps
        f = np.clip(0.5 + (s - n / 4) / w, 0, 1) * np.clip(0.5 + (3 * n / 4 - s) / w, 0, 1)
        p.phi0 = np.stack([f[None], 1 - f[None]])
        p.mu0 = np.full((1, 1, n, n), 2 * 0.817)
        phi, _ = oracle.run(p, p.phi0, p.mu0, int(60 * eps * eps / p.dt))
        # along x the diagonal coordinate s advances by 1 per cell, its normal by 1/sqrt 2
        slope_x, _ = crossing_slope(phi[0, 0, n // 2])
        slope = slope_x * math.sqrt(2.0)
    eps_eff = 2.0 / (math.pi * slope)
    factor = eps_eff / eps
    want = 1 + d if angle == 0 else 1 - d
    assert factor == pytest.approx(want, abs=0.012), (factor, want)


@pytest.mark.parametrize("dim", [2, 3])
def test_fourier_mode_decay_is_exact(dim):
    """Single phase: mu modes decay by (1 - 4 D dt sum sin^2(pi k/n)) per step."""
    n = 16
    p = W.small_multiphase(n=n, dim=dim, N=2, NM=1, bc=[W.BC_PERIODIC] * 3)
    p.A = np.array([[[1.0]], [[1.3]]])
    p.D = np.array([[[0.0]], [[0.7]]])
    p.G = 0.0
    p.dt = 0.2 * 1.0 / (2 * dim * 0.7)
    shape = (p.nz, p.ny, p.nx)
    idx = np.indices(shape)
    k = (1, 2, 3)[:dim]
    arg = sum(2 * np.pi * k[d] * (idx[2 - d] + 0.5) / n for d in range(dim))
    amp = 0.01
    mu0 = (1.0 + amp * np.cos(arg))[None]
    phi0 = np.stack([np.zeros(shape), np.ones(shape)])
    steps = 40
    phi, mu = oracle.run(p, phi0, mu0, steps)
    lam = 1 - 4 * 0.7 * p.dt * sum(math.sin(math.pi * k[d] / n) ** 2 for d in range(dim))
    np.testing.assert_allclose(mu[0] - 1.0, amp * lam ** steps * np.cos(arg), atol=1e-14)
    np.testing.assert_array_equal(phi[1], 1.0)
    np.testing.assert_array_equal(phi[0], 0.0)


def test_gaussian_diffusion_matches_continuum():
    n = 96
    p = W.small_multiphase(n=n, dim=2, N=2, NM=1, bc=[W.BC_PERIODIC] * 3)
    p.A = np.array([[[1.0]], [[1.0]]])
    p.D = np.array([[[0.0]], [[1.0]]])
    p.G = 0.0
    p.dt = 0.05
    shape = (1, n, n)
    idx = np.indices(shape)
    r2 = (idx[2] + 0.5 - n / 2) ** 2 + (idx[1] + 0.5 - n / 2) ** 2
    s0 = 8.0
    mu0 = (np.exp(-r2 / (2 * s0 ** 2)))[None]
    phi0 = np.stack([np.zeros(shape), np.ones(shape)])
    steps = 400
    _, mu = oracle.run(p, phi0, mu0, steps)
    t = steps * p.dt
    s2 = s0 ** 2 + 2 * t
    exact = (s0 ** 2 / s2) * np.exp(-r2 / (2 * s2))
    assert np.abs(mu[0] - exact).max() < 2e-3


# ------------------------------------------------------------------ invariants
@pytest.mark.parametrize("pot", ["obstacle", "well"])
@pytest.mark.parametrize("dim", [2, 3])
def test_sum_phi_one_and_mass_conserved(pot, dim):
    p = W.small_multiphase(n=12, dim=dim, N=3, NM=2, potential=pot, rotate=True, gamma3=0.3)
    steps = 15
    d0 = oracle.diag(p, p.phi0, p.mu0)
    phi, mu = oracle.run(p, p.phi0, p.mu0, steps)
    d1 = oracle.diag(p, phi, mu, t0=steps * p.dt)
    np.testing.assert_allclose(d1[:2], d0[:2], rtol=1e-13)
    assert d1[2] < 1e-14
    if pot == "obstacle":
        assert phi.min() >= 0.0


def test_local_composition_conserved_without_diffusion():
    """D = 0: c = sum h c^a(mu,T) is conserved cell by cell, including the dT/dt term."""
    p = W.small_multiphase(n=8, dim=3, N=3, NM=2)
    p.D = np.zeros_like(p.D)
    p.G, p.V = 0.05, 0.3
    steps = 5
    phi, mu = oracle.run(p, p.phi0, p.mu0, steps)

    def comp(phi, mu, t):
        out = np.zeros((2,) + phi.shape[1:])
        for z in range(p.nz):
            T = p.T0 + p.G * ((z + 0.5) - p.z0 - p.V * t)
            for y in range(p.ny):
                for x in range(p.nx):
                    h, _ = oracle.interp(phi[:, z, y, x])
                    for a in range(3):
                        c, _, _ = oracle.thermo(p, a, mu[:, z, y, x], T)
                        out[:, z, y, x] += h[a] * c
        return out

    np.testing.assert_allclose(comp(phi, mu, steps * p.dt), comp(p.phi0, p.mu0, 0.0), atol=2e-14)
    assert np.abs(mu - p.mu0).max() > 1e-4   # mu did move


def test_single_phase_domain_stays_bitwise():
    p = W.small_multiphase(n=10, dim=3, N=3, NM=2)
    shape = (p.nz, p.ny, p.nx)
    phi0 = np.stack([np.zeros(shape), np.zeros(shape), np.ones(shape)])
    phi, _ = oracle.run(p, phi0, p.mu0, 5)
    np.testing.assert_array_equal(phi, phi0)


def test_flat_interface_at_equal_mu_stays_put():
    eps = 4.0
    nx = 128
    p = planar_problem(nx, eps, "obstacle", ceq_s=0.817)    # equal c: mu frozen
    relax = int(60 * eps * eps / p.dt)
    phi, mu = oracle.run(p, p.phi0, p.mu0, relax)
    _, x0 = crossing_slope(phi[0, 0, 0])
    q = planar_problem(nx, eps, "obstacle", ceq_s=0.926)     # real two-phase alloy
    phi2, mu2 = oracle.run(q, phi, mu, 1000)
    _, x1 = crossing_slope(phi2[0, 0, 0])
    assert abs(x1 - x0) < 1e-8
    assert np.abs(mu2 - 2 * 0.817).max() < 1e-10


@pytest.mark.parametrize("R_over_Rstar,grows", [(0.7, False), (1.5, True)])
def test_gibbs_thomson_direction(R_over_Rstar, grows):
    Delta = 0.1
    Rstar = 1.0 / Delta
    n = 64
    p = W.binary_problem("gt", n, Delta=Delta, R=R_over_Rstar * Rstar, potential="obstacle")
    p.ceq = np.array([[0.817], [0.817]])     # equal compositions: mu stays frozen
    s0 = p.phi0[0].sum()
    phi, mu = oracle.run(p, p.phi0, p.mu0, 600)
    s1 = phi[0].sum()
    assert (s1 > s0) == grows
    assert abs(s1 - s0) > 5.0


def test_dendrite_2d_mirror_and_transpose_symmetry():
    p = W.dendrite_2d()
    phi, mu = oracle.run(p, p.phi0, p.mu0, 100)
    f = phi[0, 0]
    np.testing.assert_allclose(f, f.T, atol=1e-13)
    np.testing.assert_allclose(f, f[:, ::-1], atol=1e-13)
    np.testing.assert_allclose(f, f[::-1, :], atol=1e-13)


# ---------------------------------------------------------------------- tangent
def test_tangent_matches_central_differences():
    p = W.small_multiphase(n=10, dim=2, N=2, NM=1, potential="well")
    rng = np.random.default_rng(12)
    steps = 12
    v = rng.normal(size=p.phi0.shape)
    v -= v.mean(axis=0, keepdims=True)       # keep sum phi = 1 along the direction
    vm = rng.normal(size=p.mu0.shape) * 0.1
    dd = np.array([[0, 1.0], [1.0, 0]])
    dD = np.array([[[0.0]], [[1.0]]])
    for kind in ("phi", "delta", "mob", "D"):
        kw = dict(dphi0=v, dmu0=vm) if kind == "phi" else {}
        if kind == "delta":
            kw = dict(ddelta=dd)
        if kind == "mob":
            kw = dict(dmob=1.0)
        if kind == "D":
            kw = dict(dD=dD)
        _, _, tphi, tmu = oracle.run_tangent(p, p.phi0, p.mu0, steps, **kw)
        h = 1e-6

        def fwd(s):
            if kind == "phi":
                return oracle.run(p, p.phi0 + s * v, p.mu0 + s * vm, steps)
            if kind == "delta":
                return oracle.run(p, p.phi0, p.mu0, steps, delta=p.delta + s * dd)
            if kind == "mob":
                return oracle.run(p, p.phi0, p.mu0, steps, tau=1.0 / (1.0 / p.tau + s))
            return oracle.run(p, p.phi0, p.mu0, steps, D=p.D + s * dD)

        pp, mp = fwd(h)
        pm, mm = fwd(-h)
        fd_phi = (pp - pm) / (2 * h)
        fd_mu = (mp - mm) / (2 * h)
        scale = max(np.abs(fd_phi).max(), 1e-3)
        assert np.abs(tphi - fd_phi).max() / scale < 1e-6, kind
        scale = max(np.abs(fd_mu).max(), 1e-3)
        assert np.abs(tmu - fd_mu).max() / scale < 1e-6, kind
