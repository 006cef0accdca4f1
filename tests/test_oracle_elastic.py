"""Pins of the oracle's homogeneous-stiffness elasticity (Sec. 2 "Elasticity
implementation", the Fourier-space equilibrium of its homogeneous case), on
the CPU.

A laminate (fields varying along x only) has a closed-form equilibrium: the
normal stress along x is uniform, the mean strain is zero, and the in-plane
stresses follow pointwise; a uniform phase carries sigma = -C eps*; any
state's stress must be divergence-free (checked spectrally here, independently
of how the oracle solves for it); and with an isotropic stiffness the energy
of a dilatational inclusion depends on its volume only (the classical
shape independence), with a closed form in the volume fraction.
"""
import numpy as np
import pytest

import oracle
import workloads as W

C11, C12, C44 = 150.0, 60.0, 75.0


def _cubic():
    C = np.zeros((6, 6))
    C[:3, :3] = C12
    np.fill_diagonal(C[:3, :3], C11)
    C[3, 3] = C[4, 4] = C[5, 5] = C44
    return C


def _laminate(dim, e0=0.012, n=48):
    p = W.binary_problem("el_lam", n, dim=dim, ny=6, nz=5 if dim == 3 else None)
    x = (np.arange(n) + 0.5)[None, None, :]
    s = 0.5 * (1.0 + np.sin(2.0 * np.pi * x / n) * 0.9)          # smooth, strictly inside (0, 1)
    nz = 5 if dim == 3 else 1
    phi = np.zeros((2, nz, 6, n))
    phi[0] = np.broadcast_to(s, (nz, 6, n))
    phi[1] = 1.0 - phi[0]
    p.elastic_C = _cubic()
    eig = np.zeros((2, 3, 3))
    eig[0] = np.eye(3) * e0
    p.eigenstrain = eig
    return p, phi


@pytest.mark.parametrize("dim", [3, 2])
def test_laminate_closed_form(dim):
    e0 = 0.012
    p, phi = _laminate(dim, e0)
    sigma, w = oracle.elastic_fields(p, phi)
    f = phi[0]
    h = f * f * (3.0 - 2.0 * f)                 # two phases: h_0 = phi_0^2 (3 - 2 phi_0)
    # eigenstrain e0 h on the first `dim` axes; strains along y (and z) vanish
    B = (C11 + (dim - 1) * C12) * e0            # C_xx,mm eps*_mm / h
    sxx = -B * h.mean()                          # uniform, from zero mean strain
    exx = (sxx + B * h) / C11
    syy = C12 * exx - (C12 + C11 + (dim - 2) * C12) * e0 * h
    np.testing.assert_allclose(sigma[0, 0], sxx, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(sigma[1, 1], syy, rtol=1e-10, atol=1e-12)
    if dim == 3:
        np.testing.assert_allclose(sigma[2, 2], syy, rtol=1e-10, atol=1e-12)
    off = [sigma[i, j] for i in range(dim) for j in range(dim) if i != j]
    assert max(np.abs(o).max() for o in off) < 1e-12
    trace = sum(sigma[i, i] for i in range(dim))
    np.testing.assert_allclose(w[0], -e0 * trace, rtol=1e-10, atol=1e-12)
    assert np.abs(w[1]).max() == 0.0


def test_uniform_shear_eigenstrain_voigt_factor():
    # one phase everywhere with a pure shear eigenstrain eps*_xy = g: zero
    # strain, sigma = -C eps*, sigma_xy = -C66 (2 g), w = -sigma : eps* = 4 C66 g^2
    g = 0.007
    p = W.binary_problem("el_shear", 8, dim=3, ny=8, nz=8)
    p.elastic_C = _cubic()
    eig = np.zeros((2, 3, 3))
    eig[0, 0, 1] = eig[0, 1, 0] = g
    p.eigenstrain = eig
    phi = np.zeros((2, 8, 8, 8))
    phi[0] = 1.0
    sigma, w = oracle.elastic_fields(p, phi)
    np.testing.assert_allclose(sigma[0, 1], -C44 * 2.0 * g, rtol=1e-12)
    np.testing.assert_allclose(w[0], 4.0 * C44 * g * g, rtol=1e-12)


@pytest.mark.parametrize("dim", [3, 2])
def test_stress_is_divergence_free(dim):
    p = W.small_multiphase(n=16, dim=dim, N=3, NM=2, nx=16, ny=12, nz=10 if dim == 3 else None)
    p.elastic_C = _cubic()
    rng = np.random.default_rng(3)
    eig = rng.normal(scale=0.01, size=(3, 3, 3))
    p.eigenstrain = 0.5 * (eig + np.transpose(eig, (0, 2, 1)))
    sigma, _ = oracle.elastic_fields(p, p.phi0)
    nz = p.nz if dim == 3 else 1
    shape = (nz, p.ny, p.nx)
    ks = []
    for n in (p.nx, p.ny, nz)[:dim]:          # FFT order, the Nyquist index of an even extent as 0
        k = 2 * np.pi * np.fft.fftfreq(n)
        if n % 2 == 0:
            k[n // 2] = 0.0
        ks.append(k)
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    axes = (2, 3, 4) if dim == 3 else (3, 4)
    sh = np.fft.fftn(sigma, axes=axes)
    div = sum(ks[j][grids[2 - j]] * sh[:, j] for j in range(dim))
    scale = np.abs(sh).max() * max(np.abs(k).max() for k in ks)
    assert np.abs(div).max() <= 1e-11 * scale
    assert np.abs(sigma).max() > 1e-3


def _energy(w, phi):
    # E = 1/2 int sigma:(eps - eps*) = -1/2 int sigma:eps* (int sigma:eps = 0 at
    # equilibrium in a periodic box with zero mean strain) = 1/2 sum h_b w_b
    h = np.where(phi > 0.5, 1.0, 0.0)             # sharp fields: h = phi
    return 0.5 * float((h * w).sum())


def test_isotropic_dilatational_energy_is_shape_independent():
    # Homogeneous isotropic stiffness (lambda, mu) and a dilatational misfit
    # e0 in a sharp inclusion of volume fraction f: with K = lambda + 2 mu / 3
    # the equilibrium strain trace is 3 K e0 (chi - f) / (lambda + 2 mu), so
    # E = (9 K e0^2 V / 2) [f - K (f - f^2) / (lambda + 2 mu)] whatever the
    # inclusion's shape (odd extents: no Nyquist modes).
    lam, mu, e0 = 80.0, 50.0, 0.01
    C = np.zeros((6, 6))
    C[:3, :3] = lam
    np.fill_diagonal(C[:3, :3], lam + 2 * mu)
    C[3, 3] = C[4, 4] = C[5, 5] = mu
    n = 21
    p = W.binary_problem("el_eshelby", n, dim=3, ny=n, nz=n)
    p.elastic_C = C
    eig = np.zeros((2, 3, 3))
    eig[0] = np.eye(3) * e0
    p.eigenstrain = eig
    z, y, x = np.meshgrid(*[np.arange(n) - n // 2] * 3, indexing="ij")
    ball = (x ** 2 + y ** 2 + z ** 2) <= 5.3 ** 2
    cells = int(ball.sum())
    slab = np.zeros(n ** 3, bool)
    slab[:cells] = True                          # the same number of cells as planes and a partial row
    slab = slab.reshape(n, n, n)
    K = lam + 2 * mu / 3
    V = float(n ** 3)
    f = cells / V
    expect = 4.5 * K * e0 ** 2 * V * (f - K * (f - f * f) / (lam + 2 * mu))
    for shape in (ball, slab):
        phi = np.zeros((2, n, n, n))
        phi[0] = shape
        phi[1] = 1.0 - phi[0]
        _, w = oracle.elastic_fields(p, phi)
        assert _energy(w, phi) == pytest.approx(expect, rel=1e-10)


@pytest.mark.parametrize("dim", [2, 3])
def test_fields_do_not_depend_on_the_grid_spacing(dim):
    # strain is dimensionless: the same eigenstrain pattern in cells gives the
    # same stress at any dx (the wavenumbers' 1/dx cancels between the
    # displacement and its gradient); a missing dx in one of them would not
    rng = np.random.default_rng(4)
    n = 12
    nz = 10 if dim == 3 else 1
    p = W.binary_problem("el_dx", n, dim=dim, ny=11, nz=nz if dim == 3 else None,
                         bc=[W.BC_PERIODIC] * 3)
    phi = np.zeros((2, nz, 11, n))
    phi[0] = rng.uniform(0.0, 1.0, size=(nz, 11, n))
    phi[1] = 1.0 - phi[0]
    p.elastic_C = _cubic()
    eig = np.zeros((2, 3, 3))
    eig[0] = np.array([[0.01, 0.002, 0.0], [0.002, -0.004, 0.001], [0.0, 0.001, 0.006]])
    p.eigenstrain = eig
    s1, w1 = oracle.elastic_fields(p, phi)
    s2, w2 = oracle.elastic_fields(p.copy(dx=0.37), phi)
    assert np.abs(s1).max() > 0.1
    np.testing.assert_allclose(s2, s1, rtol=0, atol=1e-12 * np.abs(s1).max())
    np.testing.assert_allclose(w2, w1, rtol=0, atol=1e-12 * np.abs(w1).max())


# ------------------------------------------------ stiffness varying with the phases
def _cubic_of(c11, c12, c44):
    C = np.zeros((6, 6))
    C[:3, :3] = c12
    np.fill_diagonal(C[:3, :3], c11)
    C[3, 3] = C[4, 4] = C[5, 5] = c44
    return C


def _random_state(dim, seed=3):
    p = W.small_multiphase(n=12, dim=dim, N=3, NM=2, nx=12, ny=10, nz=8 if dim == 3 else None)
    rng = np.random.default_rng(seed)
    eig = rng.normal(scale=0.01, size=(3, 3, 3))
    p.eigenstrain = 0.5 * (eig + np.transpose(eig, (0, 2, 1)))
    return p


def test_inhomogeneous_solve_reduces_to_the_homogeneous_one():
    p = _random_state(3)
    p.elastic_C = _cubic()
    s0, w0 = oracle.elastic_fields(p, p.phi0)
    s1, w1, it = oracle.elastic_fields_inhomogeneous(p, p.phi0, [_cubic()] * 3)
    scale = np.abs(s0).max()
    assert np.abs(s1 - s0).max() <= 1e-12 * scale and it <= 2
    # the 1/2 e:C^b:e term is the same for every phase: it cancels in the
    # contraction with dh/dphi, so only differences of w matter
    d0, d1 = w0 - w0[0], w1 - w1[0]
    assert np.abs(d1 - d0).max() <= 1e-12 * np.abs(w0).max()


@pytest.mark.parametrize("dim", [3, 2])
def test_inhomogeneous_laminate_closed_form(dim):
    """Two phases with different cubic stiffnesses (contrast 2) in a laminate along
    x: sigma_xx is uniform, the strains along y (and z) vanish, and the zero mean
    of eps_xx fixes sigma_xx; every other stress follows pointwise from the local
    stiffness C(x) = sum_b C^b h_b."""
    e0 = 0.012
    p, phi = _laminate(dim, e0)
    Ca, Cb = (150.0, 60.0, 75.0), (300.0, 110.0, 130.0)
    sigma, w, it = oracle.elastic_fields_inhomogeneous(p, phi, [_cubic_of(*Ca), _cubic_of(*Cb)])
    f = phi[0]
    h = f * f * (3.0 - 2.0 * f)
    c11 = Ca[0] * h + Cb[0] * (1.0 - h)
    c12 = Ca[1] * h + Cb[1] * (1.0 - h)
    # sigma_xx = c11 (eps_xx - e0 h) - (dim - 1) c12 e0 h = S, mean(eps_xx) = 0
    S = -np.mean(e0 * h + (dim - 1) * c12 * e0 * h / c11) / np.mean(1.0 / c11)
    exx = e0 * h + (S + (dim - 1) * c12 * e0 * h) / c11
    syy = c12 * (exx - e0 * h) - c11 * e0 * h - (dim - 2) * c12 * e0 * h
    np.testing.assert_allclose(sigma[0, 0], S, rtol=1e-10)
    np.testing.assert_allclose(sigma[1, 1], syy, rtol=1e-10, atol=1e-12 * abs(S))
    if dim == 3:
        np.testing.assert_allclose(sigma[2, 2], syy, rtol=1e-10, atol=1e-12 * abs(S))
    off = [sigma[i, j] for i in range(dim) for j in range(dim) if i != j]
    assert max(np.abs(o).max() for o in off) < 1e-12 * abs(S)
    assert it > 3                                   # the contrast needs the iteration


@pytest.mark.parametrize("dim", [3, 2])
def test_inhomogeneous_stress_is_divergence_free(dim):
    p = _random_state(dim)
    C = [_cubic_of(150, 60, 75), _cubic_of(240, 90, 110), _cubic_of(110, 50, 60)]
    sigma, _, _ = oracle.elastic_fields_inhomogeneous(p, p.phi0, C)
    nz = p.nz if dim == 3 else 1
    shape = (nz, p.ny, p.nx)
    ks = []
    for n in (p.nx, p.ny, nz)[:dim]:
        k = 2 * np.pi * np.fft.fftfreq(n)
        if n % 2 == 0:
            k[n // 2] = 0.0
        ks.append(k)
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    axes = (2, 3, 4) if dim == 3 else (3, 4)
    sh = np.fft.fftn(sigma, axes=axes)
    div = sum(ks[j][grids[2 - j]] * sh[:, j] for j in range(dim))
    assert np.abs(div).max() <= 1e-10 * np.abs(sh).max() * max(np.abs(k).max() for k in ks)


def test_inhomogeneous_potentials_are_the_phase_derivative_of_the_energy():
    """w_b contracted with the change of h_b is the change of the equilibrium
    elastic energy E = 1/2 int e : C(phi) : e (= -1/2 int sigma : eps* at
    equilibrium with zero mean strain), checked by central differences of two
    whole solves along a random direction in phi that keeps sum phi = 1 (the
    directions the step moves in; on them sum h = 1, so C(x) = sum_b C^b h_b
    exactly)."""
    p = _random_state(3, seed=5)
    C = [_cubic_of(150, 60, 75), _cubic_of(240, 90, 110), _cubic_of(110, 50, 60)]
    eig = np.asarray(p.eigenstrain)

    def energy(phi):
        sigma, _, _ = oracle.elastic_fields_inhomogeneous(p, phi, C, tol=1e-14)
        E = np.einsum("amn,a...->mn...", eig, oracle.interp_field(phi))
        return -0.5 * float((sigma * E).sum())

    rng = np.random.default_rng(9)
    d = rng.normal(size=p.phi0.shape) * 0.05
    d -= d.mean(axis=0, keepdims=True)           # along sum phi = 1, where sum h = 1 too
    s = 1e-4
    dE = (energy(p.phi0 + s * d) - energy(p.phi0 - s * d)) / (2 * s)
    _, w, _ = oracle.elastic_fields_inhomogeneous(p, p.phi0, C, tol=1e-14)
    dh = (oracle.interp_field(p.phi0 + s * d) - oracle.interp_field(p.phi0 - s * d)) / (2 * s)
    pred = float((w * dh).sum())
    assert pred == pytest.approx(dE, rel=1e-6)
    # without the 1/2 e:C^b:e term the derivative would be wrong by far more
    sig, _, _ = oracle.elastic_fields_inhomogeneous(p, p.phi0, C, tol=1e-14)
    w_no = -np.einsum("ij...,bij->b...", sig, eig)
    assert abs(float((w_no * dh).sum()) - dE) > 1e-3 * abs(dE)


def test_steps_with_per_phase_stiffnesses():
    """run() with one stiffness per phase: equal stiffnesses step like the
    homogeneous solve; a contrast changes the trajectory."""
    p = _random_state(2, seed=7)
    p.elastic_C = _cubic()
    a = oracle.run(p, p.phi0, p.mu0, 3)
    q = p.copy(elastic_C=None)
    b = oracle.run(q, p.phi0, p.mu0, 3, elastic_C_phases=[_cubic()] * 3)
    assert max(np.abs(a[0] - b[0]).max(), np.abs(a[1] - b[1]).max()) < 1e-12
    c = oracle.run(q, p.phi0, p.mu0, 3, elastic_C_phases=[_cubic(), _cubic_of(300, 110, 130), _cubic()])
    assert np.abs(c[0] - a[0]).max() > 1e-9
