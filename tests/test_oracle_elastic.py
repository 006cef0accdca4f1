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
