"""Pins of the oracle's phi noise and moving frame (CPU).

The noise variate is pinned by its distribution (uniform on a 2^-24 grid in
[-1/2, 1/2): mean, variance 1/12, no lag-1 correlation, dependence on every
counter input); its place in the step by the projection identity of an
interior simplex cell; the moving frame by its definition, by the equivalence
of a lab origin with a moved temperature field, and by commuting with a step
on a state that is uniform along the last axis near the dropped planes.
"""
import numpy as np
import pytest

import oracle
import workloads as W


def test_noise_variate_distribution():
    n = 200_000
    xs = np.array([oracle.noise(12345, 7, k) for k in range(n)])
    assert xs.min() >= -0.5 and xs.max() < 0.5
    grid = (xs + 0.5) * 2.0 ** 24
    assert np.array_equal(grid, np.round(grid))               # 24-bit values
    assert abs(xs.mean()) < 4 * np.sqrt(1 / 12 / n)           # mean 0
    assert abs(xs.var() - 1 / 12) < 0.01 / 12                  # variance 1/12
    assert abs(np.corrcoef(xs[:-1], xs[1:])[0, 1]) < 4 / np.sqrt(n)
    h, _ = np.histogram(xs, bins=16, range=(-0.5, 0.5))
    assert (np.abs(h - n / 16) < 5 * np.sqrt(n / 16)).all()


def test_noise_variate_depends_on_seed_step_and_counter():
    a = oracle.noise(1, 2, 3)
    assert a == oracle.noise(1, 2, 3)
    assert len({a, oracle.noise(2, 2, 3), oracle.noise(1, 3, 3), oracle.noise(1, 2, 4)}) == 4


def _interior_cell(prob, phi_a, phi_b, lo=0.05):
    # a cell whose phases are all strictly inside (0, 1), before and after
    # one step with and without noise (no clamping by the projection)
    ok = np.ones(prob.phi0.shape[1:], bool)
    for f in (prob.phi0, phi_a, phi_b):
        ok &= (f > lo).all(axis=0) & (f < 1 - lo).all(axis=0)
    idx = np.argwhere(ok)
    assert len(idx), "no interior cell"
    return tuple(idx[len(idx) // 2])


@pytest.mark.parametrize("step0,z_origin", [(0, 0), (11, 5)])
def test_noise_enters_as_projected_rate_increment(step0, z_origin):
    # simplex projection of an interior point: phi = v - (sum v - 1) / N, so
    # the noise changes phi_a by dt amp (xi_a - mean_b xi_b)
    p = W.small_multiphase(n=14, dim=3, N=3, NM=2, nx=16, ny=13, nz=12)
    amp, seed = 0.02, 99
    base = oracle.run(p, p.phi0, p.mu0, 1, step0=step0, z_origin=z_origin)
    nz = oracle.run(p, p.phi0, p.mu0, 1, step0=step0, z_origin=z_origin, noise_amp=amp, noise_seed=seed)
    z, y, x = _interior_cell(p, base[0], nz[0])
    gcell = x + p.nx * (y + p.ny * (z + z_origin))
    xi = np.array([oracle.noise(seed, step0, gcell * 3 + a) for a in range(3)])
    expect = p.dt * amp * (xi - xi.mean())
    got = nz[0][:, z, y, x] - base[0][:, z, y, x]
    np.testing.assert_allclose(got, expect, rtol=1e-9, atol=1e-15)


def test_noise_leaves_pure_cells_and_sum_alone():
    p = W.binary_problem("n", 24, dim=3, R=6.0, nz=20)
    a = oracle.run(p, p.phi0, p.mu0, 3)
    b = oracle.run(p, p.phi0, p.mu0, 3, noise_amp=0.05, noise_seed=3)
    pure = (p.phi0 == 1.0).any(axis=0)
    far = pure.copy()
    for ax in (0, 1, 2):      # pure with a pure neighbourhood three cells wide
        for s in (-3, -2, -1, 1, 2, 3):
            far &= np.roll(pure, s, axis=ax)
    assert far.any()
    assert np.array_equal(a[0][:, far], b[0][:, far])
    assert np.abs(b[0].sum(axis=0) - 1).max() < 1e-13
    assert np.abs(b[0] - a[0]).max() > 0


def test_shift_definition():
    rng = np.random.default_rng(0)
    phi = rng.random((3, 6, 5, 4))
    mu = rng.random((2, 6, 5, 4))
    p2, m2 = oracle.shift(3, phi, mu, 2, [0.3, -0.4])
    assert np.array_equal(p2[:, :4], phi[:, 2:]) and np.array_equal(m2[:, :4], mu[:, 2:])
    assert (p2[:2, 4:] == 0).all() and (p2[2, 4:] == 1).all()
    assert (m2[0, 4:] == 0.3).all() and (m2[1, 4:] == -0.4).all()
    q2, n2 = oracle.shift(2, phi[:, :1], mu[:, :1], 1, [0.3, -0.4])   # 2-D: along y
    assert np.array_equal(q2[:, :, :4], phi[:, :1, 1:]) and (q2[2, :, 4:] == 1).all()


@pytest.mark.parametrize("dx", [1.0, 0.5])
def test_lab_origin_equals_moved_temperature_field(dx):
    """A grid whose first cell is lab cell s sees the temperature field moved
    by s dx (at a spacing other than 1 too)."""
    p = W.eutectic_3d(n=24, steps=5)
    p = p.copy(dx=dx, dt=p.dt * dx * dx)
    p.nz = 20
    p.phi0, p.mu0 = p.phi0[:, :20], p.mu0[:, :20]
    s = 4
    a = oracle.run(p, p.phi0, p.mu0, 2, z_origin=s)
    b = oracle.run(p, p.phi0, p.mu0, 2, z0=p.z0 - s * p.dx)
    assert max(np.abs(a[0] - b[0]).max(), np.abs(a[1] - b[1]).max()) < 1e-12


def test_shift_commutes_with_a_step_on_a_z_uniform_base():
    # isothermal directional state: lamellae uniform along z up to the front,
    # uniform liquid at mu_fill above it; no-flux z
    p = W.eutectic_3d(n=24, steps=5)
    p.nz = 24
    p.G = 0.0
    lam = p.phi0[:, :1].copy()            # the bottom plane's lamellae, repeated up to z = 11
    phi = np.repeat(lam, 24, axis=1)
    phi[:, 12:] = 0.0
    phi[2, 12:] = 1.0
    mu = np.repeat(p.mu0[:, :1], 24, axis=1)
    mu_fill = p.mu0[:, -1, 0, 0]
    mu[:, 12:] = mu_fill[:, None, None, None]
    k = 3
    a = oracle.run(p, phi, mu, 1)
    a = oracle.shift(3, a[0], a[1], k, mu_fill)
    sp, sm = oracle.shift(3, phi, mu, k, mu_fill)
    b = oracle.run(p, sp, sm, 1, z_origin=k)
    # the far end differs: one holds liquid stepped once, the other fresh liquid
    top = 24 - k - 2
    assert np.array_equal(a[0][:, :top], b[0][:, :top]) and np.array_equal(a[1][:, :top], b[1][:, :top])
