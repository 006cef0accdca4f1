"""Covariance of the oracle's step under the symmetries of the grid.

Covered: axis permutations and mirrors with rotated anisotropic pairs (3-D);
periodic translations; and the no-flux boundary as the mirror-extended
periodic domain.

The model of Sec. 2 is written in lab coordinates except for the anisotropy.
The anisotropy a_c depends on each pair's interface normal in its crystal
frame, i.e. on R_ab q_ab, with R_ab the pair's rotation.  A permutation or
reflection P of the grid axes maps the lab-frame vector q to P q.  So moving
the state by P and every rotation R_ab to R_ab P^T gives the same crystal
frame normals at the moved cells.  Everything else is a scalar field or an
isotropic coefficient.  The step is therefore covariant: stepping the moved
state equals moving the stepped state, up to the rounding of sums taken in
another axis order.

The setting makes that exact.  Every axis is periodic and there is no
temperature gradient, so no axis is special.  Three phases with two solutes
and rotated anisotropic pairs are used, with and without the anti-trapping
current.  The test catches a slip that treats one axis differently from the
others: a tangential gradient taken along the wrong axis, a face divergence
that skips an axis, or a rotation applied by rows in one place and by
columns in another.
"""
import numpy as np
import pytest

import oracle
import workloads as W

STEPS = 6


def _problem(n=10):
    p = W.small_multiphase(n=n, dim=3, N=3, NM=2, rotate=True, bc=[W.BC_PERIODIC] * 3)
    p.G = 0.0
    p.V = 0.0
    return p


def _axis_matrix(perm, flip):
    """The 3x3 map of lab vector components (x, y, z) for an array move that
    transposes the spatial axes [z][y][x] by `perm` (new array axis k is old
    array axis perm[k]) and then reverses the new array axes listed in `flip`."""
    S = np.zeros((3, 3))
    for k in range(3):
        S[2 - k, 2 - perm[k]] = 1.0
    for k in flip:
        S[2 - k] *= -1.0
    return S


def _move(f, perm, flip):
    g = np.transpose(f, (0,) + tuple(1 + np.array(perm)))
    for k in flip:
        g = np.flip(g, axis=1 + k)
    return np.ascontiguousarray(g)


MOVES = [
    ((0, 2, 1), ()),        # swap x and y
    ((2, 1, 0), ()),        # swap x and z
    ((1, 2, 0), ()),        # cyclic x -> z -> y -> x
    ((0, 1, 2), (2,)),      # mirror x
    ((2, 0, 1), (0, 1)),    # a rotation of the cube with reflections
]


@pytest.mark.parametrize("at", [0, 1])
@pytest.mark.parametrize("perm,flip", MOVES)
def test_step_is_covariant_under_grid_symmetries(perm, flip, at):
    p = _problem()
    ref_phi, ref_mu = oracle.run(p, p.phi0, p.mu0, STEPS, anti_trapping=at)
    S = _axis_matrix(perm, flip)
    q = p.copy(rot=np.einsum("abij,jk->abik", p.rot, S.T))
    phi, mu = oracle.run(q, _move(p.phi0, perm, flip), _move(p.mu0, perm, flip), STEPS, anti_trapping=at)
    err = max(np.abs(phi - _move(ref_phi, perm, flip)).max(), np.abs(mu - _move(ref_mu, perm, flip)).max())
    assert err < 1e-12, err


def test_the_rotations_matter_on_this_state():
    """The rotated crystal frames change the trajectory by far more than the tolerance,
    and so does moving the state without rotating the frames along with it."""
    p = _problem()
    ref_phi, _ = oracle.run(p, p.phi0, p.mu0, STEPS)
    plain = p.copy(rot=np.broadcast_to(np.eye(3), p.rot.shape).copy())
    phi0, _ = oracle.run(plain, p.phi0, p.mu0, STEPS)
    assert np.abs(phi0 - ref_phi).max() > 1e-6
    perm, flip = MOVES[2]
    phi1, _ = oracle.run(p, _move(p.phi0, perm, flip), _move(p.mu0, perm, flip), STEPS)
    assert np.abs(phi1 - _move(ref_phi, perm, flip)).max() > 1e-6


def test_axis_matrix_moves_a_gradient_like_the_array():
    """The component map S matches the array move: the gradient of a linear-in-cells
    ramp moves as S times the gradient (checked by central differences)."""
    n = 8
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    f = (0.3 * x + 0.5 * y + 0.7 * z)[None].astype(float)    # gradient (0.3, 0.5, 0.7) in (x, y, z)
    for perm, flip in MOVES:
        g = _move(f, perm, flip)[0]
        c = n // 2
        grad = np.array([(g[c, c, c + 1] - g[c, c, c - 1]) / 2, (g[c, c + 1, c] - g[c, c - 1, c]) / 2,
                         (g[c + 1, c, c] - g[c - 1, c, c]) / 2])
        np.testing.assert_allclose(grad, _axis_matrix(perm, flip) @ np.array([0.3, 0.5, 0.7]), atol=1e-12)


@pytest.mark.parametrize("shift", [(3, 0, 0), (0, 5, 0), (0, 0, 7), (4, 9, 2)])
def test_step_commutes_with_periodic_translation(shift):
    """On a periodic grid a translation by whole cells is a symmetry: rolling the state
    rolls the trajectory (same arithmetic in the same order, so to round-off)."""
    p = _problem()
    ref_phi, ref_mu = oracle.run(p, p.phi0, p.mu0, STEPS, anti_trapping=1)
    roll = lambda f: np.ascontiguousarray(np.roll(f, shift, axis=(1, 2, 3)))
    phi, mu = oracle.run(p, roll(p.phi0), roll(p.mu0), STEPS, anti_trapping=1)
    assert max(np.abs(phi - roll(ref_phi)).max(), np.abs(mu - roll(ref_mu)).max()) < 1e-13


def _mirror_extend(f, axes):
    """Double the grid along each array axis in `axes` by appending the mirror image
    (cell 2n-1-i holds cell i)."""
    for ax in axes:
        f = np.concatenate([f, np.flip(f, axis=ax)], axis=ax)
    return np.ascontiguousarray(f)


@pytest.mark.parametrize("dim", [2, 3])
def test_no_flux_boundary_is_the_mirror_extended_periodic_domain(dim):
    """The no-flux boundary takes the ghost cell equal to the adjacent interior cell,
    i.e. zero gradient across the boundary face.  A domain of n cells with no-flux
    faces therefore steps exactly like the first half of a periodic domain of 2n cells
    that holds the state and its mirror image.  The mirror is a symmetry of the model
    there: unrotated cubic anisotropy, and no temperature gradient along the mirrored
    axes (in 3-D the pulled gradient runs along the periodic z axis and stays on).
    The anti-trapping current is on."""
    n = 10
    bc = [W.BC_NOFLUX, W.BC_NOFLUX, W.BC_PERIODIC]
    p = W.small_multiphase(n=n, dim=dim, N=3, NM=2, rotate=False, nz=8 if dim == 3 else None, bc=bc)
    if dim == 2:
        p.G = 0.0
        p.V = 0.0
    ref_phi, ref_mu = oracle.run(p, p.phi0, p.mu0, STEPS, anti_trapping=1)
    axes = (2, 3)                       # y and x of [field][z][y][x]
    big = p.copy(nx=2 * n, ny=2 * n, bc=[W.BC_PERIODIC] * 3)
    phi, mu = oracle.run(big, _mirror_extend(p.phi0, axes), _mirror_extend(p.mu0, axes), STEPS, anti_trapping=1)
    err = max(np.abs(phi[..., :n, :n] - ref_phi).max(), np.abs(mu[..., :n, :n] - ref_mu).max())
    assert err < 1e-13, err
    # the extended run keeps its mirror symmetry, and the boundary cells did change
    assert np.abs(phi - _mirror_extend(phi[..., :n, :n], axes)).max() < 1e-13
    assert np.abs(ref_phi - p.phi0)[..., [0, n - 1], :].max() > 1e-6
