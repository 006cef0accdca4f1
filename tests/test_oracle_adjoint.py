"""The oracle's reverse adjoint (a tape recorded over each step and swept
backwards) against its forward-mode tangent (dot-product test: <lambda, J v>
from the tangent equals <J^T lambda, v> from the reverse sweep) and against
central finite differences of the plain FP64 step, which neither of the
two derivative modes shares."""
import numpy as np
import pytest

import oracle
import workloads as W


def _problems():
    yield W.binary_problem("adj_well", 20, delta=0.02, Delta=0.2, R=5.0, potential="well", ny=18, tau=1.25,
                           dt=0.2 * 0.25 / 1.45), 12
    yield W.binary_problem("adj_ob", 18, delta=0.03, Delta=0.2, R=5.0, potential="obstacle", ny=16,
                           bc=[W.BC_NOFLUX, W.BC_PERIODIC, W.BC_PERIODIC]), 10
    yield W.small_multiphase(n=12, dim=2, N=3, NM=2, nx=14, ny=12, rotate=True), 6
    yield W.binary_problem("adj3", 8, dim=3, delta=0.03, R=3.0, potential="well", ny=7, nz=6,
                           bc=[W.BC_PERIODIC, W.BC_NOFLUX, W.BC_PERIODIC]), 5
    # a grid spacing of one half (dt scaled with dx^2)
    q = W.small_multiphase(n=12, dim=2, N=3, NM=2, nx=14, ny=12, rotate=True)
    yield q.copy(dx=0.5, dt=q.dt * 0.25), 6


@pytest.mark.parametrize("case", range(5))
def test_reverse_sweep_equals_the_tangent(case):
    p, steps = list(_problems())[case]
    N, NM = p.n_phases, p.n_components - 1
    rng = np.random.default_rng(case)
    lp = rng.normal(size=p.phi0.shape)
    lm = rng.normal(size=p.mu0.shape)
    dphi0, dmu0, dth = oracle.run_adjoint(p, p.phi0, p.mu0, steps, lp, lm)
    vp = rng.normal(size=p.phi0.shape)
    vm = rng.normal(size=p.mu0.shape)
    P = N * (N - 1) // 2
    vt = rng.normal(size=P + 1 + N * NM * NM)
    dd = np.zeros((N, N))
    k = 0
    for a in range(N):
        for b in range(a + 1, N):
            dd[a, b] = vt[k]
            k += 1
    _, _, tphi, tmu = oracle.run_tangent(p, p.phi0, p.mu0, steps, dphi0=vp, dmu0=vm, ddelta=dd, dmob=vt[P],
                                         dD=vt[P + 1:].reshape(N, NM, NM))
    lhs = (lp * tphi).sum() + (lm * tmu).sum()
    rhs = (dphi0 * vp).sum() + (dmu0 * vm).sum() + (dth * vt).sum()
    assert rhs == pytest.approx(lhs, rel=1e-12)


def test_reverse_sweep_matches_central_differences():
    p, steps = next(_problems())
    rng = np.random.default_rng(7)
    lp = rng.normal(size=p.phi0.shape)
    lm = rng.normal(size=p.mu0.shape)
    _, _, dth = oracle.run_adjoint(p, p.phi0, p.mu0, steps, lp, lm)

    def loss(**ov):
        phi, mu = oracle.run(p, p.phi0, p.mu0, steps, **ov)
        return (lp * phi).sum() + (lm * mu).sum()

    h = 1e-5
    d = p.delta[0, 1]
    dl = lambda s: np.array([[0, d + s], [d + s, 0]])
    fd = (loss(delta=dl(h)) - loss(delta=dl(-h))) / (2 * h)
    assert dth[0] == pytest.approx(fd, rel=1e-6)
    mob = 1.0 / p.tau
    fd = (loss(tau=1 / (mob + h)) - loss(tau=1 / (mob - h))) / (2 * h)
    assert dth[1] == pytest.approx(fd, rel=1e-6)
