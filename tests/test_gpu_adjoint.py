"""GPU discrete adjoint (ms_grad) against the oracle's forward-mode tangent
(dot-product test, FP64), and against central finite differences and the
FP32 build on the 2-D 256^2 well-potential adjoint workload."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def _adjoint(prob, steps, every, lam_phi, lam_mu, dtype="f64"):
    import torch
    from paper_2404_01035_gb300 import Simulation
    sim = Simulation(prob, dtype=dtype)
    sim.set_fields(prob.phi0, prob.mu0)
    sim.enable_checkpoints(every)
    sim.step(steps)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    dparams, dphi0, dmu0 = sim.grad(torch.tensor(lam_phi, dtype=tdt, device="cuda"),
                                    torch.tensor(lam_mu, dtype=tdt, device="cuda"))
    phi_T, _ = sim.get_fields()
    sim.close()
    return dparams, dphi0.cpu().numpy(), dmu0.cpu().numpy(), phi_T


def _dot_product_check(prob, steps, every, seed):
    rng = np.random.default_rng(seed)
    N, NM = prob.n_phases, prob.n_components - 1
    lam_phi = rng.normal(size=prob.phi0.shape)
    lam_mu = rng.normal(size=prob.mu0.shape)
    dparams, dphi0, dmu0, _ = _adjoint(prob, steps, every, lam_phi, lam_mu)
    # direction in (phi0, mu0, theta)
    v_phi = rng.normal(size=prob.phi0.shape)
    v_mu = rng.normal(size=prob.mu0.shape)
    P = N * (N - 1) // 2
    v_theta = rng.normal(size=P + 1 + N * NM * NM)
    dd = np.zeros((N, N))
    k = 0
    for a in range(N):
        for b in range(a + 1, N):
            dd[a, b] = v_theta[k]
            k += 1
    _, _, tphi, tmu = oracle.run_tangent(prob, prob.phi0, prob.mu0, steps, dphi0=v_phi, dmu0=v_mu,
                                         ddelta=dd, dmob=v_theta[P],
                                         dD=v_theta[P + 1:].reshape(N, NM, NM))
    lhs = (lam_phi * tphi).sum() + (lam_mu * tmu).sum()
    rhs = (dphi0 * v_phi).sum() + (dmu0 * v_mu).sum() + (dparams * v_theta).sum()
    assert rhs == pytest.approx(lhs, rel=1e-9), (lhs, rhs)
    # parameter gradients one by one against single-parameter tangents
    for k in range(P + 1):
        e = np.zeros_like(v_theta)
        e[k] = 1.0
        dd = np.zeros((N, N))
        if k < P:
            a, b = [(a, b) for a in range(N) for b in range(a + 1, N)][k]
            dd[a, b] = 1.0
        _, _, tphi, tmu = oracle.run_tangent(prob, prob.phi0, prob.mu0, steps, ddelta=dd,
                                             dmob=1.0 if k == P else 0.0)
        ref = (lam_phi * tphi).sum() + (lam_mu * tmu).sum()
        assert dparams[k] == pytest.approx(ref, rel=1e-9, abs=1e-12)


def test_adjoint_2d_binary_well_matches_oracle_tangent():
    p = W.binary_problem("adj", 40, delta=0.02, Delta=0.2, R=8.0, potential="well", ny=36,
                         tau=1.25, dt=0.2 * 0.25 / 1.45)
    _dot_product_check(p, steps=90, every=25, seed=1)


def test_adjoint_2d_binary_obstacle_noflux_matches_oracle_tangent():
    p = W.binary_problem("adj_ob", 34, delta=0.03, Delta=0.2, R=7.0, potential="obstacle", ny=30,
                         bc=[W.BC_NOFLUX, W.BC_PERIODIC, W.BC_PERIODIC])
    _dot_product_check(p, steps=40, every=16, seed=2)


def test_adjoint_2d_three_phase_ternary_matches_oracle_tangent():
    p = W.small_multiphase(n=20, dim=2, N=3, NM=2, nx=26, ny=21, rotate=True)
    _dot_product_check(p, steps=24, every=10, seed=3)


def test_adjoint_at_a_grid_spacing_of_one_half():
    # the reverse passes' face gradients, divergences and mu flux at dx = 1/2
    p = W.binary_problem("adjdx", 24, delta=0.02, Delta=0.2, R=6.0, potential="well", ny=20,
                         tau=1.25, dt=0.2 * 0.25 / 1.45)
    p = p.copy(dx=0.5, dt=0.25 * p.dt, eps=0.5 * p.eps)
    _dot_product_check(p, 12, 5, seed=17)


def test_adjoint_3d_binary_matches_oracle_tangent():
    p = W.binary_problem("adj3", 14, dim=3, delta=0.03, R=4.0, potential="well", ny=12, nz=11,
                         bc=[W.BC_PERIODIC, W.BC_NOFLUX, W.BC_PERIODIC])
    _dot_product_check(p, steps=12, every=5, seed=4)


# ---------------------------------------------------- the 256^2 adjoint workload
def _adjoint_well_2d_setup(dtype, n=256, steps=2000):
    import torch
    from paper_2404_01035_gb300 import Simulation
    target = W.adjoint_well_2d(n=n, steps=steps, delta=0.03, mob=1.0)
    sim = Simulation(target, dtype="f64")
    sim.set_fields(target.phi0, target.mu0)
    sim.step(steps)
    phi_hat, _ = sim.get_fields()
    sim.close()
    evalp = W.adjoint_well_2d(n=n, steps=steps, delta=0.02, mob=0.8)
    return evalp, phi_hat


def _loss(prob, phi_hat, steps, dtype="f64", phi0=None, **override):
    from paper_2404_01035_gb300 import Simulation
    sim = Simulation(prob, dtype=dtype, **override)
    sim.set_fields(prob.phi0 if phi0 is None else phi0, prob.mu0)
    sim.step(steps)
    phi, _ = sim.get_fields()
    sim.close()
    return 0.5 * ((phi.astype(np.float64) - phi_hat) ** 2).sum()


def _adjoint_well_2d_grad(prob, phi_hat, steps, dtype):
    import torch
    from paper_2404_01035_gb300 import Simulation
    sim = Simulation(prob, dtype=dtype)
    sim.set_fields(prob.phi0, prob.mu0)
    sim.enable_checkpoints(prob.meta["ckpt_every"])
    sim.step(steps)
    phi, _ = sim.get_fields()
    tdt = torch.float64 if dtype == "f64" else torch.float32
    dparams, dphi0, _ = sim.grad(torch.tensor(phi.astype(np.float64) - phi_hat, dtype=tdt, device="cuda"))
    sim.close()
    return dparams, dphi0.cpu().numpy()


def test_adjoint_well_2d_gradients_match_central_differences_and_fp32():
    steps = 2000
    prob, phi_hat = _adjoint_well_2d_setup("f64", steps=steps)
    g64, dphi0 = _adjoint_well_2d_grad(prob, phi_hat, steps, "f64")
    h = 1e-4
    d = prob.delta[0, 1]
    dl = lambda s: np.array([[0, d + s], [d + s, 0]])
    fd_delta = (_loss(prob, phi_hat, steps, delta=dl(h)) - _loss(prob, phi_hat, steps, delta=dl(-h))) / (2 * h)
    mob = 1.0 / prob.tau
    fd_mob = (_loss(prob, phi_hat, steps, tau=1 / (mob + h)) -
              _loss(prob, phi_hat, steps, tau=1 / (mob - h))) / (2 * h)
    Dl = prob.D.copy()
    Dp, Dm = Dl.copy(), Dl.copy()
    Dp[1, 0, 0] += h
    Dm[1, 0, 0] -= h
    fd_D = (_loss(prob, phi_hat, steps, D=Dp) - _loss(prob, phi_hat, steps, D=Dm)) / (2 * h)
    assert g64[0] == pytest.approx(fd_delta, rel=1e-5)
    assert g64[1] == pytest.approx(fd_mob, rel=1e-5)
    assert g64[3] == pytest.approx(fd_D, rel=1e-5)
    # directional derivative w.r.t. phi0 inside the interface (0.01 < phi < 0.99)
    rng = np.random.default_rng(7)
    inter = (prob.phi0[0] > 0.01) & (prob.phi0[0] < 0.99)
    v = np.zeros_like(prob.phi0)
    v[0] = rng.normal(size=inter.shape) * inter
    v[1] = -v[0]
    fd_phi = (_loss(prob, phi_hat, steps, phi0=prob.phi0 + h * v) -
              _loss(prob, phi_hat, steps, phi0=prob.phi0 - h * v)) / (2 * h)
    assert (dphi0 * v).sum() == pytest.approx(fd_phi, rel=1e-5)
    # FP32 build of the same gradient
    g32, _ = _adjoint_well_2d_grad(prob, phi_hat, steps, "f32")
    for k in (0, 1, 3):
        assert g32[k] == pytest.approx(g64[k], rel=1e-2)


@pytest.mark.parametrize("case", ["well2d", "ternary2d", "binary3d", "thin2d"])
def test_gradients_equal_the_oracle_reverse_sweep(case):
    # ms_grad (FP64) against the oracle's own reverse adjoint, element by element
    if case == "well2d":
        p = W.binary_problem("adjr", 40, delta=0.02, Delta=0.2, R=8.0, potential="well", ny=36,
                             tau=1.25, dt=0.2 * 0.25 / 1.45)
        steps, every = 60, 25
    elif case == "binary3d":
        # 3-D faces and tangential neighbours, periodic and no-flux axes
        p = W.binary_problem("adjr3", 10, dim=3, delta=0.03, R=3.5, potential="well", ny=9, nz=8,
                             bc=[W.BC_PERIODIC, W.BC_NOFLUX, W.BC_PERIODIC])
        steps, every = 8, 3
    elif case == "thin2d":
        # rows of two cells along y: every cell is at both ends of that axis,
        # so its value sits at both ghost images (periodic x, no-flux y)
        p = W.binary_problem("adjt", 24, delta=0.02, Delta=0.2, R=6.0, potential="well", ny=2,
                             bc=[W.BC_PERIODIC, W.BC_NOFLUX, W.BC_PERIODIC])
        steps, every = 12, 5
    else:
        p = W.small_multiphase(n=16, dim=2, N=3, NM=2, nx=18, ny=16, rotate=True)
        steps, every = 16, 6
    rng = np.random.default_rng(21)
    lam_phi = rng.normal(size=p.phi0.shape)
    lam_mu = rng.normal(size=p.mu0.shape)
    dparams, dphi0, dmu0, _ = _adjoint(p, steps, every, lam_phi, lam_mu)
    ophi0, omu0, oth = oracle.run_adjoint(p, p.phi0, p.mu0, steps, lam_phi, lam_mu)
    np.testing.assert_allclose(dparams, oth, rtol=1e-9, atol=1e-12 * np.abs(oth).max())
    assert np.abs(dphi0 - ophi0).max() <= 1e-9 * np.abs(ophi0).max()
    assert np.abs(dmu0 - omu0).max() <= 1e-9 * np.abs(omu0).max()
