"""Parity at the workloads' own step counts, through the C ABI:

* the 3-D directional eutectic recipe (lamellae of seeded widths 8-24 in the
  bottom 20 planes, pulled frozen gradient, no-flux z, periodic x/y,
  anisotropic solid-liquid pairs) at 64^3 for its full 2000 steps in FP32,
  in the split launch the benchmark selects, element by element against the
  FP64 oracle;
* the 2-D 256^2 well-potential adjoint workload's 2000-step forward run in
  FP32 and FP64 against the oracle;
* the torch.autograd.Function over the steps (GPSteps): .backward() equals
  ms_grad and central finite differences.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def _split_launch(sim, tx=128, ty=6, zchunk=12):
    tiles = sim.tiles()
    want = [i for i, t in enumerate(tiles) if t[2] == 1 and t[0] == tx and t[1] == ty]
    if not want:
        want = [i for i, t in enumerate(tiles) if t[2] == 1]
    sim.set_launch(want[0], zchunk)


def test_eutectic_recipe_64_cubed_full_2000_steps_fp32():
    from paper_2404_01035_gb300 import Simulation
    p = W.eutectic_3d(n=64, steps=2000)
    steps = 2000
    sim = Simulation(p, dtype="f32")
    _split_launch(sim)
    sim.set_fields(p.phi0, p.mu0)
    m0 = sim.diag()["mass"]
    sim.step(steps)
    m1 = sim.diag()["mass"]
    phi, mu = sim.get_fields()
    sim.close()
    ophi, omu = oracle.run(p, p.phi0, p.mu0, steps)
    dphi = np.abs(phi.astype(np.float64) - ophi).max()
    dmu = np.abs(mu.astype(np.float64) - omu).max()
    assert dphi <= 1e-3 and dmu <= 1e-3, (dphi, dmu)
    # the run is not trivial: the interfaces moved
    assert np.abs(ophi - p.phi0).max() > 0.5
    np.testing.assert_allclose(m1, m0, rtol=1e-5)


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-10), ("f32", 1e-3)])
def test_adjoint_workload_forward_2000_steps(dtype, tol):
    from paper_2404_01035_gb300 import Simulation
    p = W.adjoint_well_2d(n=256, steps=2000, delta=0.02, mob=0.8)
    steps = 2000
    sim = Simulation(p, dtype=dtype)
    sim.set_fields(p.phi0, p.mu0)
    sim.step(steps)
    phi, mu = sim.get_fields()
    sim.close()
    ophi, omu = oracle.run(p, p.phi0, p.mu0, steps)
    err = max(np.abs(phi.astype(np.float64) - ophi).max(), np.abs(mu.astype(np.float64) - omu).max())
    assert err <= tol, err
    assert np.abs(ophi - p.phi0).max() > 0.1


def test_autograd_function_backward_matches_ms_grad_and_finite_differences():
    import torch
    from paper_2404_01035_gb300 import Simulation
    from paper_2404_01035_gb300.autograd import GPSteps, overrides_of, theta_of
    n, steps, every = 48, 120, 40
    target = W.adjoint_well_2d(n=n, steps=steps, delta=0.03, mob=1.0)
    t = Simulation(target, dtype="f64")
    t.set_fields(target.phi0, target.mu0)
    t.step(steps)
    phi_hat = torch.tensor(t.get_fields()[0], device="cuda")
    t.close()
    p = W.adjoint_well_2d(n=n, steps=steps, delta=0.02, mob=0.8)
    sim = Simulation(p, dtype="f64")
    theta0 = theta_of(p)

    def loss(theta, phi0, mu0):
        phi, _ = GPSteps.apply(phi0, mu0, theta, sim, steps, every)
        return 0.5 * ((phi - phi_hat) ** 2).sum()

    theta = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    phi0 = torch.tensor(p.phi0, device="cuda", requires_grad=True)
    mu0 = torch.tensor(p.mu0, device="cuda", requires_grad=True)
    L = loss(theta, phi0, mu0)
    L.backward()
    g_theta = theta.grad.numpy()
    g_phi0 = phi0.grad.cpu().numpy()
    assert mu0.grad is not None and mu0.grad.shape == mu0.shape
    # the same gradient straight from ms_grad
    ref = Simulation(p, dtype="f64")
    ref.set_fields(p.phi0, p.mu0)
    ref.enable_checkpoints(every)
    ref.step(steps)
    phiT = torch.tensor(ref.get_fields()[0], device="cuda")
    dparams, dphi0, _ = ref.grad(phiT - phi_hat)
    ref.close()
    np.testing.assert_allclose(g_theta, dparams, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(g_phi0, dphi0.cpu().numpy(), rtol=0, atol=1e-13)
    # central differences (FP64) on delta, 1/tau, D^liq and a direction in phi0
    h = 1e-4

    def loss_at(theta_np, phi0_np):
        with torch.no_grad():
            return float(loss(torch.tensor(theta_np), torch.tensor(phi0_np, device="cuda"),
                              torch.tensor(p.mu0, device="cuda")))

    for k in (0, 1, 3):
        e = np.zeros_like(theta0)
        e[k] = h
        fd = (loss_at(theta0 + e, p.phi0) - loss_at(theta0 - e, p.phi0)) / (2 * h)
        assert g_theta[k] == pytest.approx(fd, rel=1e-5), (k, g_theta[k], fd)
    rng = np.random.default_rng(11)
    inter = (p.phi0[0] > 0.01) & (p.phi0[0] < 0.99)
    v = np.zeros_like(p.phi0)
    v[0] = rng.normal(size=inter.shape) * inter
    v[1] = -v[0]
    fd = (loss_at(theta0, p.phi0 + h * v) - loss_at(theta0, p.phi0 - h * v)) / (2 * h)
    assert (g_phi0 * v).sum() == pytest.approx(fd, rel=1e-5)
    sim.close()
