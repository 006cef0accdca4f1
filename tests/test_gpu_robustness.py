"""Failure paths through the C ABI, without any device fault: a device
allocation refused by the caller's allocator while elasticity is turned on,
the adjoint recording rules of ms_update_params, a non-finite state loaded
from the host, the bounded-wait self-test, and host-side fault injection."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def _flaky_allocator():
    from paper_2404_01035_gb300._binding import TorchAllocator

    class Flaky(TorchAllocator):
        refuse = False

        def _do_alloc(self, nbytes, user):
            if self.refuse:
                return None
            return super()._do_alloc(nbytes, user)

    return Flaky()


def _cubic(c11=150.0, c12=60.0, c44=75.0):
    C = np.zeros((6, 6))
    C[:3, :3] = c12
    np.fill_diagonal(C[:3, :3], c11)
    C[3, 3] = C[4, 4] = C[5, 5] = c44
    return C


def _err(a, b):
    return max(np.abs(a[0] - b[0]).max(), np.abs(a[1] - b[1]).max())


def test_failed_elasticity_setup_keeps_the_previous_parameters():
    from paper_2404_01035_gb300 import Simulation
    from paper_2404_01035_gb300._binding import MSError
    p = W.small_multiphase(n=16, dim=2, N=3, NM=2, nx=32, ny=24, bc=[3, 3, 3])
    rng = np.random.default_rng(4)
    e = rng.normal(scale=0.01, size=(3, 3, 3))
    e = 0.5 * (e + np.transpose(e, (0, 2, 1)))
    e[-1] = 0.0
    alloc = _flaky_allocator()
    sim = Simulation(p, dtype="f64", allocator=alloc)
    sim.set_fields(p.phi0, p.mu0)
    sim.step(4)
    alloc.refuse = True
    with pytest.raises(MSError) as ex:
        sim.update_params(elastic_C=_cubic(), eigenstrain=e)
    assert ex.value.status == 3           # MS_ERR_OOM, nothing committed
    alloc.refuse = False
    sim.step(4)                           # runs with the old parameters (no elasticity)
    g = sim.get_fields()
    o = oracle.run(p, p.phi0, p.mu0, 8)
    assert _err(g, o) <= 1e-10
    # a later successful update turns elasticity on
    sim.update_params(elastic_C=_cubic(), eigenstrain=e)
    sim.step(3)
    g = sim.get_fields()
    sim.close()
    pe = p.copy(elastic_C=_cubic(), eigenstrain=e)
    o = oracle.run(pe, o[0], o[1], 3, t0=8 * p.dt, step0=8)
    assert _err(g, o) <= 1e-10


def test_update_params_while_recording_refuses_extensions_and_restarts_the_recording():
    import torch
    from paper_2404_01035_gb300 import Simulation
    from paper_2404_01035_gb300._binding import MSError
    p = W.binary_problem("rec", 32, delta=0.03, Delta=0.2, R=7.0, potential="well", ny=28)
    sim = Simulation(p, dtype="f64")
    sim.set_fields(p.phi0, p.mu0)
    sim.enable_checkpoints(4)
    for bad in ({"noise_amp": 0.01}, {"anti_trapping": 1}, {"grain_growth": 1}):
        with pytest.raises(MSError) as ex:
            sim.update_params(**bad)
        assert ex.value.status == 9
    sim.step(6)
    sim.update_params(tau=1.1)            # the recording restarts here
    sim.step(6)
    lam = torch.tensor(np.random.default_rng(9).normal(size=p.phi0.shape), device="cuda")
    dA, phiA, _ = sim.grad(lam)
    sim.close()
    # the same 6 steps recorded from the state at the update
    ref = Simulation(p, dtype="f64")
    ref.set_fields(p.phi0, p.mu0)
    ref.step(6)
    mid = ref.get_fields()
    ref.close()
    rb = Simulation(p, dtype="f64", tau=1.1)
    rb.set_fields(*mid)
    rb.enable_checkpoints(4)
    rb.step(6)
    dB, phiB, _ = rb.grad(lam)
    rb.close()
    np.testing.assert_allclose(dA, dB, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(phiA.cpu().numpy(), phiB.cpu().numpy(), rtol=0, atol=1e-13)


def test_adjoint_is_refused_on_a_slab_with_halo_faces():
    # the reverse step maps ghost positions back to their cells by the
    # boundary rule, which a halo face does not have: refused, not wrong
    from paper_2404_01035_gb300 import Simulation
    from paper_2404_01035_gb300._binding import MS_BC_HALO, MSError
    p = W.binary_problem("slab", 8, dim=3, delta=0.03, R=3.0, potential="well", ny=7, nz=6,
                         bc=[W.BC_PERIODIC, W.BC_PERIODIC, MS_BC_HALO])
    sim = Simulation(p, dtype="f64")
    with pytest.raises(MSError) as ex:
        sim.enable_checkpoints(4)
    assert ex.value.status == 9 and "halo" in str(ex.value)
    sim.close()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_non_finite_state_is_reported(dtype):
    from paper_2404_01035_gb300 import Simulation
    from paper_2404_01035_gb300._binding import MSError
    p = W.small_multiphase(n=12, dim=3, N=3, NM=2)
    phi = p.phi0.copy()
    phi[1, 3, 4, 5] = np.nan
    sim = Simulation(p, dtype=dtype)
    sim.set_fields(phi, p.mu0)
    sim.sync()                            # nothing has looked at the state yet
    with pytest.raises(MSError) as ex:
        sim.diag()
    assert ex.value.status == 5           # MS_ERR_NONFINITE
    with pytest.raises(MSError) as ex:
        sim.sync()                        # sticky
    assert ex.value.status == 5
    sim.close()
    # the periodic diagnostics inside ms_step find it too
    sim = Simulation(p, dtype=dtype)
    sim.set_fields(p.phi0, p.mu0)
    sim.set_diag_every(2)
    sim.step(4)
    sim.sync()                            # a finite run stays clean
    mu = p.mu0.copy()
    mu[0, 0, 0, 0] = np.inf
    sim.set_fields(p.phi0, mu)
    sim.step(2)
    with pytest.raises(MSError) as ex:
        sim.sync()
    assert ex.value.status == 5
    sim.close()


def test_bounded_wait_gives_up_and_the_device_stays_usable():
    from paper_2404_01035_gb300 import Simulation
    from paper_2404_01035_gb300._binding import MSError
    p = W.small_multiphase(n=12, dim=2, N=3, NM=2, nx=20, ny=18)
    sim = Simulation(p, dtype="f64")
    sim.set_fields(p.phi0, p.mu0)
    sim.sync()
    with pytest.raises(MSError):
        sim.selftest_timeout(10)          # below the accepted range
    sim.selftest_timeout(2_000_000)       # 2 ms
    with pytest.raises(MSError) as ex:
        sim.sync()
    assert ex.value.status == 6           # MS_ERR_TIMEOUT
    with pytest.raises(MSError) as ex:
        sim.sync()                        # sticky
    assert ex.value.status == 6
    sim.close()
    # another context on the same device steps as before
    other = Simulation(p, dtype="f64")
    other.set_fields(p.phi0, p.mu0)
    other.step(10)
    other.sync()
    g = other.get_fields()
    other.close()
    assert _err(g, oracle.run(p, p.phi0, p.mu0, 10)) <= 1e-10


def test_injected_fault_stops_the_step_loop(monkeypatch):
    from paper_2404_01035_gb300 import Simulation
    from paper_2404_01035_gb300._binding import MSError
    p = W.small_multiphase(n=12, dim=2, N=3, NM=2, nx=20, ny=18)
    monkeypatch.setenv("MS_FAULT", "step:5,code:6")
    sim = Simulation(p, dtype="f64")
    monkeypatch.delenv("MS_FAULT")
    sim.set_fields(p.phi0, p.mu0)
    with pytest.raises(MSError) as ex:
        sim.step(10)
    assert ex.value.status == 6
    assert sim.time()[0] == 5             # steps 0..4 ran, step 5 was refused
    g = sim.get_fields()
    assert _err(g, oracle.run(p, p.phi0, p.mu0, 5)) <= 1e-10
    for call in (lambda: sim.step(1), sim.sync):
        with pytest.raises(MSError) as ex:
            call()
        assert ex.value.status == 6
    sim.close()
