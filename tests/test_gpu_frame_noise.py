"""GPU phi noise and moving frame against the FP64 oracle (through the C ABI)."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def _sim(prob, dtype, **launch):
    from paper_2404_01035_gb300 import Simulation
    sim = Simulation(prob, dtype=dtype)
    if launch.get("split"):
        tiles = sim.tiles()
        sim.set_launch([i for i, t in enumerate(tiles) if t[2] == 1][0], 16)
    sim.set_fields(prob.phi0, prob.mu0)
    return sim


def _err(a, b):
    return max(np.abs(a[0] - b[0]).max(), np.abs(a[1] - b[1]).max())


def _noisy(p, amp=0.02, seed=4242):
    p.noise_amp, p.noise_seed = amp, seed
    return p


def test_noise_fp64_matches_oracle():
    p = _noisy(W.small_multiphase(n=14, dim=3, N=3, NM=2, nx=30, ny=17, nz=15))
    sim = _sim(p, "f64")
    sim.step(20)
    g = sim.get_fields()
    sim.close()
    o = oracle.run(p, p.phi0, p.mu0, 20)
    assert _err(g, o) <= 1e-10


@pytest.mark.parametrize("split", [False, True])
def test_noise_fp32_matches_oracle(split):
    p = _noisy(W.small_multiphase(n=20, dim=3, N=3, NM=2, nx=70, ny=37, nz=30))
    sim = _sim(p, "f32", split=split)
    sim.step(200)
    g = sim.get_fields()
    sim.close()
    o = oracle.run(p, p.phi0, p.mu0, 200)
    assert _err(g, o) <= 1e-3


def test_noise_and_lab_origin_2d_fp64():
    p = _noisy(W.small_multiphase(n=30, dim=2, N=3, NM=2, nx=40, ny=33))
    p.meta["z_origin"] = 7
    sim = _sim(p, "f64")
    sim.step(15)
    g = sim.get_fields()
    sim.close()
    o = oracle.run(p, p.phi0, p.mu0, 15, z_origin=7)
    assert _err(g, o) <= 1e-10


@pytest.mark.parametrize("dim", [3, 2])
def test_shift_then_steps_match_oracle_fp64(dim):
    if dim == 3:
        p = W.eutectic_3d(n=24, steps=10)
        p.nz = 24
        p.phi0, p.mu0 = p.phi0[:, :24], p.mu0[:, :24]
    else:
        p = W.small_multiphase(n=30, dim=2, N=3, NM=2, nx=40, ny=33)
    _noisy(p, 0.01, 17)
    mu_fill = p.mu0.reshape(p.mu0.shape[0], -1)[:, -1]
    sim = _sim(p, "f64")
    sim.step(5)
    sim.shift(3, mu_fill)
    sim.step(5)
    g = sim.get_fields()
    sim.close()
    a = oracle.run(p, p.phi0, p.mu0, 5)
    a = oracle.shift(dim, a[0], a[1], 3, mu_fill)
    o = oracle.run(p, a[0], a[1], 5, t0=5 * p.dt, step0=5, z_origin=3)
    assert _err(g, o) <= 1e-10


def test_front_and_moving_frame():
    p = W.eutectic_3d(n=32, steps=10)
    sim = _sim(p, "f32")
    phi, _ = sim.get_fields()
    solid = (phi[-1] != 1.0).any(axis=(1, 2))
    assert sim.front() == int(np.nonzero(solid)[0].max())
    mu_fill = p.mu0[:, -1, 0, 0]
    keep = sim.front() - 3
    sim.step_moving_frame(40, keep, mu_fill, check_every=20)
    assert sim.front() <= keep + 1
    phi, mu = sim.get_fields()
    assert (phi[-1, -3:] == 1.0).all()                  # fresh liquid at the far end
    assert np.abs(phi.sum(axis=0) - 1).max() < 1e-5
    sim.close()


def test_noise_is_refused_by_the_adjoint_and_the_batch():
    from paper_2404_01035_gb300 import Simulation
    from paper_2404_01035_gb300.batch import Batch
    p = _noisy(W.adjoint_well_2d(n=32, steps=10, delta=0.02, mob=1.0))
    sim = Simulation(p, dtype="f64")
    with pytest.raises(Exception):
        sim.enable_checkpoints(5)
    sim.close()
    with pytest.raises(Exception):
        Batch([p])
