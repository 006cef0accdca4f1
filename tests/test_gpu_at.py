"""GPU anti-trapping current (Eq. jatr) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import pick_cells, windowed_one_step

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_TOL = 1e-3


def _run(prob, steps, dtype, split=False, zchunk=16):
    from paper_2404_01035_gb300 import Simulation
    sim = Simulation(prob, dtype=dtype)
    if split:
        tiles = sim.tiles()
        sim.set_launch([i for i, t in enumerate(tiles) if t[2] == 1][0], zchunk)
    sim.set_fields(prob.phi0, prob.mu0)
    sim.step(steps)
    phi, mu = sim.get_fields()
    sim.close()
    return phi.astype(np.float64), mu.astype(np.float64)


def _err(a, b):
    return max(np.abs(a[0] - b[0]).max(), np.abs(a[1] - b[1]).max())


def _at(p):
    p.anti_trapping = 1
    return p


@pytest.mark.parametrize("bc", [[3, 3, 3], [3, 1, 1]])
def test_3d_multiphase_fp64(bc):
    p = _at(W.small_multiphase(n=14, dim=3, N=3, NM=2, nx=30, ny=17, nz=15, bc=bc))
    g = _run(p, 20, "f64")
    o = oracle.run(p, p.phi0, p.mu0, 20)
    assert _err(g, o) <= FP64_TOL
    # and the current did act
    off = oracle.run(p, p.phi0, p.mu0, 20, anti_trapping=0)
    assert _err(off, o) > 1e-5


@pytest.mark.parametrize("split", [False, True])
def test_grid_spacing_other_than_one(split):
    # dx = 1/2 (interface width in cells held, dt ~ dx^2): the current's face
    # gradients, rates and divergence against the oracle, FP64 fused and the
    # FP32 split step (whose work list the interface kernel fills)
    p = _at(W.small_multiphase(n=14, dim=3, N=3, NM=2, nx=30, ny=17, nz=15, bc=[3, 1, 1]))
    p = p.copy(dx=0.5, dt=0.25 * p.dt, eps=0.5 * p.eps)
    g = _run(p, 40 if split else 20, "f32" if split else "f64", split=split)
    o = oracle.run(p, p.phi0, p.mu0, 40 if split else 20)
    assert _err(g, o) <= (FP32_TOL if split else FP64_TOL)
    off = oracle.run(p, p.phi0, p.mu0, 40 if split else 20, anti_trapping=0)
    assert _err(off, o) > 1e-5


@pytest.mark.parametrize("potential", ["obstacle", "well"])
def test_2d_binary_seed_fp64(potential):
    p = _at(W.binary_problem("at2d", 48, dim=2, R=8.0, potential=potential, bc=[1, 1, 1]))
    g = _run(p, 200, "f64")
    o = oracle.run(p, p.phi0, p.mu0, 200)
    assert _err(g, o) <= FP64_TOL


def test_2d_multiphase_fp32():
    p = _at(W.small_multiphase(n=30, dim=2, N=3, NM=2, nx=70, ny=45))
    g = _run(p, 300, "f32")
    o = oracle.run(p, p.phi0, p.mu0, 300)
    assert _err(g, o) <= FP32_TOL


@pytest.mark.parametrize("zchunk", [5, 16])
def test_3d_split_fp32(zchunk):
    # the split step (bulk stream + interface kernel), then the correction
    p = _at(W.eutectic_3d(n=48, steps=10))
    p.nz = 40
    p.phi0, p.mu0 = p.phi0[:, :40], p.mu0[:, :40]
    g = _run(p, 200, "f32", split=True, zchunk=zchunk)
    o = oracle.run(p, p.phi0, p.mu0, 200)
    assert _err(g, o) <= FP32_TOL


def test_3d_eight_phases_fp32():
    p = _at(W.multigrain_3d(n=40, grains=7, R=5.0, min_sep=14.0, seed=3))
    g = _run(p, 100, "f32", split=True)
    o = oracle.run(p, p.phi0, p.mu0, 100)
    assert _err(g, o) <= FP32_TOL


def test_refused_by_the_adjoint_the_batch_and_halo_faces():
    from paper_2404_01035_gb300 import Simulation
    from paper_2404_01035_gb300.batch import Batch
    p = _at(W.binary_problem("at_ref", 32, dim=2, R=6.0))
    sim = Simulation(p, dtype="f64")
    with pytest.raises(Exception):
        sim.enable_checkpoints(5)
    sim.close()
    with pytest.raises(Exception):
        Batch([p])
    q = _at(W.small_multiphase(n=12, dim=3, N=3, NM=2, nx=16, ny=12, nz=10, bc=[3, 3, 16]))
    with pytest.raises(Exception):
        Simulation(q, dtype="f64")


def test_eutectic_3d_full_size_sampled_one_step_fp32():
    # 256^3 eutectic in the tuned launch, 300 steps with the current, then one
    # step checked at sampled cells (random, interface, corners) against the
    # oracle on a window (radius 3: mu needs phi^{n+1} of the neighbours)
    from paper_2404_01035_gb300 import Simulation
    p = _at(W.eutectic_3d())
    rng = np.random.default_rng(5)
    sim = Simulation(p, dtype="f32")
    sim.set_fields(p.phi0, p.mu0)
    sim.tune(None, steps_per_trial=5)
    sim.set_fields(p.phi0, p.mu0)
    sim.step(300)
    phi_n, mu_n = sim.get_fields()
    t_n = sim.time()[1]
    sim.step(1)
    phi_1, mu_1 = sim.get_fields()
    sim.close()
    cells = pick_cells(phi_n, rng)
    ophi, omu = windowed_one_step(p, phi_n, mu_n, cells, t0=t_n, r=3)
    gphi = np.array([phi_1[:, z, y, x] for (z, y, x) in cells])
    gmu = np.array([mu_1[:, z, y, x] for (z, y, x) in cells])
    assert np.abs(gphi - ophi).max() <= 2e-5
    assert np.abs(gmu - omu).max() <= 2e-5
