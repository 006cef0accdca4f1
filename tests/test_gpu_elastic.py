"""GPU elasticity (homogeneous stiffness, FFT equilibrium before every step)
against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def _cubic(c11=150.0, c12=60.0, c44=75.0):
    C = np.zeros((6, 6))
    C[:3, :3] = c12
    np.fill_diagonal(C[:3, :3], c11)
    C[3, 3] = C[4, 4] = C[5, 5] = c44
    return C


def _elastic(p, scale=0.01, seed=5):
    rng = np.random.default_rng(seed)
    N = p.n_phases
    e = rng.normal(scale=scale, size=(N, 3, 3))
    e = 0.5 * (e + np.transpose(e, (0, 2, 1)))
    e[-1] = 0.0                         # the matrix / liquid carries none
    p.elastic_C, p.eigenstrain = _cubic(), e
    return p


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


@pytest.mark.parametrize("dim", [3, 2])
def test_fp64_matches_oracle(dim):
    p = _elastic(W.small_multiphase(n=20, dim=dim, N=3, NM=2, nx=24, ny=20, nz=18 if dim == 3 else None, bc=[3, 3, 3]))
    g = _run(p, 20, "f64")
    o = oracle.run(p, p.phi0, p.mu0, 20)
    assert _err(g, o) <= 1e-10
    off = oracle.run(p, p.phi0, p.mu0, 20, elastic_C=None)
    assert _err(off, o) > 1e-6          # the elastic force acted


def test_fp64_at_a_grid_spacing_of_one_half():
    # the FFT equilibrium and the step's own dx terms together at dx = 1/2
    p = _elastic(W.small_multiphase(n=20, dim=3, N=3, NM=2, nx=24, ny=20, nz=18, bc=[3, 3, 3]))
    p = p.copy(dx=0.5, dt=0.25 * p.dt, eps=0.5 * p.eps)
    g = _run(p, 30, "f64")
    o = oracle.run(p, p.phi0, p.mu0, 30)
    assert _err(g, o) <= 1e-10
    off = oracle.run(p, p.phi0, p.mu0, 30, elastic_C=None)
    assert _err(off, o) > 1e-6


@pytest.mark.parametrize("zchunk", [6, 16])
def test_fp32_split_matches_oracle(zchunk):
    p = _elastic(W.small_multiphase(n=24, dim=3, N=3, NM=2, nx=48, ny=40, nz=36, bc=[3, 3, 3]))
    g = _run(p, 100, "f32", split=True, zchunk=zchunk)
    o = oracle.run(p, p.phi0, p.mu0, 100)
    assert _err(g, o) <= 1e-3


def test_fp32_eight_phases():
    p = _elastic(W.multigrain_3d(n=40, grains=7, R=5.0, min_sep=14.0, seed=3))
    g = _run(p, 60, "f32", split=True)
    o = oracle.run(p, p.phi0, p.mu0, 60)
    assert _err(g, o) <= 1e-3


def test_refusals():
    from paper_2404_01035_gb300 import Simulation
    from paper_2404_01035_gb300.batch import Batch
    p = _elastic(W.binary_problem("el_ref", 32, dim=2, R=6.0))
    q = p.copy(bc=[3, 1, 1])               # the FFT equilibrium needs periodic boundaries
    with pytest.raises(Exception):
        Simulation(q, dtype="f64")
    with pytest.raises(Exception):
        Simulation(p.copy(grain_growth=1), dtype="f64")
    sim = Simulation(p, dtype="f64")
    with pytest.raises(Exception):
        sim.enable_checkpoints(5)
    sim.close()
    with pytest.raises(Exception):
        Batch([p])


def test_turning_elasticity_off_and_on_mid_run():
    from paper_2404_01035_gb300 import Simulation
    p = _elastic(W.small_multiphase(n=16, dim=2, N=3, NM=2, nx=32, ny=24, bc=[3, 3, 3]))
    sim = Simulation(p, dtype="f64")
    sim.set_fields(p.phi0, p.mu0)
    sim.step(5)
    sim.update_params(elastic_C=None)      # off: the step must stop reading the potentials
    sim.step(5)
    sim.update_params()                     # on again
    sim.step(5)
    g = sim.get_fields()
    sim.close()
    a = oracle.run(p, p.phi0, p.mu0, 5)
    a = oracle.run(p, a[0], a[1], 5, t0=5 * p.dt, step0=5, elastic_C=None)
    o = oracle.run(p, a[0], a[1], 5, t0=10 * p.dt, step0=10)
    assert _err(g, o) <= 1e-10
