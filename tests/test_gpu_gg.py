"""GPU grain growth (GRAINGROWTH = 1) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("dim,grains", [(2, 3), (2, 2), (3, 3), (3, 8)])
def test_fp64_matches_oracle_and_holds_mu(dim, grains):
    p = W.grain_growth(n=36 if dim == 3 else 64, dim=dim, grains=grains, nz=30 if dim == 3 else None)
    p.mu0 = p.mu0 + 0.25   # any held value
    g = _run(p, 60, "f64")
    o = oracle.run(p, p.phi0, p.mu0, 60)
    assert _err(g, o) <= 1e-10
    assert np.array_equal(g[1], p.mu0)


@pytest.mark.parametrize("zchunk", [7, 16])
def test_fp32_split_eight_grains(zchunk):
    p = W.grain_growth(n=48, dim=3, grains=8, nz=40)
    g = _run(p, 200, "f32", split=True, zchunk=zchunk)
    o = oracle.run(p, p.phi0, p.mu0, 200)
    assert _err(g, o) <= 1e-3
    assert np.array_equal(g[1], p.mu0.astype(np.float32).astype(np.float64))


def test_fp32_circle_rate():
    # the curvature-driven area loss of a circular grain on the GPU
    import math
    p = W.binary_problem("gg_gpu_circle", 128, dim=2, R=40.0, Delta=0.3)
    p.grain_growth = 1
    from paper_2404_01035_gb300 import Simulation
    sim = Simulation(p, dtype="f32")
    sim.set_fields(p.phi0, p.mu0)
    a0 = sim.get_fields()[0][0].astype(np.float64).sum()
    sim.step(2000)
    a1 = sim.get_fields()[0][0].astype(np.float64).sum()
    sim.close()
    rate = (a1 - a0) / (2000 * p.dt)
    assert rate == pytest.approx(-2.0 * math.pi * p.gamma[0, 1] / p.tau, rel=0.03)


def test_refused_with_anti_trapping_adjoint_and_batch():
    from paper_2404_01035_gb300 import Simulation
    from paper_2404_01035_gb300.batch import Batch
    p = W.grain_growth(n=32, dim=2, grains=2)
    sim = Simulation(p, dtype="f64")
    with pytest.raises(Exception):
        sim.enable_checkpoints(5)
    sim.close()
    with pytest.raises(Exception):
        Batch([p])
    with pytest.raises(Exception):
        Simulation(p.copy(anti_trapping=1), dtype="f64")
