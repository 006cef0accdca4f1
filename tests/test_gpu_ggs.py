"""Sparse grain growth (ms_ggs_*: few grains stored per cell, the projection
over the locally active grains) against the FP64 oracle with the same
reading, through the C ABI."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def _run(prob, steps, dtype, phi0=None):
    from paper_2404_01035_gb300.sparse_gg import SparseGrainGrowth
    s = SparseGrainGrowth(prob, dtype=dtype)
    s.set_fields(prob.phi0 if phi0 is None else phi0)
    s.step(steps)
    s.sync()
    phi = s.get_fields()
    listed, n = s.stats()
    s.close()
    assert n == steps
    return phi.astype(np.float64), listed


@pytest.mark.parametrize("dim,grains,n,steps", [(2, 32, 128, 60), (3, 8, 48, 30)])
def test_fp64_matches_the_oracle(dim, grains, n, steps):
    p = W.sparse_grain_growth(n=n, dim=dim, grains=grains)
    if dim == 3:
        p = p.copy(bc=[3, 3, 1])
    g, listed = _run(p, steps, "f64")
    o, _ = oracle.run(p, p.phi0, p.mu0, steps)
    assert np.abs(g - o).max() <= 1e-10
    assert np.abs(o - p.phi0).max() > 0.1      # the boundaries moved
    assert 0 < listed < p.nx * p.ny * p.nz    # bulk cells were not listed
    assert (o > 0).sum(axis=0).max() <= 8


def test_grid_spacing_other_than_one_fp64():
    # the sparse kernels' own gradients and divergences at dx = 1/2
    p = W.sparse_grain_growth(n=64, dim=2, grains=16)
    p = p.copy(dx=0.5, dt=0.25 * p.dt, eps=0.5 * p.eps)
    g, _ = _run(p, 40, "f64")
    o, _ = oracle.run(p, p.phi0, p.mu0, 40)
    assert np.abs(g - o).max() <= 1e-10
    assert np.abs(o - p.phi0).max() > 1e-3


def test_fp32_matches_the_oracle():
    p = W.sparse_grain_growth(n=128, dim=2, grains=32)
    g, _ = _run(p, 200, "f32")
    o, _ = oracle.run(p, p.phi0, p.mu0, 200)
    assert np.abs(g - o).max() <= 1e-3


def test_two_grains_equal_the_dense_path():
    # with two grains the locally active set is the global one: the dense
    # grain-growth context and the sparse one step the same equation
    from paper_2404_01035_gb300 import Simulation
    p = W.grain_growth(n=64, dim=2, grains=2)
    s, _ = _run(p, 80, "f64")
    sim = Simulation(p, dtype="f64")
    sim.set_fields(p.phi0, p.mu0)
    sim.step(80)
    d, _ = sim.get_fields()
    sim.close()
    assert np.abs(s - d).max() <= 1e-12


def test_refusals_and_the_overflow_status():
    from paper_2404_01035_gb300._binding import MSError
    from paper_2404_01035_gb300.sparse_gg import SparseGrainGrowth
    p = W.sparse_grain_growth(n=32, dim=2, grains=10)
    d = p.delta.copy()
    d[0, 1] = d[1, 0] = 0.02
    for bad in (p.copy(delta=d), p.copy(potential="well")):
        with pytest.raises(MSError) as ex:
            SparseGrainGrowth(bad, dtype="f64")
        assert ex.value.status == 9
    g3 = p.gamma3.copy()
    g3[0, 1, 2] = 3.0
    with pytest.raises(MSError):
        SparseGrainGrowth(p.copy(gamma3=g3), dtype="f64")
    # a cell holding 9 grains is refused at the input
    phi = np.zeros((10, 1, 32, 32))
    phi[:, 0, 5, 5] = 0.1
    phi[0] = np.where(phi[0] == 0, 1.0, phi[0])
    s = SparseGrainGrowth(p, dtype="f64")
    with pytest.raises(MSError) as ex:
        s.set_fields(phi)
    assert ex.value.status == 7
    s.close()
    # a stencil that would need more than 8 grains: a 3-grain cell whose four
    # face neighbours are four other pure grains and whose corners two more
    phi = np.zeros((10, 1, 32, 32))
    phi[0] = 1.0
    phi[:, 0, 10, 10] = 0.0
    phi[1:4, 0, 10, 10] = [0.4, 0.3, 0.3]
    for k, (y, x) in enumerate([(9, 10), (11, 10), (10, 9), (10, 11)]):
        phi[:, 0, y, x] = 0.0
        phi[4 + k, 0, y, x] = 1.0
    phi[:, 0, 9, 11] = 0.0
    phi[8, 0, 9, 11] = 1.0
    phi[:, 0, 11, 9] = 0.0
    phi[9, 0, 11, 9] = 1.0
    s = SparseGrainGrowth(p, dtype="f64")
    s.set_fields(phi)
    s.step(2)
    with pytest.raises(MSError) as ex:
        s.sync()
    assert ex.value.status == 7
    s.close()
