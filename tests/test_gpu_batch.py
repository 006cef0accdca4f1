"""Batched persistent launch: every simulation of a batch matches its own
single-simulation run (same arithmetic, separately compiled kernel: equal to
FP32 rounding) and, for small ones, the FP64 oracle."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def _standalone(p, steps):
    from paper_2404_01035_gb300 import Simulation
    sim = Simulation(p, dtype="f32")
    sim.set_fields(p.phi0, p.mu0)
    sim.step(steps)
    out = sim.get_fields()
    sim.close()
    return out


def _mixed_batch():
    sims = []
    for i, (nx, ny, d, D) in enumerate([(64, 64, 0.01, 0.1), (96, 70, 0.05, 0.4), (45, 130, 0.03, 0.25),
                                        (160, 96, 0.02, 0.3), (33, 33, 0.04, 0.15), (70, 45, 0.0, 0.2)]):
        p = W.binary_problem(f"b{i}", nx, ny=ny, delta=d, Delta=D, R=6.0, potential="obstacle",
                             dtype_note="f32")
        if i == 5:
            p.bc = [W.BC_NOFLUX, W.BC_PERIODIC, W.BC_PERIODIC]
        sims.append(p)
    return sims


def test_batch_matches_standalone_runs_and_oracle():
    from paper_2404_01035_gb300.batch import Batch
    probs = _mixed_batch()
    b = Batch(probs)
    for i, p in enumerate(probs):
        b.set_fields(i, p.phi0, p.mu0)
    b.step(130)       # two launches with different parity
    b.step(170)
    b.sync()
    for i, p in enumerate(probs):
        phi, mu = b.get_fields(i)
        sphi, smu = _standalone(p, 300)
        assert np.abs(phi - sphi).max() <= 1e-5 and np.abs(mu - smu).max() <= 1e-5, i
        if p.nx * p.ny <= 64 * 64:
            ophi, omu = oracle.run(p, p.phi0, p.mu0, 300)
            assert max(np.abs(phi - ophi).max(), np.abs(mu - omu).max()) <= 1e-3
    assert b.cells == sum(p.nx * p.ny for p in probs)
    b.close()


def test_simulations_at_different_grid_spacings_in_one_batch():
    # each simulation's own dx (interface width in cells held, dt ~ dx^2)
    from paper_2404_01035_gb300.batch import Batch
    probs = []
    for i, dx in enumerate((1.0, 0.5, 0.25)):
        p = W.binary_problem(f"dx{i}", 48, ny=40, delta=0.03, Delta=0.2, R=6.0, potential="obstacle",
                             dtype_note="f32")
        probs.append(p.copy(dx=dx, dt=p.dt * dx * dx, eps=p.eps * dx))
    b = Batch(probs)
    for i, p in enumerate(probs):
        b.set_fields(i, p.phi0, p.mu0)
    b.step(200)
    b.sync()
    for i, p in enumerate(probs):
        phi, mu = b.get_fields(i)
        ophi, omu = oracle.run(p, p.phi0, p.mu0, 200)
        assert max(np.abs(phi - ophi).max(), np.abs(mu - omu).max()) <= 1e-3, i
        assert np.abs(ophi - p.phi0).max() > 1e-3
    b.close()


def test_batch_of_512_dendrites_runs_500_steps():
    from paper_2404_01035_gb300.batch import Batch
    probs = W.batched_dendrites_2d()
    b = Batch(probs)
    for i, p in enumerate(probs):
        b.set_fields(i, p.phi0, p.mu0)
    b.step(500)
    b.sync()
    rng = np.random.default_rng(0)
    for i in rng.choice(len(probs), size=4, replace=False):
        p = probs[i]
        phi, mu = b.get_fields(int(i))
        sphi, smu = _standalone(p, 500)
        assert np.abs(phi - sphi).max() <= 1e-5 and np.abs(mu - smu).max() <= 1e-5, i
        assert np.abs(phi.sum(axis=0) - 1).max() < 1e-5
    b.close()


@pytest.mark.parametrize("ty", [4, 16])
def test_every_tile_height_matches_standalone_runs(ty):
    from paper_2404_01035_gb300.batch import Batch
    probs = _mixed_batch()
    b = Batch(probs)
    assert b.tile_height() == 8
    b.set_tile(ty)
    assert b.tile_height() == ty
    for i, p in enumerate(probs):
        b.set_fields(i, p.phi0, p.mu0)
    b.step(120)
    b.sync()
    for i, p in enumerate(probs):
        phi, mu = b.get_fields(i)
        sphi, smu = _standalone(p, 120)
        assert np.abs(phi - sphi).max() <= 1e-5 and np.abs(mu - smu).max() <= 1e-5, (ty, i)
    with pytest.raises(Exception):
        b.set_tile(12)
    b.close()


def test_tuner_restores_the_states_and_keeps_a_compiled_height():
    from paper_2404_01035_gb300.batch import Batch
    probs = _mixed_batch()
    b = Batch(probs)
    for i, p in enumerate(probs):
        b.set_fields(i, p.phi0, p.mu0)
    b.step(40)
    before = [b.get_fields(i) for i in range(len(probs))]
    ms = b.tune(steps_per_trial=30)
    assert ms > 0 and b.tile_height() in (4, 8, 16)
    for i in range(len(probs)):   # the trials left the states as they were
        phi, mu = b.get_fields(i)
        assert np.array_equal(phi, before[i][0]) and np.array_equal(mu, before[i][1])
    b.step(60)                    # and stepping continues from them
    b.sync()
    for i, p in enumerate(probs):
        phi, mu = b.get_fields(i)
        sphi, smu = _standalone(p, 100)
        assert np.abs(phi - sphi).max() <= 1e-5 and np.abs(mu - smu).max() <= 1e-5, i
    b.close()
