"""GPU parity: the CUDA step (through the C ABI) against the FP64 oracle.

Bars: FP64 GPU build within 1e-10 of the oracle; FP32 GPU build within 1e-3
(max |d phi|, |d mu|) after 1000 steps; bit-exact where the arithmetic is
identical by construction (tile shapes, checkpoints, bulk cells).
"""
import numpy as np
import pytest

import oracle
import workloads as W

from gpu_util import pick_cells, windowed_one_step

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
FP32_TOL = 1e-3


def gpu_run(prob, steps, dtype, phi0=None, mu0=None, **kw):
    from paper_2404_01035_gb300 import Simulation
    sim = Simulation(prob, dtype=dtype)
    sim.set_fields(prob.phi0 if phi0 is None else phi0, prob.mu0 if mu0 is None else mu0)
    for k, v in kw.items():
        getattr(sim, k)(*v)
    sim.step(steps)
    sim.sync()
    phi, mu = sim.get_fields()
    sim.close()
    return phi.astype(np.float64), mu.astype(np.float64)


def max_err(a, b):
    return max(np.abs(a[0] - b[0]).max(), np.abs(a[1] - b[1]).max())


# ------------------------------------------------------------ whole-grid runs
def test_dendrite_2d_fp64_1000_steps():
    p = W.dendrite_2d()
    g = gpu_run(p, p.steps, "f64")
    o = oracle.run(p, p.phi0, p.mu0, p.steps)
    assert max_err(g, o) <= FP64_TOL


def test_dendrite_2d_fp32_1000_steps():
    p = W.dendrite_2d()
    g = gpu_run(p, p.steps, "f32")
    o = oracle.run(p, p.phi0, p.mu0, p.steps)
    assert max_err(g, o) <= FP32_TOL


def test_anisotropic_2d_fp32_1000_steps():
    p = W.binary_problem("aniso", 96, delta=0.04, Delta=0.25, R=8.0, potential="obstacle", ny=80)
    g = gpu_run(p, 1000, "f32")
    o = oracle.run(p, p.phi0, p.mu0, 1000)
    assert max_err(g, o) <= FP32_TOL
    assert np.abs(g[0] - p.phi0).max() > 0.1   # the seed did evolve


@pytest.mark.parametrize("pot", ["obstacle", "well"])
def test_3d_three_phase_ternary_fp64(pot):
    p = W.small_multiphase(n=20, dim=3, N=3, NM=2, nx=37, ny=21, nz=19, potential=pot,
                           rotate=True, gamma3=0.4)
    g = gpu_run(p, 40, "f64")
    o = oracle.run(p, p.phi0, p.mu0, 40)
    assert max_err(g, o) <= FP64_TOL


def test_3d_three_phase_ternary_fp32_1000_steps():
    p = W.small_multiphase(n=16, dim=3, N=3, NM=2, nx=20, ny=18, nz=16, rotate=True)
    g = gpu_run(p, 1000, "f32")
    o = oracle.run(p, p.phi0, p.mu0, 1000)
    assert max_err(g, o) <= FP32_TOL


@pytest.mark.parametrize("dtype,steps,tol", [("f64", 30, FP64_TOL), ("f32", 300, FP32_TOL)])
def test_3d_eight_phase_multigrain(dtype, steps, tol):
    p = W.multigrain_3d(n=40, grains=7, R=5.0, min_sep=14.0, seed=3)
    g = gpu_run(p, steps, dtype)
    o = oracle.run(p, p.phi0, p.mu0, steps)
    assert max_err(g, o) <= tol


def _split_tile(prob):
    from paper_2404_01035_gb300 import Simulation
    sim = Simulation(prob, dtype="f32")
    tiles = sim.tiles()
    sim.close()
    return [i for i, t in enumerate(tiles) if t[2] == 1][0], tiles


def test_3d_eight_phase_multigrain_split_variant():
    # the split step with 8 phases: rows around a grain hold few phases and
    # take the compact update (MODE 0 of the interface kernel)
    p = W.multigrain_3d(n=40, grains=7, R=5.0, min_sep=14.0, seed=3)
    t, _ = _split_tile(p)
    g = gpu_run(p, 300, "f32", set_launch=(t, 16))
    o = oracle.run(p, p.phi0, p.mu0, 300)
    assert max_err(g, o) <= FP32_TOL


def test_3d_eight_phase_dense_split_matches_fused():
    # every phase everywhere: rows whose box holds more than 4 phases go to
    # the second interface launch (MODE 1); agreement with the fused kernel
    # to FP32 rounding after 20 steps, bitwise across z-chunks
    p = W.small_multiphase(n=20, dim=3, N=8, NM=1, nx=70, ny=37, nz=30)
    t, tiles = _split_tile(p)
    fused = gpu_run(p, 20, "f32", set_launch=(0, 0))
    a = gpu_run(p, 20, "f32", set_launch=(t, 16))
    b = gpu_run(p, 20, "f32", set_launch=(t, 5))
    assert max_err(a, fused) <= 1e-6
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_2d_three_phase_ternary(dtype):
    p = W.small_multiphase(n=30, dim=2, N=3, NM=2, nx=70, ny=45, rotate=True, gamma3=0.3)
    steps = 60 if dtype == "f64" else 400
    g = gpu_run(p, steps, dtype)
    o = oracle.run(p, p.phi0, p.mu0, steps)
    assert max_err(g, o) <= (FP64_TOL if dtype == "f64" else FP32_TOL)


def test_3d_binary_noflux_everywhere_fp64():
    p = W.binary_problem("b3", 26, dim=3, delta=0.03, R=6.0, ny=23, nz=29,
                         bc=[W.BC_NOFLUX] * 3)
    g = gpu_run(p, 50, "f64")
    o = oracle.run(p, p.phi0, p.mu0, 50)
    assert max_err(g, o) <= FP64_TOL


# ---------------------------------------------------------------- edge cases
@pytest.mark.parametrize("shape", [(3, 3, 3), (1, 5, 40), (33, 1, 9), (7, 9, 1)])
def test_degenerate_3d_extents_fp64(shape):
    nx, ny, nz = shape
    p = W.small_multiphase(n=8, dim=3, N=3, NM=2, nx=nx, ny=ny, nz=nz)
    g = gpu_run(p, 10, "f64")
    o = oracle.run(p, p.phi0, p.mu0, 10)
    assert max_err(g, o) <= FP64_TOL


def test_one_row_strip_2d_fp64():
    p = W.binary_problem("strip", 200, ny=1, R=0.0, potential="well")
    x = np.arange(200) + 0.5
    s = 0.5 * (1 + np.tanh((x - 60) / 6.0)) * 0.5 * (1 + np.tanh((140 - x) / 6.0))
    p.phi0 = np.stack([s[None, None], 1 - s[None, None]])
    p.mu0 = np.full((1, 1, 1, 200), 1.634)
    g = gpu_run(p, 200, "f64")
    o = oracle.run(p, p.phi0, p.mu0, 200)
    assert max_err(g, o) <= FP64_TOL


@pytest.mark.parametrize("dim,dtype,steps,tol", [(2, "f64", 40, FP64_TOL), (3, "f64", 30, FP64_TOL),
                                                   (3, "f32", 200, FP32_TOL)])
def test_grid_spacing_other_than_one(dim, dtype, steps, tol):
    # dx = 1/2 with the interface width in cells held (eps = 2) and dt ~ dx^2:
    # every dx-scaled term of the step (gradients, divergences, Laplacians,
    # the temperature position) against the oracle, which a refinement test
    # pins on its own
    p = W.small_multiphase(n=20, dim=dim, N=3, NM=2, rotate=True)
    p = p.copy(dx=0.5, dt=0.25 * p.dt, eps=0.5 * p.eps)
    g = gpu_run(p, steps, dtype)
    o = oracle.run(p, p.phi0, p.mu0, steps)
    assert max_err(g, o) <= tol
    assert np.abs(o[0] - p.phi0).max() > 1e-3   # the state moved


def test_zero_steps_is_identity():
    p = W.dendrite_2d()
    g = gpu_run(p, 0, "f64")
    assert np.array_equal(g[0], p.phi0) and np.array_equal(g[1], p.mu0)


def test_single_phase_domain_stays_bitwise_fp32():
    p = W.small_multiphase(n=24, dim=3, N=3, NM=2)
    shape = (p.nz, p.ny, p.nx)
    phi0 = np.stack([np.zeros(shape), np.zeros(shape), np.ones(shape)])
    g = gpu_run(p, 50, "f32", phi0=phi0)
    assert np.array_equal(g[0], phi0)


# --------------------------------------------------- invariants, diagnostics
@pytest.mark.parametrize("dtype,rtol", [("f64", 1e-12), ("f32", 1e-5)])
def test_mass_conservation_and_diag_match_oracle(dtype, rtol):
    from paper_2404_01035_gb300 import Simulation
    p = W.small_multiphase(n=20, dim=3, N=3, NM=2, nx=33, ny=20, nz=18, rotate=True)
    sim = Simulation(p, dtype=dtype)
    sim.set_fields(p.phi0, p.mu0)
    d0 = sim.diag()
    o0 = oracle.diag(p, sim.get_fields()[0], sim.get_fields()[1])
    np.testing.assert_allclose(d0["mass"], o0[:2], rtol=1e-12 if dtype == "f64" else 1e-6)
    sim.step(200)
    d1 = sim.diag()
    sim.close()
    np.testing.assert_allclose(d1["mass"], d0["mass"], rtol=rtol)
    assert d1["sum_err"] < (1e-13 if dtype == "f64" else 1e-5)
    assert d1["phi_min"] >= 0.0 and d1["phi_max"] <= 1.0 + 1e-6
    assert d1["nonfinite"] == 0
    assert 0 < d1["mu_diffusion_number"] <= 1.0
    assert d1["step"] == 200 and d1["t"] == pytest.approx(200 * p.dt)


def test_tile_shapes_and_zchunks_agree():
    # each instantiation is compiled on its own, so FMA contraction may round
    # differently between tile shapes: agreement to FP32 rounding, bitwise
    # across z-chunks of one tile shape (same machine code)
    from paper_2404_01035_gb300 import Simulation
    p = W.small_multiphase(n=20, dim=3, N=3, NM=2, nx=70, ny=37, nz=45, rotate=True)
    ref = None
    sim = Simulation(p, dtype="f32")
    variants = [(t, z) for t in range(len(sim.tiles())) for z in (0, 5, 16)]
    per_tile = {}
    for t, z in variants:
        sim.set_fields(p.phi0, p.mu0)
        sim.set_launch(t, z)
        sim.step(20)
        phi, mu = sim.get_fields()
        if ref is None:
            ref = (phi, mu)
        # (separately compiled instantiations contract FMAs differently; after
        # 20 steps that is a few ulp of |mu| ~ 1.2, hence 5e-6)
        assert max(np.abs(phi - ref[0]).max(), np.abs(mu - ref[1]).max()) <= 5e-6, (t, z)
        if t in per_tile:
            assert np.array_equal(phi, per_tile[t][0]) and np.array_equal(mu, per_tile[t][1]), (t, z)
        per_tile[t] = (phi, mu)
    sim.close()


def test_checkpoint_restore_is_bitwise_and_views_match():
    from paper_2404_01035_gb300 import Simulation
    import torch
    p = W.small_multiphase(n=16, dim=3, N=3, NM=2, nx=30, ny=17, nz=15)
    sim = Simulation(p, dtype="f32")
    sim.set_fields(p.phi0, p.mu0)
    sim.step(7)
    blob = sim.checkpoint()
    sim.step(9)
    a = sim.get_fields()
    vphi, vmu = sim.fields()
    torch.cuda.synchronize()
    assert np.array_equal(vphi.cpu().numpy(), a[0]) and np.array_equal(vmu.cpu().numpy(), a[1])
    sim.restore(blob)
    assert sim.time()[0] == 7
    sim.step(9)
    b = sim.get_fields()
    sim.close()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_bulk_phi_reuse_survives_state_loads_and_adjoint_recompute():
    # Bulk rows whose pure phase is unchanged keep phi from the ping-pong
    # partner buffer.  Loading a state, restoring a checkpoint and the
    # adjoint's recompute (which reuses the code buffers) must leave every
    # later step bitwise equal to a fresh context started from the same state.
    from paper_2404_01035_gb300 import Simulation
    import torch
    p = W.eutectic_3d(n=48, steps=10)
    p.nz = 40
    p.phi0, p.mu0 = p.phi0[:, :40], p.mu0[:, :40]
    sim = Simulation(p, dtype="f32")
    for t, (tx, ty, split) in enumerate(sim.tiles()):
        sim.set_launch(t, 16)
        sim.set_fields(p.phi0, p.mu0)
        sim.step(9)
        blob = sim.checkpoint()
        sim.set_fields(p.phi0[::-1].copy(), p.mu0)   # another state over the same buffers
        sim.step(3)
        sim.restore(blob)
        sim.step(6)
        a = sim.get_fields()
        ref = Simulation(p, dtype="f32")
        ref.set_launch(t, 16)
        ref.restore(blob)
        ref.step(6)
        b = ref.get_fields()
        ref.close()
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), (tx, ty, split)
    sim.close()
    # adjoint recompute (3-D binary, FP64: the fused kernel's phi reuse)
    q = W.binary_problem("reuse", 24, dim=3, R=6.0, nz=20)
    sim = Simulation(q, dtype="f64")
    sim.set_fields(q.phi0, q.mu0)
    sim.enable_checkpoints(4)
    sim.step(10)
    blob = sim.checkpoint()
    lam = torch.ones((2, 20, 24, 24), dtype=torch.float64, device="cuda")
    sim.grad(lam, want_fields=False)
    sim.step(5)
    a = sim.get_fields()
    sim.close()
    ref = Simulation(q, dtype="f64")
    ref.restore(blob)
    ref.step(5)
    b = ref.get_fields()
    ref.close()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_switching_between_split_and_fused_steps_mid_run():
    # The split step marks bulk rows whose pure phase held over two steps
    # (phi is then kept from the ping-pong partner); the fused step reads the
    # partner's codes instead.  Alternating the two on one context, without
    # reloading the state, must still track the oracle.
    from paper_2404_01035_gb300 import Simulation
    p = W.eutectic_3d(n=48, steps=10)
    p.nz = 40
    p.phi0, p.mu0 = p.phi0[:, :40], p.mu0[:, :40]
    sim = Simulation(p, dtype="f32")
    tiles = sim.tiles()
    split = [i for i, t in enumerate(tiles) if t[2] == 1][0]
    fused = [i for i, t in enumerate(tiles) if t[2] == 0][0]
    sim.set_fields(p.phi0, p.mu0)
    for r in range(8):
        sim.set_launch(split if r % 2 == 0 else fused, 8 if r % 4 < 2 else 16)
        sim.step(4 + r % 3)
    g = sim.get_fields()
    sim.close()
    o = oracle.run(p, p.phi0, p.mu0, sum(4 + r % 3 for r in range(8)))
    assert max_err(g, o) <= FP32_TOL


def test_device_and_host_field_io_agree():
    from paper_2404_01035_gb300 import Simulation
    import torch
    p = W.small_multiphase(n=16, dim=2, N=3, NM=2, nx=40, ny=33)
    sim = Simulation(p, dtype="f64")
    tphi = torch.tensor(p.phi0, device="cuda")
    tmu = torch.tensor(p.mu0, device="cuda")
    sim.set_fields(tphi, tmu)
    sim.step(5)
    h = sim.get_fields()
    dphi = torch.empty_like(tphi)
    dmu = torch.empty_like(tmu)
    sim.get_fields_into(dphi, dmu, on_device=True)
    sim.close()
    assert np.array_equal(dphi.cpu().numpy(), h[0]) and np.array_equal(dmu.cpu().numpy(), h[1])


def test_autotuner_picks_a_variant_and_caches(tmp_path):
    from paper_2404_01035_gb300 import Simulation
    p = W.eutectic_3d(n=64, steps=10)
    sim = Simulation(p, dtype="f32")
    sim.set_fields(p.phi0, p.mu0)
    cache = str(tmp_path / "tune.json")
    ms = sim.tune(cache, steps_per_trial=5)
    assert ms > 0
    assert sim.time()[0] == 0            # state restored
    ms2 = sim.tune(cache, steps_per_trial=5)
    assert ms2 == pytest.approx(ms, rel=1e-5)
    sim.close()


# -------------------------------------------------- full-size, sampled parity
def _full_size_sampled(prob, dtype, warm_steps, seed, tol):
    from paper_2404_01035_gb300 import Simulation
    rng = np.random.default_rng(seed)
    sim = Simulation(prob, dtype=dtype)
    sim.set_fields(prob.phi0, prob.mu0)
    sim.step(warm_steps)
    phi_n, mu_n = sim.get_fields()
    t_n = sim.time()[1]
    sim.step(1)
    phi_1, mu_1 = sim.get_fields()
    d = sim.diag()
    sim.close()
    cells = pick_cells(phi_n, rng)
    ophi, omu = windowed_one_step(prob, phi_n, mu_n, cells, t0=t_n)
    gphi = np.array([phi_1[:, z, y, x] for (z, y, x) in cells])
    gmu = np.array([mu_1[:, z, y, x] for (z, y, x) in cells])
    assert np.abs(gphi - ophi).max() <= tol
    assert np.abs(gmu - omu).max() <= tol
    assert d["nonfinite"] == 0
    return d


def test_eutectic_3d_full_size_sampled_parity_fp32():
    p = W.eutectic_3d()
    _full_size_sampled(p, "f32", warm_steps=300, seed=1, tol=2e-5)


def test_eutectic_3d_full_size_invariants_2000_steps():
    from paper_2404_01035_gb300 import Simulation
    p = W.eutectic_3d()
    sim = Simulation(p, dtype="f32")
    sim.set_fields(p.phi0, p.mu0)
    d0 = sim.diag()
    sim.step(p.steps)
    d1 = sim.diag()
    sim.close()
    np.testing.assert_allclose(d1["mass"], d0["mass"], rtol=2e-5)
    assert d1["sum_err"] < 1e-5 and d1["phi_min"] >= 0 and d1["nonfinite"] == 0


def test_multigrain_3d_full_size_sampled_parity_fp32():
    p = W.multigrain_3d()
    _full_size_sampled(p, "f32", warm_steps=20, seed=2, tol=2e-5)
