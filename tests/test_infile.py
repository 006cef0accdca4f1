"""The paper-format input reader (`paper_2404_01035_gb300.infile`), on the CPU.

Expected values are typed from the format the paper prints (Sec. "Input
files"), not computed by the reader: pair lists in the order 12, 13, ..., 23;
per-phase lists headed by the phase index; BOUNDARY codes per face; the
Tempgrady tuple.  A spec written out and read back must drive the oracle
exactly like the workload it came from.
"""
import ctypes
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W
from paper_2404_01035_gb300 import infile as I
from paper_2404_01035_gb300.simulation import make_grid, make_params

TERNARY_3D = """
## a hand-written three-phase ternary deck in the paper's format
DIMENSION = 3;
MESH_X = 12;  MESH_Y = 10;  MESH_Z = 8;
DELTA_X = 0.5; DELTA_Y = 0.5; DELTA_Z = 0.5;
DELTA_t = 0.004;
NUMPHASES = 3;
NUMCOMPONENTS = 3;
NTIMESTEPS = 250;
COMPONENTS = {Al, Cu, Ag};
PHASES = {alpha, beta, liquid};
GAMMA = {1.1, 0.9, 1.3};                     # 12, 13, 23
DIFFUSIVITY = {1, 0, 0.01, 0.02};            # diagonal: phase 0, D11, D22
DIFFUSIVITY = {0, 2, 1.0, 0.8, 0.1};         # full: phase 2, D11, D22, D12
BOUNDARY = {phi, 3, 3, 1, 1, 3, 3};
BOUNDARY = {mu, 3, 3, 1, 1, 3, 3};
BOUNDARY = {c, 3, 3, 1, 1, 3, 3};
BOUNDARY = {T, 1, 1, 1, 1, 1, 1};            # the frozen temperature: not used
BOUNDARY_VALUE = {phi, 0, 0, 0, 0, 0, 0};
epsilon = 2.5;
tau = 0.8;
Tau = {0.28};                                # pairwise relaxation: not used
Function_anisotropy = 1;
Anisotropy_type = 4;
dab = {0.01, 0.02, 0.03};
Rotation_matrix = {0, 2, 0, 0, 30};
Rotation_matrix = {1, 2, 90, 0, 0};
Function_W = 2;
Gamma_abc = {4.5};
ISOTHERMAL = 0;
Equilibrium_temperature = 1.0;
Tempgrady = {0.97, 0.2, 40, 3, 0.05};
Function_F = 1;
A = {0, 1.0, 1.1, 0.05};                     # phase 0: A11, A22, A12
A = {1, 0.9, 1.2, -0.02};
A = {2, 1.0, 1.0, 0.0};
ceq = {0, 0, 0.8, 0.1};
ceq = {0, 2, 0.4, 0.3};                      # the liquid's value again: not used for phase 0
ceq = {1, 1, 0.1, 0.7};
ceq = {2, 2, 0.4, 0.3};
slopes = {0, 0, -0.1, 0.02};
slopes = {1, 1, 0.05, -0.03};
slopes = {2, 2, 0.0, 0.0};
Noise_phasefield = 1;
Amp_Noise_Phase = 0.02;
SAVET = 50;
"""


def test_parse_values_lists_comments_and_repeats():
    kv = I.parse("A = 1;  # one\nB = {1, x, 'y', 2e-3};\nB = {};\nC = word;\n## D = 5;\n")
    assert kv["A"] == [1.0]
    assert kv["B"] == [[1.0, "x", "y", 0.002], []]
    assert kv["C"] == ["word"]
    assert "D" not in kv
    for bad in ("A 1;", "A = {1, 2;", "1A = 3;"):
        with pytest.raises(ValueError):
            I.parse(bad)


def test_ternary_deck_maps_onto_the_spec():
    s = I.read_infile(TERNARY_3D)
    assert (s.dim, s.nx, s.ny, s.nz, s.n_phases, s.n_components) == (3, 12, 10, 8, 3, 3)
    assert (s.dx, s.dt, s.eps, s.tau, s.steps) == (0.5, 0.004, 2.5, 0.8, 250)
    assert s.bc == [3, 1, 3] and s.potential == "well"
    np.testing.assert_array_equal(s.gamma, [[0, 1.1, 0.9], [1.1, 0, 1.3], [0.9, 1.3, 0]])
    np.testing.assert_array_equal(s.delta, [[0, 0.01, 0.02], [0.01, 0, 0.03], [0.02, 0.03, 0]])
    np.testing.assert_array_equal(s.D[0], [[0.01, 0], [0, 0.02]])
    np.testing.assert_array_equal(s.D[1], np.zeros((2, 2)))
    np.testing.assert_array_equal(s.D[2], [[1.0, 0.1], [0.1, 0.8]])
    np.testing.assert_array_equal(s.A[0], [[1.0, 0.05], [0.0, 1.1]])      # i <= j entries
    np.testing.assert_array_equal(s.A[1], [[0.9, -0.02], [0.0, 1.2]])
    np.testing.assert_array_equal(s.ceq, [[0.8, 0.1], [0.1, 0.7], [0.4, 0.3]])
    np.testing.assert_array_equal(s.slopes, [[-0.1, 0.02], [0.05, -0.03], [0.0, 0.0]])
    assert s.gamma3[0, 1, 2] == s.gamma3[2, 1, 0] == 4.5 and s.gamma3[0, 0, 1] == 0.0
    # T = 0.97 + (0.2 / 40) (s - 3 - 0.05 t) along the last axis
    assert (s.T0, s.G, s.z0, s.V, s.T_ref) == (0.97, 0.2 / 40, 3.0, 0.05, 1.0)
    assert s.noise_amp == 0.02
    assert s.meta["phases"] == ["alpha", "beta", "liquid"]
    assert s.meta["components"] == ["Al", "Cu", "Ag"]
    assert s.meta["ignored"] == ["Tau"]
    assert s.meta["savet"] == 50
    # rotations: 30 degrees about z for (0, 2), 90 degrees about x for (1, 2)
    c, h = math.cos(math.radians(30)), math.sin(math.radians(30))
    np.testing.assert_allclose(s.rot[0, 2], [[c, -h, 0], [h, c, 0], [0, 0, 1]], atol=1e-15)
    np.testing.assert_allclose(s.rot[2, 0], s.rot[0, 2], atol=0)
    np.testing.assert_allclose(s.rot[1, 2] @ [0, 1, 0], [0, 0, 1], atol=1e-15)   # y turns into z
    np.testing.assert_array_equal(s.rot[0, 1], np.eye(3))


def test_euler_rotation_order_and_inverse():
    # Rz Ry Rx: x first.  (90, 90, 0) takes y -> z (x-turn) -> +x (y-turn), while
    # the other order (y-turn first) would leave y alone and then take it to z
    R = I.euler_rotation(90, 90, 0)
    np.testing.assert_allclose(R @ [0, 1, 0], [1, 0, 0], atol=1e-15)
    np.testing.assert_allclose(I.euler_rotation(0, 0, 90) @ [1, 0, 0], [0, 1, 0], atol=1e-15)
    rng = np.random.default_rng(3)
    for _ in range(20):
        ang = rng.uniform(-170, 170, 3)
        ang[1] = rng.uniform(-85, 85)
        R = I.euler_rotation(*ang)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-14)
        np.testing.assert_allclose(I._euler_angles(R), ang, atol=1e-9)


@pytest.mark.parametrize("edit,match", [
    (("Function_F = 1;", "Function_F = 3;"), "CALPHAD"),
    (("BOUNDARY = {mu, 3, 3, 1, 1, 3, 3};", "BOUNDARY = {mu, 3, 3, 2, 2, 3, 3};"), "not supported"),
    (("BOUNDARY = {phi, 3, 3, 1, 1, 3, 3};", "BOUNDARY = {phi, 3, 1, 1, 1, 3, 3};"), "differ"),
    (("BOUNDARY = {c, 3, 3, 1, 1, 3, 3};", "BOUNDARY = {c, 1, 1, 1, 1, 3, 3};"), "other fields"),
    (("DELTA_Z = 0.5;", "DELTA_Z = 0.25;"), "uniform"),
    (("Anisotropy_type = 4;", "Anisotropy_type = 6;"), "four-fold"),
    (("GAMMA = {1.1, 0.9, 1.3};", "GAMMA = {1.1, 0.9};"), "pair values"),
    (("A = {1, 0.9, 1.2, -0.02};", "A = {1, 0.9, 1.2, -0.02, 7};"), "off-diagonal"),
    (("DIMENSION = 3;", "DIMENSION = 4;"), "DIMENSION"),
    (("BOUNDARY_VALUE = {phi, 0, 0, 0, 0, 0, 0};", "BOUNDARY_VALUE = {phi, 0, 0, 0.1, 0, 0, 0};"), "non-zero flux"),
    (("Rotation_matrix = {0, 2, 0, 0, 30};", "Rotation_matrix = {0, 3, 0, 0, 30};"), "phase index"),
    (("Rotation_matrix = {0, 2, 0, 0, 30};", "Rotation_matrix = {2, 2, 0, 0, 30};"), "two different"),
    (("ceq = {1, 1, 0.1, 0.7};", "ceq = {1, 1, 0.1};"), "values"),
    (("Tempgrady = {0.97, 0.2, 40, 3, 0.05};", "Tempgrady = {0.97, 0.2, 0, 3, 0.05};"), "DISTANCE"),
    (("DIFFUSIVITY = {1, 0, 0.01, 0.02};", "DIFFUSIVITY = {1, 1.5, 0.01, 0.02};"), "phase index"),
])
def test_unsupported_input_is_refused(edit, match):
    old, new = edit
    assert TERNARY_3D.count(old) == 1
    with pytest.raises(ValueError, match=match):
        I.read_infile(TERNARY_3D.replace(old, new))


def test_calphad_deck_reads_with_the_parabolic_coefficients_on_request():
    s = I.read_infile(TERNARY_3D.replace("Function_F = 1;", "Function_F = 3;"), free_energy="parabolic")
    np.testing.assert_array_equal(s.ceq[0], [0.8, 0.1])


def test_elasticity_needs_one_homogeneous_stiffness():
    base = TERNARY_3D + "EIGEN_STRAIN = {0, 0.01, 0.02, 0.03, 0.004, 0.005, 0.006};\n"
    iso = base + "VOIGT_ISOTROPIC = {0, 3.0, 1.0, 1.0};\nVOIGT_ISOTROPIC = {2, 3.0, 1.0, 1.0};\n"
    s = I.read_infile(iso, elasticity=True)
    C = np.array([[3, 1, 1, 0, 0, 0], [1, 3, 1, 0, 0, 0], [1, 1, 3, 0, 0, 0],
                  [0, 0, 0, 1, 0, 0], [0, 0, 0, 0, 1, 0], [0, 0, 0, 0, 0, 1]], dtype=float)
    np.testing.assert_array_equal(s.elastic_C, C)
    np.testing.assert_array_equal(s.eigenstrain[0], [[0.01, 0.006, 0.005], [0.006, 0.02, 0.004],
                                                     [0.005, 0.004, 0.03]])
    np.testing.assert_array_equal(s.eigenstrain[1], np.zeros((3, 3)))
    assert I.read_infile(iso).elastic_C is None          # elasticity is opt-in
    tet = base + "VOIGT_TETRAGONAL = {0, 3.0, 1.0, 0.8, 2.5, 0.9, 0.7};\n"
    C = I.read_infile(tet, elasticity=True).elastic_C
    assert (C[0, 0], C[1, 1], C[2, 2], C[0, 1], C[0, 2], C[1, 2], C[3, 3], C[4, 4], C[5, 5]) == \
        (3.0, 3.0, 2.5, 1.0, 0.8, 0.8, 0.9, 0.9, 0.7)
    with pytest.raises(ValueError, match="homogeneous"):
        I.read_infile(base + "VOIGT_CUBIC = {0, 3.0, 1.0, 1.0};\nVOIGT_CUBIC = {2, 6.0, 2.0, 2.0};\n",
                      elasticity=True)


def _same_spec(a, b):
    for k in ("dim", "nx", "ny", "n_phases", "n_components", "dx", "dt", "eps", "tau", "potential",
              "T_ref", "T0", "G", "z0", "V"):
        assert getattr(a, k) == pytest.approx(getattr(b, k), rel=1e-15, abs=1e-15), k
    assert list(a.bc)[: a.dim] == list(b.bc)[: b.dim]
    for k in ("gamma", "delta", "D", "A", "ceq", "slopes"):
        np.testing.assert_allclose(np.asarray(getattr(a, k)), np.asarray(getattr(b, k)), atol=1e-15, err_msg=k)
    np.testing.assert_allclose(a.rot, b.rot, atol=1e-14)
    ga, gb = getattr(a, "gamma3", None), getattr(b, "gamma3", None)
    assert (ga is None or not np.any(ga)) == (gb is None or not np.any(gb))
    if ga is not None and np.any(ga):
        np.testing.assert_allclose(ga, gb, atol=1e-15)


@pytest.mark.parametrize("make", [
    lambda: W.dendrite_2d(),
    lambda: W.small_multiphase(n=10, dim=3, N=3, NM=2, rotate=True),
    lambda: W.small_multiphase(n=12, dim=2, N=4, NM=1, potential="well", gamma3=2.0),
])
def test_written_deck_reads_back_and_drives_the_oracle_identically(make):
    p = make()
    p.f0 = np.zeros(p.n_phases)        # the infile has no isothermal offsets
    s = I.read_infile(I.write_infile(p))
    _same_spec(s, p)
    a = oracle.run(p, p.phi0, p.mu0, 3)
    b = oracle.run(s, p.phi0, p.mu0, 3)
    assert max(np.abs(a[0] - b[0]).max(), np.abs(a[1] - b[1]).max()) < 1e-13


def test_spec_marshals_like_the_workload_problem():
    p = W.small_multiphase(n=10, dim=3, N=3, NM=2, rotate=True)
    p.f0 = np.zeros(3)
    s = I.read_infile(I.write_infile(p))
    ka, kb = [], []
    pa, pb = make_params(p, "f64", ka), make_params(s, "f64", kb)
    for name, ctype in pa._fields_:
        if ctype is ctypes.c_void_p:
            continue                   # addresses: the arrays behind them are compared below
        assert getattr(pa, name) == pytest.approx(getattr(pb, name), abs=1e-14), name
    assert len(ka) == len(kb)
    for x, y in zip(ka, kb):
        np.testing.assert_allclose(x, y, atol=1e-14)
    ga, gb = make_grid(p), make_grid(s)
    assert (ga.dim, ga.nx, ga.ny, ga.nz, ga.dx, list(ga.bc)) == (gb.dim, gb.nx, gb.ny, gb.nz, gb.dx, list(gb.bc))


def test_filling_shapes_sharp():
    s = I.read_infile(TERNARY_3D)
    fill = """
    FILLCUBE = {0, 2, 3, 1, 5, 6, 4};          # cells x 2..5, y 3..6, z 1..4
    #FILLSPHERE = {1, 6, 5, 4, 3};             # commented out
    FILLSPHERE = {1, 9, 2, 6, 1.5};
    """
    phi = I.read_filling(fill, s, diffuse=False)
    assert phi.shape == (3, 8, 10, 12)
    np.testing.assert_array_equal(phi.sum(axis=0), 1.0)
    assert phi[0].sum() == 4 * 4 * 4
    assert phi[0, 1:5, 3:7, 2:6].min() == 1.0
    # sphere of radius 1.5 about cell (9, 2, 6): cells at distance < 1.5 (1 + 6 + 12 = 19)
    assert phi[1].sum() == 19
    assert phi[2].sum() == 8 * 10 * 12 - 64 - 19


def test_filling_later_lines_paint_over_and_profiles_are_diffuse():
    s = I.read_infile(TERNARY_3D.replace("DIMENSION = 3;", "DIMENSION = 2;").replace("MESH_X = 12;", "MESH_X = 64;")
                      .replace("MESH_Y = 10;", "MESH_Y = 64;").replace("Function_W = 2;", "Function_W = 1;"))
    assert s.dim == 2 and s.nz == 1 and s.potential == "obstacle"
    fill = "FILLCYLINDER = {0, 32, 32, 0, 0, 20};\nFILLELLIPSE = {1, 32, 32, 6, 0.6, 30};\n"
    sharp = I.read_filling(fill, s, diffuse=False)
    # ellipse: semi-axes 6 and 4.8 (eccentricity 0.6) painted over the disc
    assert abs(sharp[1].sum() - math.pi * 6 * 4.8) < 0.1 * math.pi * 6 * 4.8
    assert abs(sharp[0].sum() - (math.pi * 400 - math.pi * 6 * 4.8)) < 0.03 * math.pi * 400
    phi = I.read_filling(fill, s)
    np.testing.assert_allclose(phi.sum(axis=0), 1.0, atol=1e-14)
    assert phi.min() >= 0.0
    # the disc's boundary along +x, beyond the ellipse's compact profile: phi_0 is
    # exactly 1/2 at radius 20, and the sine profile spans pi^2 eps / 4 cells
    row = phi[0, 0, 32]
    assert row[52] == 0.5
    half = math.pi ** 2 * (s.eps / s.dx) / 8
    assert row[52 - int(half) + 1] < 1.0 and row[52 - int(half) - 1] == 1.0
    assert row[52 + int(half) - 1] > 0.0 and row[52 + int(half) + 1] == 0.0


def test_liquid_mu_gives_the_liquid_its_composition():
    s = I.read_infile(TERNARY_3D)
    for c in ([0.4, 0.3], [0.2, 0.5]):
        mu = I.liquid_mu(s, c)
        for T in (0.9, 1.0, 1.1):
            cl, _, _ = oracle.thermo(s, s.n_phases - 1, mu, T)
            np.testing.assert_allclose(cl, c, atol=1e-14)


FILLING_2D = """
FILLCYLINDER = {0, 16, 16, 0, 0, 6};
FILLCUBE = {1, 30, 4, 0, 40, 12, 0};
"""


def test_run_driver_dry_run(tmp_path, capsys):
    """The command-line driver reads and checks a deck and a filling file and
    reports them without a GPU (--dry-run)."""
    import json
    from paper_2404_01035_gb300 import run
    deck = (TERNARY_3D.replace("DIMENSION = 3;", "DIMENSION = 2;").replace("MESH_X = 12;", "MESH_X = 48;")
            .replace("MESH_Y = 10;", "MESH_Y = 32;") + "cfill = {2, 2, 0.35, 0.25};\n")
    (tmp_path / "deck.in").write_text(deck)
    (tmp_path / "fill.in").write_text(FILLING_2D)
    rc = run.main([str(tmp_path / "deck.in"), str(tmp_path / "fill.in"), "--dry-run"])
    assert rc == 0
    info = json.loads(capsys.readouterr().out.strip().splitlines()[-1])["inputs"]
    assert info["grid"] == [2, 48, 32, 1] and info["steps"] == 250 and info["save_every"] == 50
    assert info["library_check"] == "ok" and 0.004 < info["dt_bound"]
    assert info["bc"] == [3, 1] and info["potential"] == "well" and info["ignored_keys"] == ["Tau"]
    s = I.read_infile(deck)
    np.testing.assert_allclose(info["mu0"], I.liquid_mu(s, [0.35, 0.25]), atol=1e-15)
    assert sum(info["phase_fractions"]) == pytest.approx(1.0, abs=1e-14)
    assert 0.0 < info["phase_fractions"][0] < info["phase_fractions"][2]
    with pytest.raises(ValueError, match="CALPHAD"):
        (tmp_path / "bad.in").write_text(deck.replace("Function_F = 1;", "Function_F = 2;"))
        run.main([str(tmp_path / "bad.in"), str(tmp_path / "fill.in"), "--dry-run"])
    # a time step above the library's stability bound is refused before any GPU work
    capsys.readouterr()
    (tmp_path / "fast.in").write_text(deck.replace("DELTA_t = 0.004;", "DELTA_t = 0.5;"))
    assert run.main([str(tmp_path / "fast.in"), str(tmp_path / "fill.in"), "--dry-run"]) == 2
    info = json.loads(capsys.readouterr().out.strip().splitlines()[-1])["inputs"]
    assert "stability" in info["library_check"] and 0.0 < info["dt_bound"] < 0.5


DECKS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "decks")


def test_bundled_deck_passes_the_library_checks():
    """The deck the GPU driver test runs is one the library accepts: ms_create on
    the CPU gets through the parameter, stability and compiled-kernel checks and
    stops only at the device allocation (MS_ERR_OOM without a GPU)."""
    from paper_2404_01035_gb300 import _binding as B
    s = I.read_infile(os.path.join(DECKS, "ternary_2d.in"))
    keep = []
    params = make_params(s, "f64", keep)
    grid = make_grid(s)
    h = ctypes.c_void_p()
    rc = B.lib().ms_create(ctypes.byref(grid), s.n_phases, s.n_components, ctypes.byref(params),
                           None, None, ctypes.byref(h))
    msg = B.lib().ms_last_error(None).decode()
    assert rc == 3 and "allocation" in msg, (rc, msg)
    phi = I.read_filling(os.path.join(DECKS, "ternary_2d.fill"), s)
    assert phi[0].max() == 1.0 and phi[1].max() == 1.0 and phi[2].min() == 0.0
    o = oracle.run(s, phi, np.broadcast_to(I.liquid_mu(s, [0.38, 0.33])[:, None, None, None],
                                            (2,) + phi.shape[1:]).copy(), 40)
    assert np.isfinite(o[0]).all() and np.isfinite(o[1]).all()


class _OracleSim:
    """Stands in for Simulation in the driver's CPU test: the same calls, the
    oracle's step behind them."""
    fail_at = None

    def __init__(self, spec, dtype="f32"):
        self.spec = spec

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False

    def set_fields(self, phi, mu):
        self.phi, self.mu = np.array(phi, dtype=float), np.array(mu, dtype=float)
        self.n, self.t = 0, 0.0

    def step(self, k):
        self.phi, self.mu = oracle.run(self.spec, self.phi, self.mu, k, t0=self.t, step0=self.n)
        self.n += k
        self.t = self.n * self.spec.dt

    def diag(self):
        from paper_2404_01035_gb300._binding import MSError
        if self.fail_at is not None and self.n >= self.fail_at:
            raise MSError(5, "non-finite state")
        return {"mass": self.mu.reshape(self.mu.shape[0], -1).sum(axis=1), "sum_err": 0.0,
                "phi_min": float(self.phi.min()), "phi_max": float(self.phi.max()), "nonfinite": 0.0,
                "step": self.n, "t": self.t}

    def get_fields(self):
        return self.phi.copy(), self.mu.copy()

    def step_moving_frame(self, n, keep, mu_fill, check_every=100):
        self.frame_calls = getattr(self, "frame_calls", []) + [(n, keep, list(mu_fill), check_every)]
        self.step(n)

    def checkpoint(self):
        import pickle
        return pickle.dumps((self.phi, self.mu, self.n, self.t))

    def restore(self, blob):
        import pickle
        self.phi, self.mu, self.n, self.t = pickle.loads(blob)


def test_run_driver_loop_and_snapshots_with_the_oracle_behind_it(tmp_path, monkeypatch, capsys):
    """The driver's stepping, diagnostics and snapshot files, with the GPU
    simulation replaced by the oracle: snapshots every SAVET steps, named by
    step, holding the state the oracle reaches in one run of as many steps."""
    import json
    from paper_2404_01035_gb300 import run, simulation
    monkeypatch.setattr(simulation, "Simulation", _OracleSim)
    deck, fill = os.path.join(DECKS, "ternary_2d.in"), os.path.join(DECKS, "ternary_2d.fill")
    out = tmp_path / "out"
    assert run.main([deck, fill, "--out", str(out)]) == 0
    files = sorted(os.listdir(out))
    assert files == ["step_0000000000.npz", "step_0000000020.npz", "step_0000000040.npz"]
    s = I.read_infile(deck)
    phi0 = I.read_filling(fill, s)
    mu0 = np.broadcast_to(I.liquid_mu(s, [0.38, 0.33])[:, None, None, None], (2,) + phi0.shape[1:]).copy()
    np.testing.assert_array_equal(np.load(out / files[0])["phi"], phi0)
    o_phi, o_mu = oracle.run(s, phi0, mu0, 40)
    last = np.load(out / files[2])
    assert max(np.abs(last["phi"] - o_phi).max(), np.abs(last["mu"] - o_mu).max()) < 1e-14
    assert int(last["step"]) == 40 and float(last["t"]) == pytest.approx(40 * s.dt, rel=1e-12)
    lines = [json.loads(x) for x in capsys.readouterr().out.strip().splitlines()]
    assert [d["step"] for d in lines[1:]] == [20, 40]
    # --steps and --save-every override the deck; a non-finite state ends the run with code 3
    _OracleSim.fail_at = 15
    try:
        assert run.main([deck, fill, "--out", str(tmp_path / "o2"), "--steps", "30", "--save-every", "10"]) == 3
    finally:
        _OracleSim.fail_at = None
    assert sorted(os.listdir(tmp_path / "o2")) == ["step_0000000000.npz", "step_0000000010.npz"]


def test_a_shape_on_the_grid_edge_has_no_interface_there():
    """A box laid on the lower y edge (a solid against the no-flux wall) is full up
    to the wall; its profile sits only at its free top and sides."""
    s = I.read_infile(os.path.join(DECKS, "ternary_2d.in"))
    phi = I.read_filling("FILLCUBE = {1, 20, 0, 0, 35, 9, 0};", s)
    col = phi[1, 0, :, 27]                  # through the box, along y
    assert col[0] == 1.0 and col[4] == 1.0   # no diffuse layer at the wall
    assert 0.0 < col[9] < 1.0
    assert col[9] > col[10] > col[11]
    row = phi[1, 0, 2, :]                   # along x: the box's sides are diffuse
    assert 0.0 < row[20] < 1.0 and 0.0 < row[35] < 1.0 and row[27] == 1.0


def _read_vtk(path):
    """A reader for the legacy VTK files the driver writes (header lines, then
    one big-endian FP64 block per scalar)."""
    data = open(path, "rb").read()
    pos, header, fields = 0, {}, {}

    def line():
        nonlocal pos
        end = data.index(b"\n", pos)
        s = data[pos:end].decode()
        pos = end + 1
        return s

    assert line().startswith("# vtk DataFile")
    header["title"] = line()
    assert line() == "BINARY" and line() == "DATASET STRUCTURED_POINTS"
    header["dims"] = [int(v) for v in line().split()[1:]]
    header["origin"] = [float(v) for v in line().split()[1:]]
    header["spacing"] = [float(v) for v in line().split()[1:]]
    n = int(line().split()[1])
    while pos < len(data):
        name = line().split()[1]
        assert line() == "LOOKUP_TABLE default"
        fields[name] = np.frombuffer(data[pos:pos + 8 * n], dtype=">f8")
        pos += 8 * n + 1
    return header, fields


def test_run_driver_writes_vtk_snapshots(tmp_path, monkeypatch):
    from paper_2404_01035_gb300 import run, simulation
    monkeypatch.setattr(simulation, "Simulation", _OracleSim)
    deck, fill = os.path.join(DECKS, "ternary_2d.in"), os.path.join(DECKS, "ternary_2d.fill")
    out = tmp_path / "vtk"
    assert run.main([deck, fill, "--out", str(out), "--format", "vtk", "--steps", "20"]) == 0
    assert sorted(os.listdir(out)) == ["step_0000000000.vtk", "step_0000000020.vtk"]
    head, fields = _read_vtk(out / "step_0000000020.vtk")
    s = I.read_infile(deck)
    assert head["dims"] == [56, 40, 1] and head["spacing"] == [1.0, 1.0, 1.0] and head["origin"] == [0.5] * 3
    assert list(fields) == ["phi_alpha", "phi_beta", "phi_liquid", "mu_0", "mu_1"]
    phi0 = I.read_filling(fill, s)
    mu0 = np.broadcast_to(I.liquid_mu(s, [0.38, 0.33])[:, None, None, None], (2,) + phi0.shape[1:]).copy()
    o_phi, o_mu = oracle.run(s, phi0, mu0, 20)
    np.testing.assert_array_equal(fields["phi_beta"], o_phi[1].ravel())   # x fastest, as the array
    np.testing.assert_array_equal(fields["mu_1"], o_mu[1].ravel())


def test_single_names_and_improper_rotations():
    s = I.read_infile(TERNARY_3D.replace("PHASES = {alpha, beta, liquid};", "PHASES = solid;"))
    assert s.meta["phases"] == ["solid"]
    s.rot[0, 1] = s.rot[1, 0] = np.diag([1.0, 1.0, -1.0])          # a mirror, not a rotation
    with pytest.raises(ValueError, match="proper rotation"):
        I.write_infile(s)


def test_run_driver_checkpoint_and_restart(tmp_path, monkeypatch):
    """A run stopped at step 20 with --checkpoint and resumed with --restart ends
    where an uninterrupted run ends (the oracle standing in for the GPU)."""
    from paper_2404_01035_gb300 import run, simulation
    monkeypatch.setattr(simulation, "Simulation", _OracleSim)
    deck, fill = os.path.join(DECKS, "ternary_2d.in"), os.path.join(DECKS, "ternary_2d.fill")
    a, b = tmp_path / "a", tmp_path / "b"
    assert run.main([deck, fill, "--out", str(a), "--steps", "20", "--checkpoint"]) == 0
    assert (a / "checkpoint.bin").exists()
    assert run.main([deck, "--restart", str(a / "checkpoint.bin"), "--out", str(b), "--steps", "40"]) == 0
    assert sorted(os.listdir(b)) == ["step_0000000040.npz"]
    s = I.read_infile(deck)
    phi0 = I.read_filling(fill, s)
    mu0 = np.broadcast_to(I.liquid_mu(s, [0.38, 0.33])[:, None, None, None], (2,) + phi0.shape[1:]).copy()
    o_phi, o_mu = oracle.run(s, phi0, mu0, 40)
    last = np.load(b / "step_0000000040.npz")
    np.testing.assert_array_equal(last["phi"], o_phi)
    np.testing.assert_array_equal(last["mu"], o_mu)
    with pytest.raises(SystemExit):
        run.main([deck, "--out", str(b)])                       # neither a filling nor a restart
    with pytest.raises(SystemExit):
        run.main([deck, fill, "--restart", str(a / "checkpoint.bin")])   # both


def test_run_driver_moving_frame_from_the_shift_keys(tmp_path, monkeypatch, capsys):
    """Shift = 1, Shiftj = j in the deck: the driver steps in the moving frame that
    keeps the front at j, refilling with liquid of the alloy's chemical potential."""
    import json
    from paper_2404_01035_gb300 import run, simulation
    made = []

    class Sim(_OracleSim):
        def __init__(self, spec, dtype="f32"):
            super().__init__(spec, dtype)
            made.append(self)

    monkeypatch.setattr(simulation, "Simulation", Sim)
    deck = open(os.path.join(DECKS, "ternary_2d.in")).read() + "Shift = 1;\nShiftj = 24;\n"
    (tmp_path / "shift.in").write_text(deck)
    fill = os.path.join(DECKS, "ternary_2d.fill")
    assert run.main([str(tmp_path / "shift.in"), fill, "--out", str(tmp_path / "o"), "--steps", "40"]) == 0
    s = I.read_infile(deck)
    mu = list(I.liquid_mu(s, [0.38, 0.33]))
    assert made[0].frame_calls == [(20, 24, mu, 20), (20, 24, mu, 20)]
    info = json.loads(capsys.readouterr().out.strip().splitlines()[0])["inputs"]
    assert info["moving_frame"] == {"on": True, "keep": 24}


def test_spec_copies_like_the_workload_problem():
    """The slab decomposition derives each slab's problem with copy(); a spec
    read from a deck supports the same call."""
    s = I.read_infile(TERNARY_3D)
    sub = s.copy(nz=3, bc=[s.bc[0], s.bc[1], 16], phi0=None, mu0=None, meta={**s.meta, "z_origin": 5})
    assert (sub.nz, sub.bc, sub.meta["z_origin"], s.nz) == (3, [3, 1, 16], 5, 8)
    assert make_grid(sub).z_origin == 5 and make_grid(sub).nz == 3


def test_elasticity_survives_writing_and_reading():
    p = W.small_multiphase(n=8, dim=3, N=3, NM=2)
    p.f0 = np.zeros(3)
    C = np.zeros((6, 6))
    C[:3, :3] = 1.2
    C[np.arange(3), np.arange(3)] = 3.0
    C[3, 3] = C[4, 4] = C[5, 5] = 0.9
    E = np.zeros((3, 3, 3))
    E[0] = [[0.01, 0.002, 0.0], [0.002, 0.01, 0.001], [0.0, 0.001, 0.012]]
    p.elastic_C, p.eigenstrain = C, E
    text = I.write_infile(p)
    assert "VOIGT_CUBIC = {0, 3.0, 1.2, 0.9};" in text
    s = I.read_infile(text, elasticity=True)
    np.testing.assert_array_equal(s.elastic_C, C)
    np.testing.assert_array_equal(s.eigenstrain, E)
    a = oracle.run(p, p.phi0, p.mu0, 2)
    b = oracle.run(s, p.phi0, p.mu0, 2)
    assert max(np.abs(a[0] - b[0]).max(), np.abs(a[1] - b[1]).max()) < 1e-13
    T = C.copy()
    T[2, 2], T[5, 5] = 2.5, 0.7                                  # tetragonal
    p.elastic_C = T
    np.testing.assert_array_equal(I.read_infile(I.write_infile(p), elasticity=True).elastic_C, T)
    T[0, 3] = 0.1                                                # neither form
    p.elastic_C = T
    with pytest.raises(ValueError, match="Voigt form"):
        I.write_infile(p)


def test_graingrowth_key():
    assert I.read_infile(TERNARY_3D).grain_growth == 0
    s = I.read_infile(TERNARY_3D + "GRAINGROWTH = 1;\n")
    assert s.grain_growth == 1
    assert I.read_infile(I.write_infile(s)).grain_growth == 1


def test_boundary_values_on_periodic_axes_are_not_used():
    s = I.read_infile(TERNARY_3D.replace("BOUNDARY_VALUE = {phi, 0, 0, 0, 0, 0, 0};",
                                         "BOUNDARY_VALUE = {phi, 0.3, 0.3, 0, 0, 0.2, 0.2};"))
    assert s.bc == [3, 1, 3]
