"""Readers and a writer for the paper's input files (Sec. "Input files").

The paper's solvers take their parameters from a text file of `KEY = value;`
lines (`#` starts a comment; a value is a scalar, a word, or a `{...}` list;
some keys repeat, one line per phase or pair), and their initial condition
from a filling file of FILLCUBE / FILLCYLINDER / FILLSPHERE / FILLELLIPSE
lines.  This module maps both onto the library's inputs:

* `read_infile` returns a `ModelSpec`, the grid and parameters in the form
  `Simulation` takes (every key it uses is listed in `_USED`; the rest are
  recorded in `spec.meta["ignored"]`);
* `write_infile` writes a spec back in the same format;
* `read_filling` paints the filling file's shapes into phi, sharp or with
  the 1-D equilibrium profile of the spec's potential across each shape's
  boundary.

The infile format keeps the paper's key names and list orders.  Where the
paper leaves a detail open, the reading taken is stated beside the key.
Input the library does not implement is refused with a ValueError rather than
silently changed: CALPHAD free energies (Function_F != 1), Dirichlet / free /
"complex" boundaries, different codes on the two faces of one axis, a
non-uniform grid spacing, an anisotropy other than four-fold, and (with
elasticity on) stiffnesses that differ between phases.
"""
from __future__ import annotations

import math
import os
import re
from dataclasses import dataclass, field, replace
from typing import Dict, List, Optional, Union

import numpy as np

BC_NOFLUX, BC_PERIODIC = 1, 3

Scalar = Union[float, str]


# ------------------------------------------------------------------ parsing
def _token(t: str) -> Scalar:
    t = t.strip().strip('"').strip("'")
    try:
        return float(t)
    except ValueError:
        return t


def parse(text: str) -> Dict[str, List[Union[Scalar, List[Scalar]]]]:
    """`KEY = value;` lines -> {KEY: [value of each occurrence, in order]}.

    A `{a, b, ...}` value becomes a list (empty for `{}`); numbers become
    floats, anything else stays a string.  Keys keep their case (the paper
    has both `tau` and `Tau`)."""
    out: Dict[str, list] = {}
    body = "\n".join(line.split("#", 1)[0] for line in text.splitlines())
    for stmt in body.split(";"):
        stmt = stmt.strip()
        if not stmt:
            continue
        if "=" not in stmt:
            raise ValueError(f"not a KEY = value statement: {stmt!r}")
        key, val = (s.strip() for s in stmt.split("=", 1))
        if not re.fullmatch(r"[A-Za-z_][A-Za-z0-9_]*", key):
            raise ValueError(f"bad key {key!r}")
        if val.startswith("{"):
            if not val.endswith("}"):
                raise ValueError(f"unclosed list for {key}: {val!r}")
            inner = val[1:-1].strip()
            v = [] if not inner else [_token(x) for x in inner.split(",")]
        else:
            v = _token(val)
        out.setdefault(key, []).append(v)
    return out


# ------------------------------------------------------------------ the spec
@dataclass
class ModelSpec:
    """Grid, parameters and options of one simulation, in the attribute form
    `Simulation` (and the batched and sharded forms) read."""

    dim: int
    nx: int
    ny: int
    nz: int
    n_phases: int
    n_components: int
    bc: List[int]
    dx: float
    dt: float
    eps: float
    tau: float
    potential: str
    gamma: np.ndarray
    delta: np.ndarray
    rot: np.ndarray
    gamma3: Optional[np.ndarray]
    D: np.ndarray
    A: np.ndarray
    ceq: np.ndarray
    slopes: np.ndarray
    f0: np.ndarray
    T_ref: float = 0.0
    T0: float = 0.0
    G: float = 0.0
    z0: float = 0.0
    V: float = 0.0
    steps: int = 0
    noise_amp: float = 0.0
    noise_seed: int = 0
    anti_trapping: int = 0
    grain_growth: int = 0
    elastic_C: Optional[np.ndarray] = None
    eigenstrain: Optional[np.ndarray] = None
    phi0: Optional[np.ndarray] = None   # an initial state may ride along (read_filling fills none in)
    mu0: Optional[np.ndarray] = None
    meta: dict = field(default_factory=dict)

    @property
    def n_mu(self) -> int:
        return self.n_components - 1

    def copy(self, **kw) -> "ModelSpec":
        """A copy with the given fields replaced (the slab decomposition makes
        its sub-domains this way)."""
        return replace(self, **kw)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz


# keys the reader maps onto the spec
_USED = {
    "DIMENSION", "MESH_X", "MESH_Y", "MESH_Z", "DELTA_X", "DELTA_Y", "DELTA_Z", "DELTA_t",
    "NUMPHASES", "NUMCOMPONENTS", "NTIMESTEPS", "GAMMA", "DIFFUSIVITY", "BOUNDARY",
    "BOUNDARY_VALUE", "epsilon", "tau", "Function_anisotropy", "Anisotropy_type", "dab",
    "Rotation_matrix", "Function_W", "Gamma_abc", "ISOTHERMAL", "T", "Tempgrady",
    "Equilibrium_temperature", "Function_F", "A", "ceq", "slopes", "Noise_phasefield",
    "Amp_Noise_Phase", "EIGEN_STRAIN", "VOIGT_ISOTROPIC", "VOIGT_CUBIC", "VOIGT_TETRAGONAL",
    "COMPONENTS", "PHASES", "cfill", "SAVET", "Shift", "Shiftj", "GRAINGROWTH",
}


def _one(kv, key, default=None, required=True):
    if key not in kv:
        if required and default is None:
            raise ValueError(f"missing key {key}")
        return default
    return kv[key][-1]


def _num(kv, key, default=None):
    v = _one(kv, key, default)
    if isinstance(v, list) or isinstance(v, str):
        raise ValueError(f"{key} must be a number, got {v!r}")
    return float(v)


def _pairs(N):
    """Pairs (a, b), a < b, in the order GAMMA and dab list them: 12, 13, ..., 23, ..."""
    return [(a, b) for a in range(N) for b in range(a + 1, N)]


def _triples(N):
    return [(a, b, c) for a in range(N) for b in range(a + 1, N) for c in range(b + 1, N)]


def _pair_matrix(vals, N, key):
    P = _pairs(N)
    vals = [float(v) for v in vals]
    if len(vals) == 1 and len(P) > 1:
        vals = vals * len(P)          # one value for every pair
    if len(vals) != len(P):
        raise ValueError(f"{key} needs {len(P)} pair values (12, 13, ..., 23, ...), got {len(vals)}")
    M = np.zeros((N, N))
    for (a, b), v in zip(P, vals):
        M[a, b] = M[b, a] = v
    return M


def euler_rotation(ax: float, ay: float, az: float) -> np.ndarray:
    """R = Rz(az) Ry(ay) Rx(ax), angles in degrees (rotation about x first).
    q' = R q is the pair's interface normal in its crystal frame (Eq. aniso_eqn);
    on a 2-D grid only az acts, as the in-plane rotation."""
    x, y, z = (math.radians(v) for v in (ax, ay, az))
    Rx = np.array([[1, 0, 0], [0, math.cos(x), -math.sin(x)], [0, math.sin(x), math.cos(x)]])
    Ry = np.array([[math.cos(y), 0, math.sin(y)], [0, 1, 0], [-math.sin(y), 0, math.cos(y)]])
    Rz = np.array([[math.cos(z), -math.sin(z), 0], [math.sin(z), math.cos(z), 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def _phase(v, N, key) -> int:
    a = int(v)
    if a != v or not 0 <= a < N:
        raise ValueError(f"{key}: phase index {v!r} is not one of 0..{N - 1}")
    return a


def _names(v):
    return [] if v is None else [str(x) for x in (v if isinstance(v, list) else [v])]


def _sym_from_list(vals, n, key):
    """[diag_1..diag_n, off_12, off_13, ..., off_23, ...] -> symmetric n x n."""
    off = [(i, j) for i in range(n) for j in range(i + 1, n)]
    if len(vals) != n + len(off):
        raise ValueError(f"{key} needs {n} diagonal and {len(off)} off-diagonal values, got {len(vals)}")
    M = np.diag([float(v) for v in vals[:n]])
    for (i, j), v in zip(off, vals[n:]):
        M[i, j] = M[j, i] = float(v)
    return M


def _axis_codes(kv, dim):
    """BOUNDARY = {field, X+, X-, Y+, Y-, Z+, Z-} (or fewer faces) -> one code per
    axis.  phi, mu and c must agree (the library applies one rule per axis to
    the whole state); T is frozen and its entry is not used."""
    codes = None
    for entry in kv.get("BOUNDARY", []):
        if not isinstance(entry, list) or len(entry) < 3:
            raise ValueError(f"BOUNDARY entry {entry!r}: expected {{field, X+, X-, ...}}")
        name = str(entry[0])
        if name == "T":
            continue
        faces = [int(v) for v in entry[1:]]
        axes = []
        for d in range(dim):
            if 2 * d + 1 >= len(faces):
                raise ValueError(f"BOUNDARY {name}: no codes for axis {'xyz'[d]}")
            hi, lo = faces[2 * d], faces[2 * d + 1]
            if hi != lo:
                raise ValueError(f"BOUNDARY {name}: the two faces of axis {'xyz'[d]} differ ({hi}, {lo})")
            if hi not in (BC_NOFLUX, BC_PERIODIC):
                raise ValueError(f"BOUNDARY {name}: code {hi} on axis {'xyz'[d]} is not supported "
                                 "(1 = no-flux and 3 = periodic are)")
            axes.append(hi)
        if codes is not None and axes != codes:
            raise ValueError(f"BOUNDARY {name}: codes {axes} differ from the other fields' {codes}")
        codes = axes
    if codes is None:
        codes = [BC_PERIODIC] * dim
    # BOUNDARY_VALUE = {field, X+, X-, ...}: a no-flux face takes zero flux only
    for entry in kv.get("BOUNDARY_VALUE", []):
        if not isinstance(entry, list) or len(entry) < 2 or str(entry[0]) == "T":
            continue
        vals = [float(v) for v in entry[1:]]
        for d in range(dim):
            if codes[d] == BC_NOFLUX and any(vals[i] != 0.0 for i in (2 * d, 2 * d + 1) if i < len(vals)):
                raise ValueError(f"BOUNDARY_VALUE {entry[0]}: a non-zero flux on axis {'xyz'[d]} is not "
                                 "supported (no-flux faces take zero flux)")
    return codes + [BC_PERIODIC] * (3 - dim)


def _stiffness(kv, N):
    """VOIGT_ISOTROPIC / VOIGT_CUBIC = {phase, c11, c12, c44},
    VOIGT_TETRAGONAL = {phase, c11, c12, c13, c33, c44, c66} -> one 6x6 Voigt
    matrix (every phase must give the same: the library's stiffness is
    homogeneous)."""
    Cs = {}
    for key in ("VOIGT_ISOTROPIC", "VOIGT_CUBIC", "VOIGT_TETRAGONAL"):
        for e in kv.get(key, []):
            a = _phase(e[0], N, key)
            v = [float(x) for x in e[1:]]
            if len(v) != (6 if key == "VOIGT_TETRAGONAL" else 3):
                raise ValueError(f"{key} entry {e!r} has the wrong number of constants")
            C = np.zeros((6, 6))
            if key == "VOIGT_TETRAGONAL":
                c11, c12, c13, c33, c44, c66 = v
                C[0, 0] = C[1, 1] = c11
                C[2, 2] = c33
                C[0, 1] = C[1, 0] = c12
                C[0, 2] = C[2, 0] = C[1, 2] = C[2, 1] = c13
                C[3, 3] = C[4, 4] = c44
                C[5, 5] = c66
            else:
                c11, c12, c44 = v
                C[:3, :3] = c12
                for i in range(3):
                    C[i, i] = c11
                    C[3 + i, 3 + i] = c44
            Cs[a] = C
    if not Cs:
        raise ValueError("elasticity needs a VOIGT_ISOTROPIC, VOIGT_CUBIC or VOIGT_TETRAGONAL entry")
    ref = next(iter(Cs.values()))
    for a, C in Cs.items():
        if not np.allclose(C, ref, rtol=1e-12, atol=0.0):
            raise ValueError("the phases' stiffnesses differ; the library's elasticity takes one "
                             "homogeneous stiffness")
    return ref


def _eigenstrain(kv, N):
    """EIGEN_STRAIN = {phase, e_xx, e_yy, e_zz, e_yz, e_xz, e_xy} (tensor
    components) -> [N][3][3]; phases without an entry have none."""
    E = np.zeros((N, 3, 3))
    for e in kv.get("EIGEN_STRAIN", []):
        if len(e) != 7:
            raise ValueError(f"EIGEN_STRAIN entry {e!r}: expected {{phase, xx, yy, zz, yz, xz, xy}}")
        a = _phase(e[0], N, "EIGEN_STRAIN")
        xx, yy, zz, yz, xz, xy = (float(v) for v in e[1:7])
        E[a] = [[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]]
    return E


def read_infile(src: str, *, free_energy: Optional[str] = None, elasticity: bool = False,
                anti_trapping: bool = False, grain_growth: bool = False,
                noise_seed: int = 0) -> ModelSpec:
    """Map an infile (a path or its text) onto a ModelSpec.

    The options switch on what the paper selects elsewhere than in the infile
    keys read here: `elasticity` (then VOIGT_* and EIGEN_STRAIN are used),
    `anti_trapping`, and `grain_growth` (which the key GRAINGROWTH = 1 also
    turns on).  `free_energy="parabolic"` reads the
    parabolic coefficients A, ceq, slopes of a file whose Function_F names a
    CALPHAD database (which the library does not evaluate)."""
    text = open(src).read() if os.path.exists(src) else src
    kv = parse(text)
    dim = int(_num(kv, "DIMENSION"))
    if dim not in (2, 3):
        raise ValueError(f"DIMENSION must be 2 or 3, got {dim}")
    nx, ny = int(_num(kv, "MESH_X")), int(_num(kv, "MESH_Y"))
    nz = int(_num(kv, "MESH_Z", 1.0)) if dim == 3 else 1
    dx = _num(kv, "DELTA_X")
    for k in ("DELTA_Y",) + (("DELTA_Z",) if dim == 3 else ()):
        if k in kv and not math.isclose(_num(kv, k), dx, rel_tol=1e-12):
            raise ValueError(f"{k} differs from DELTA_X: the library's grid spacing is uniform")
    N = int(_num(kv, "NUMPHASES"))
    K = int(_num(kv, "NUMCOMPONENTS"))
    NM = K - 1
    if N < 2 or NM < 1:
        raise ValueError("NUMPHASES must be >= 2 and NUMCOMPONENTS >= 2")
    ff = int(_num(kv, "Function_F", 1.0))
    if ff != 1 and free_energy != "parabolic":
        raise ValueError(f"Function_F = {ff} needs a CALPHAD database; pass free_energy='parabolic' "
                         "to use the file's parabolic coefficients (A, ceq, slopes) instead")

    gamma = _pair_matrix(_one(kv, "GAMMA"), N, "GAMMA")
    aniso = int(_num(kv, "Function_anisotropy", 0.0))
    delta = np.zeros((N, N))
    if aniso:
        if int(_num(kv, "Anisotropy_type", 4.0)) != 4:
            raise ValueError("only the four-fold anisotropy (Anisotropy_type = 4) is supported")
        delta = _pair_matrix(_one(kv, "dab"), N, "dab")
    rot = np.broadcast_to(np.eye(3), (N, N, 3, 3)).copy()
    for e in kv.get("Rotation_matrix", []):
        if len(e) != 5:
            raise ValueError(f"Rotation_matrix entry {e!r}: expected {{a, b, ax, ay, az}}")
        a, b = _phase(e[0], N, "Rotation_matrix"), _phase(e[1], N, "Rotation_matrix")
        if a == b:
            raise ValueError("Rotation_matrix: a pair needs two different phases")
        R = euler_rotation(*(float(v) for v in e[2:5]))
        rot[a, b] = rot[b, a] = R
    gamma3 = None
    g3 = kv.get("Gamma_abc", [[]])[-1]
    if g3:
        T3 = _triples(N)
        vals = [float(v) for v in g3]
        if len(vals) == 1 and len(T3) > 1:
            vals = vals * len(T3)
        if len(vals) != len(T3):
            raise ValueError(f"Gamma_abc needs {len(T3)} triple values (123, 124, ...), got {len(vals)}")
        gamma3 = np.zeros((N, N, N))
        for (a, b, c), v in zip(T3, vals):
            for p in ((a, b, c), (a, c, b), (b, a, c), (b, c, a), (c, a, b), (c, b, a)):
                gamma3[p] = v

    D = np.zeros((N, NM, NM))
    for e in kv.get("DIFFUSIVITY", []):
        diag, a = int(e[0]), _phase(e[1], N, "DIFFUSIVITY")
        vals = e[2:]
        if diag:
            if len(vals) != NM:
                raise ValueError(f"DIFFUSIVITY of phase {a}: {NM} diagonal values expected")
            D[a] = np.diag([float(v) for v in vals])
        else:
            D[a] = _sym_from_list(vals, NM, f"DIFFUSIVITY of phase {a}")
    A = np.zeros((N, NM, NM))
    for e in kv.get("A", []):
        a = _phase(e[0], N, "A")
        M = _sym_from_list(e[1:], NM, f"A of phase {a}") if len(e) - 1 > NM else np.diag([float(v) for v in e[1:]])
        A[a] = np.triu(M)             # the parabolic form uses A_ij with i <= j
    ceq = np.zeros((N, NM))
    slopes = np.zeros((N, NM))
    for key, out in (("ceq", ceq), ("slopes", slopes)):
        for e in kv.get(key, []):
            a, b = _phase(e[0], N, key), _phase(e[1], N, key)
            if len(e) != 2 + NM:
                raise ValueError(f"{key} entry {e!r}: expected {{a, b}} and {NM} values")
            if a == b:                # phase a's own value; the {a, b != a} entries repeat the liquid's
                out[a] = [float(v) for v in e[2:2 + NM]]

    T_ref = _num(kv, "Equilibrium_temperature", 0.0)
    T0 = G = z0 = V = 0.0
    isothermal = int(_num(kv, "ISOTHERMAL", 0.0))
    if "Tempgrady" in kv and not isothermal:
        tg = _one(kv, "Tempgrady")
        if not isinstance(tg, list) or len(tg) != 5:
            raise ValueError("Tempgrady needs {BASETEMP, DELTAT, DISTANCE, OFFSET, VELOCITY}")
        base, dT, dist, off, vel = (float(v) for v in tg)
        if dist == 0.0:
            raise ValueError("Tempgrady: DISTANCE must not be 0")
        # T = BASETEMP + (DELTAT / DISTANCE) (s - OFFSET - VELOCITY t), s along the grid's last axis
        T0, G, z0, V = base, dT / dist, off, vel
    else:
        T0 = _num(kv, "T", T_ref)

    spec = ModelSpec(
        dim=dim, nx=nx, ny=ny, nz=nz, n_phases=N, n_components=K, bc=_axis_codes(kv, dim), dx=dx,
        dt=_num(kv, "DELTA_t"), eps=_num(kv, "epsilon"), tau=_num(kv, "tau"),
        potential="obstacle" if int(_num(kv, "Function_W", 1.0)) == 1 else "well",
        gamma=gamma, delta=delta, rot=rot, gamma3=gamma3, D=D, A=A, ceq=ceq, slopes=slopes,
        f0=np.zeros(N), T_ref=T_ref, T0=T0, G=G, z0=z0, V=V,
        steps=int(_num(kv, "NTIMESTEPS", 0.0)),
        anti_trapping=int(bool(anti_trapping)),
        grain_growth=int(bool(grain_growth) or bool(int(_num(kv, "GRAINGROWTH", 0.0)))),
        noise_seed=int(noise_seed))
    if int(_num(kv, "Function_W", 1.0)) not in (1, 2):
        raise ValueError("Function_W must be 1 (obstacle) or 2 (well)")
    if int(_num(kv, "Noise_phasefield", 0.0)):
        spec.noise_amp = _num(kv, "Amp_Noise_Phase", 0.0)
    if elasticity:
        spec.elastic_C = _stiffness(kv, N)
        spec.eigenstrain = _eigenstrain(kv, N)
    cfill = {}
    for e in kv.get("cfill", []):
        if int(e[0]) == int(e[1]):    # phase a's own fill composition, like ceq
            cfill[int(e[0])] = [float(v) for v in e[2:2 + NM]]
    spec.meta = {
        "cfill": cfill,
        "savet": int(_num(kv, "SAVET", 0.0)),
        # moving frame (SHIFT): on, and the index along the last axis the front is kept at
        "shift": int(_num(kv, "Shift", 0.0)),
        "shiftj": int(_num(kv, "Shiftj", 0.0)),
        "phases": _names(_one(kv, "PHASES", [], required=False)),
        "components": _names(_one(kv, "COMPONENTS", [], required=False)),
        "ignored": sorted(k for k in kv if k not in _USED),
    }
    return spec


# ------------------------------------------------------------------ writing
def _fmt(v) -> str:
    if isinstance(v, str):
        return v
    if isinstance(v, (int, np.integer)):
        return str(int(v))          # phase indices and flags
    return repr(float(v))


def _list(vals) -> str:
    return "{" + ", ".join(_fmt(v) for v in vals) + "}"


def write_infile(spec) -> str:
    """The spec (any object with ModelSpec's attributes) as an infile that
    `read_infile` maps back onto the same spec."""
    N, NM = int(spec.n_phases), int(spec.n_components) - 1
    L = [f"DIMENSION = {int(spec.dim)};", f"MESH_X = {int(spec.nx)};", f"MESH_Y = {int(spec.ny)};",
         f"MESH_Z = {int(spec.nz) if spec.dim == 3 else 1};", f"DELTA_X = {_fmt(spec.dx)};",
         f"DELTA_Y = {_fmt(spec.dx)};", f"DELTA_Z = {_fmt(spec.dx)};", f"DELTA_t = {_fmt(spec.dt)};",
         f"NUMPHASES = {N};", f"NUMCOMPONENTS = {NM + 1};",
         f"NTIMESTEPS = {int(getattr(spec, 'steps', 0))};",
         f"GAMMA = {_list(spec.gamma[a, b] for a, b in _pairs(N))};"]
    for a in range(N):
        off = [spec.D[a, i, j] for i in range(NM) for j in range(i + 1, NM)]
        L.append(f"DIFFUSIVITY = {_list([0, a] + [spec.D[a, i, i] for i in range(NM)] + off)};")
    bc = list(spec.bc)[: spec.dim]
    faces = [c for c in bc for _ in (0, 1)]
    for name in ("phi", "mu", "c"):
        L.append(f"BOUNDARY = {{{name}, " + ", ".join(str(int(c)) for c in faces) + "};")
    delta = np.asarray(spec.delta)
    L += [f"epsilon = {_fmt(spec.eps)};", f"tau = {_fmt(spec.tau)};",
          f"Function_anisotropy = {int(bool(np.any(delta != 0)))};", "Anisotropy_type = 4;",
          f"dab = {_list(delta[a, b] for a, b in _pairs(N))};"]
    rot = np.asarray(spec.rot) if spec.rot is not None else None
    for a, b in _pairs(N):
        if rot is not None and not np.allclose(rot[a, b], np.eye(3), atol=0.0, rtol=0.0):
            ax, ay, az = _euler_angles(rot[a, b])
            L.append(f"Rotation_matrix = {_list([a, b, ax, ay, az])};")
    L.append(f"Function_W = {1 if spec.potential == 'obstacle' else 2};")
    g3 = getattr(spec, "gamma3", None)
    L.append("Gamma_abc = " + (_list(g3[t] for t in _triples(N)) if g3 is not None else "{}") + ";")
    L += ["ISOTHERMAL = 0;", f"Equilibrium_temperature = {_fmt(spec.T_ref)};", f"T = {_fmt(spec.T0)};"]
    if spec.G != 0.0 or spec.V != 0.0 or spec.z0 != 0.0:
        L.append(f"Tempgrady = {_list([spec.T0, spec.G, 1.0, spec.z0, spec.V])};")
    L.append("Function_F = 1;")
    for a in range(N):
        off = [spec.A[a, i, j] for i in range(NM) for j in range(i + 1, NM)]
        L.append(f"A = {_list([a] + [spec.A[a, i, i] for i in range(NM)] + off)};")
    for key, arr in (("ceq", spec.ceq), ("slopes", spec.slopes)):
        for a in range(N):
            L.append(f"{key} = {_list([a, a] + list(np.asarray(arr)[a]))};")
    if getattr(spec, "noise_amp", 0.0):
        L += ["Noise_phasefield = 1;", f"Amp_Noise_Phase = {_fmt(spec.noise_amp)};"]
    if getattr(spec, "grain_growth", 0):
        L.append("GRAINGROWTH = 1;")
    C = getattr(spec, "elastic_C", None)
    if C is not None:
        key, vals = _voigt_form(np.asarray(C, dtype=float))
        E = np.asarray(spec.eigenstrain, dtype=float)
        for a in range(N):
            L.append(f"{key} = {_list([a] + vals)};")
            L.append(f"EIGEN_STRAIN = {_list([a, E[a, 0, 0], E[a, 1, 1], E[a, 2, 2], E[a, 1, 2], E[a, 0, 2], E[a, 0, 1]])};")
    return "\n".join(L) + "\n"


def _voigt_form(C: np.ndarray):
    """The stiffness as the infile's VOIGT_CUBIC or VOIGT_TETRAGONAL constants
    (the forms the reader takes); any other 6x6 matrix is refused."""
    z = C.copy()
    c11, c12, c13, c33, c44, c66 = C[0, 0], C[0, 1], C[0, 2], C[2, 2], C[3, 3], C[5, 5]
    for i, j in ((0, 0), (1, 1), (2, 2), (0, 1), (1, 0), (0, 2), (2, 0), (1, 2), (2, 1), (3, 3), (4, 4), (5, 5)):
        z[i, j] = 0.0
    tetragonal = (C[1, 1] == c11 and C[1, 0] == c12 and C[2, 0] == C[1, 2] == C[2, 1] == c13
                  and C[4, 4] == c44 and not np.any(z))
    if tetragonal and c13 == c12 and c33 == c11 and c66 == c44:
        return "VOIGT_CUBIC", [c11, c12, c44]
    if tetragonal:
        return "VOIGT_TETRAGONAL", [c11, c12, c13, c33, c44, c66]
    raise ValueError("the stiffness has neither the cubic nor the tetragonal Voigt form the infile can hold")


def _euler_angles(R: np.ndarray):
    """Angles (degrees) with euler_rotation(ax, ay, az) == R (R a proper rotation)."""
    R = np.asarray(R, dtype=float)
    if not (np.allclose(R @ R.T, np.eye(3), atol=1e-10) and np.linalg.det(R) > 0):
        raise ValueError("a pair's matrix is not a proper rotation: it has no Euler angles")
    ay = math.asin(max(-1.0, min(1.0, -R[2, 0])))
    if abs(math.cos(ay)) > 1e-12:
        ax = math.atan2(R[2, 1], R[2, 2])
        az = math.atan2(R[1, 0], R[0, 0])
    else:                             # gimbal lock: put the whole turn in ax
        az = 0.0
        ax = math.atan2(-R[1, 2], R[1, 1])
    return tuple(math.degrees(v) for v in (ax, ay, az))


# ------------------------------------------------------------------ filling
def _profile(u: np.ndarray, potential: str, eps: float) -> np.ndarray:
    """phi across a planar boundary at signed distance u (inside > 0): the
    1-D equilibrium profiles, half a sine period for the obstacle potential
    and a hyperbolic tangent for the well (Sec. 2)."""
    if potential == "obstacle":
        s = np.clip(4.0 * u / (math.pi * eps), -math.pi / 2, math.pi / 2)
        return 0.5 * (1.0 + np.sin(s))
    return 0.5 * (1.0 + np.tanh(3.0 * u / (2.0 * eps)))


def read_filling(src: str, spec, *, diffuse: bool = True, matrix: Optional[int] = None) -> np.ndarray:
    """Paint a filling file's shapes into phi [N][nz][ny][nx].

    Shapes, with positions in cell indices (cell i sits at i):
      FILLCUBE     = {phase, x0, y0, z0, x1, y1, z1}        cells x0..x1 (inclusive), ...
      FILLCYLINDER = {phase, xc, yc, z_start, z_end, radius} axis along z
      FILLSPHERE   = {phase, xc, yc, zc, radius}
      FILLELLIPSE  = {phase, xc, yc, zc, major_axis, eccentricity, angle_deg}
                     (or without zc on a 2-D grid), in the x-y plane
    Later lines paint over earlier ones; cells no shape covers hold the
    matrix phase (default: the last phase, the liquid).  A box side or a
    cylinder end on the grid's edge continues past it, so the edge is no
    interface.  With `diffuse`, each shape's indicator becomes the
    equilibrium profile of the spec's potential in the signed distance to
    its boundary (a box's distance is the box distance), so the interface
    starts near its relaxed width."""
    text = open(src).read() if os.path.exists(src) else src
    kv = parse(text)
    N = int(spec.n_phases)
    nz = int(spec.nz) if spec.dim == 3 else 1
    ny, nx = int(spec.ny), int(spec.nx)
    mat = N - 1 if matrix is None else int(matrix)
    z, y, x = np.meshgrid(np.arange(nz, dtype=float), np.arange(ny, dtype=float), np.arange(nx, dtype=float),
                          indexing="ij")
    eps_cells = float(spec.eps) / float(spec.dx)
    phi = np.zeros((N, nz, ny, nx))
    phi[mat] = 1.0
    order = []
    for line in text.splitlines():
        m = re.match(r"\s*(FILL[A-Z]+)\s*=", line.split("#", 1)[0])
        if m:
            order.append(m.group(1))
    seen = {}
    for key in order:
        e = [float(v) for v in kv[key][seen.get(key, 0)]]
        seen[key] = seen.get(key, 0) + 1
        a = int(e[0])
        if key == "FILLCUBE":
            x0, y0, z0, x1, y1, z1 = e[1:7]
            axes = [(x, x0, x1, nx), (y, y0, y1, ny)] + ([(z, z0, z1, nz)] if spec.dim == 3 else [])
            inside = np.full(x.shape, np.inf)
            excess2 = np.zeros(x.shape)
            for coord, i0, i1, n in axes:
                lo = -np.inf if i0 <= 0 else i0 - 0.5       # a side on the grid's edge continues past it
                hi = np.inf if i1 >= n - 1 else i1 + 0.5
                d = np.minimum(coord - lo, hi - coord)
                inside = np.minimum(inside, d)
                excess2 += np.maximum(-d, 0.0) ** 2
            u = np.where(inside > 0, inside, -np.sqrt(excess2))
        elif key == "FILLCYLINDER":
            xc, yc, zs, ze, r = e[1:6]
            u = r - np.hypot(x - xc, y - yc)
            if spec.dim == 3:
                lo = -np.inf if zs <= 0 else zs - 0.5
                hi = np.inf if ze >= nz - 1 else ze + 0.5
                u = np.minimum(u, np.minimum(z - lo, hi - z))
        elif key == "FILLSPHERE":
            xc, yc, zc, r = e[1:5]
            u = r - np.sqrt((x - xc) ** 2 + (y - yc) ** 2 + ((z - zc) ** 2 if spec.dim == 3 else 0.0))
        elif key == "FILLELLIPSE":
            if len(e) >= 7:
                xc, yc, zc, major, ecc, ang = e[1:7]
            else:
                xc, yc, major, ecc, ang = e[1:6]
            b = major * math.sqrt(max(0.0, 1.0 - ecc * ecc))
            t = math.radians(ang)
            xr = (x - xc) * math.cos(t) + (y - yc) * math.sin(t)
            yr = -(x - xc) * math.sin(t) + (y - yc) * math.cos(t)
            rho = np.sqrt((xr / major) ** 2 + (yr / b) ** 2)
            u = (1.0 - rho) * b          # distance scaled by the minor semi-axis
        else:
            raise ValueError(f"unknown filling key {key}")
        f = _profile(u, spec.potential, eps_cells) if diffuse else (u > 0).astype(float)
        phi *= (1.0 - f)[None]
        phi[a] += f
    return phi


def liquid_mu(spec, c) -> np.ndarray:
    """The chemical potential at which the liquid (the last phase) has
    composition c, for the parabolic free energy f(c) = sum_{i<=j} A_ij c_i c_j
    whose linear and constant coefficients vanish for the liquid (the
    equal-mu / equal-psi reading of Coeff_B, Coeff_C): mu = df/dc."""
    A = np.triu(np.asarray(spec.A, dtype=float)[int(spec.n_phases) - 1])
    return (A + A.T) @ np.asarray(c, dtype=float)
