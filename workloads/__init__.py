"""Seeded synthetic workloads for the grand-potential phase-field step.

This module only *describes* problems: grid, boundary codes, the raw material
inputs the paper's infile carries (GAMMA, dab, Rotation_matrix, DIFFUSIVITY,
A, ceq, slopes, Tempgrady, epsilon, tau, DELTA_t, Function_W) and seeded
initial fields.  It holds none of the time-step arithmetic: both the CPU
oracle and the CUDA library derive every model quantity (B, C, chi, c(mu),
psi, fluxes, projection) from these raw inputs with their own code.

Randomness comes from PCG32 (O'Neill, "PCG: a family of simple fast
space-efficient statistically good algorithms", 2014: 64-bit LCG state,
XSH-RR output), written out here so that every stream is reproducible
bit-for-bit on any host.

Coordinates: cell (i, j, k) has its centre at ((i+1/2)dx, (j+1/2)dx,
(k+1/2)dx).  Arrays are [field][z][y][x] (2-D problems use nz = 1).
Phase N-1 is the liquid, the reference phase of the parabolic free
energies (B^l = C^l = 0 convention of Sec. 3, Eqs. Coeff_B/Coeff_C).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional

import numpy as np

BASE_SEED = 20240401

BC_PERIODIC = 3  # paper boundary code 3
BC_NOFLUX = 1    # paper boundary code 1 (Neumann, zero value)


class PCG32:
    """PCG32 (XSH-RR) generator; seeded like the reference C implementation."""

    MULT = 6364136223846793005
    MASK64 = (1 << 64) - 1

    def __init__(self, seed: int, seq: int = 54):
        self.state = 0
        self.inc = ((seq << 1) | 1) & self.MASK64
        self._step()
        self.state = (self.state + seed) & self.MASK64
        self._step()

    def _step(self):
        self.state = (self.state * self.MULT + self.inc) & self.MASK64

    def next_u32(self) -> int:
        old = self.state
        self._step()
        xorshifted = (((old >> 18) ^ old) >> 27) & 0xFFFFFFFF
        rot = old >> 59
        return ((xorshifted >> rot) | (xorshifted << ((-rot) & 31))) & 0xFFFFFFFF

    def uniform(self) -> float:
        """Uniform double in [0, 1) with 53 random bits."""
        hi = self.next_u32() >> 5
        lo = self.next_u32() >> 6
        return (hi * 67108864.0 + lo) / 9007199254740992.0

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive), by rejection."""
        span = hi - lo + 1
        limit = (1 << 32) - ((1 << 32) % span)
        while True:
            r = self.next_u32()
            if r < limit:
                return lo + (r % span)


@dataclass
class Problem:
    """One simulation: grid, boundary codes, raw model inputs, initial state."""

    name: str
    dim: int
    nx: int
    ny: int
    nz: int
    n_phases: int
    n_components: int
    bc: List[int]                  # per axis x, y, z: BC_PERIODIC or BC_NOFLUX
    dx: float = 1.0
    dt: float = 0.05
    eps: float = 4.0               # epsilon: interface width parameter
    tau: float = 1.0               # relaxation constant (phase mobility = 1/tau)
    potential: str = "obstacle"   # Function_W: "obstacle" (1) or "well" (2)
    gamma: np.ndarray = None       # [N,N] symmetric, GAMMA
    delta: np.ndarray = None       # [N,N] symmetric, dab (0 = isotropic pair)
    rot: np.ndarray = None         # [N,N,3,3] rotation per pair (identity default)
    gamma3: Optional[np.ndarray] = None  # [N,N,N] symmetric, Gamma_abc
    D: np.ndarray = None           # [N,K-1,K-1] diffusivity matrices
    A: np.ndarray = None           # [N,K-1,K-1] parabolic coefficients, i<=j used
    ceq: np.ndarray = None         # [N,K-1] equilibrium compositions at T_ref
    slopes: np.ndarray = None      # [N,K-1] d c_eq / dT
    f0: np.ndarray = None          # [N] constant added to f^alpha (isothermal drive)
    T_ref: float = 0.0
    T0: float = 0.0                # T(z,t) = T0 + G (z - z0 - V t)
    G: float = 0.0
    z0: float = 0.0
    V: float = 0.0
    steps: int = 1
    noise_amp: float = 0.0         # phi noise amplitude (0 = off)
    noise_seed: int = 0
    anti_trapping: int = 0         # 1 = anti-trapping current in the mu update
    grain_growth: int = 0          # 1 = GRAINGROWTH: curvature-driven only, mu held
    active_set: int = 0            # 1 = projection over the locally active phases (sparse grain growth)
    elastic_C: Optional[np.ndarray] = None   # [6,6] Voigt stiffness (homogeneous); None = no elasticity
    eigenstrain: Optional[np.ndarray] = None # [N,3,3] eigenstrain of each phase (tensor components)
    phi0: np.ndarray = None        # [N,nz,ny,nx]
    mu0: np.ndarray = None         # [K-1,nz,ny,nx]
    meta: dict = field(default_factory=dict)

    @property
    def n_mu(self) -> int:
        return self.n_components - 1

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def copy(self, **kw) -> "Problem":
        return replace(self, **kw)


def _default_material(N: int, NM: int):
    gamma = np.ones((N, N)) - np.eye(N)
    delta = np.zeros((N, N))
    rot = np.tile(np.eye(3), (N, N, 1, 1))
    D = np.zeros((N, NM, NM))
    A = np.zeros((N, NM, NM))
    for a in range(N):
        A[a] = np.eye(NM)
    D[N - 1] = np.eye(NM)
    return gamma, delta, rot, D, A


def dt_stab(dim: int, dx: float, tau: float, gamma_max: float, delta_max: float,
            D_max: float) -> float:
    """Explicit stability estimate (dx^2/2d) min(tau/(gamma(1+15 delta)), 1/D)."""
    lim_phi = tau / (gamma_max * (1.0 + 15.0 * delta_max))
    lim_mu = 1.0 / D_max if D_max > 0 else float("inf")
    return dx * dx / (2.0 * dim) * min(lim_phi, lim_mu)


def seed_profile(u: np.ndarray, potential: str) -> np.ndarray:
    """Initial seed shape S(u), u = signed distance / eps (positive inside)."""
    if potential == "obstacle":
        lim = math.pi ** 2 / 8.0
        s = 0.5 * (1.0 + np.sin(4.0 * np.clip(u, -lim, lim) / math.pi))
        return s
    return 0.5 * (1.0 + np.tanh(1.5 * u))


def _centres(n: int, dx: float) -> np.ndarray:
    return (np.arange(n) + 0.5) * dx


def circular_seed(nx: int, ny: int, R: float, eps: float, potential: str,
                  dx: float = 1.0, cx: float = None, cy: float = None) -> np.ndarray:
    """phi_solid of one disc of radius R (cells) centred in a 2-D domain."""
    cx = nx * dx / 2.0 if cx is None else cx
    cy = ny * dx / 2.0 if cy is None else cy
    x = _centres(nx, dx)[None, :]
    y = _centres(ny, dx)[:, None]
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    return seed_profile((R * dx - r) / eps, potential)


def binary_problem(name: str, n: int, *, dim: int = 2, delta: float = 0.0,
                   Delta: float = 0.2, R: float = 10.0, potential: str = "obstacle",
                   dtype_note: str = "f64", steps: int = 1000, eps: float = 4.0,
                   tau: float = 1.0, ny: int = None, nz: int = None,
                   dt: float = None, bc=None) -> Problem:
    """Two phases (solid 0, liquid 1), binary alloy, one central seed.

    AlZn-like compositions from the paper's infile (c_eq^s = 0.926,
    c_eq^l = 0.817, A = 1 for both phases, D^s = 0, D^l = 1); the isothermal
    drive Delta enters as f0^s = -Delta so that psi^l - psi^s = Delta at the
    liquid's equilibrium potential mu_eq = 2 A c_eq^l = 1.634.
    """
    N, NM = 2, 1
    ny = n if ny is None else ny
    nz = (1 if dim == 2 else n) if nz is None else nz
    gamma, dl, rot, D, A = _default_material(N, NM)
    dl[0, 1] = dl[1, 0] = delta
    ceq = np.array([[0.926], [0.817]])
    slopes = np.zeros((N, NM))
    f0 = np.array([-Delta, 0.0])
    if dt is None:
        dt = 0.2 * dt_stab(dim, 1.0, tau, 1.0, delta, 1.0)
    if dim == 2:
        ps = circular_seed(n, ny, R, eps, potential)[None]
    else:
        x = _centres(n, 1.0)[None, None, :]
        y = _centres(ny, 1.0)[None, :, None]
        z = _centres(nz, 1.0)[:, None, None]
        r = np.sqrt((x - n / 2) ** 2 + (y - ny / 2) ** 2 + (z - nz / 2) ** 2)
        ps = seed_profile((R - r) / eps, potential)
    phi0 = np.stack([ps, 1.0 - ps])
    mu0 = np.full((NM, nz, ny, n), 2.0 * 1.0 * 0.817)
    return Problem(name=name, dim=dim, nx=n, ny=ny, nz=nz, n_phases=N, n_components=2,
                   bc=bc or [BC_PERIODIC] * 3, dt=dt, eps=eps, tau=tau, potential=potential,
                   gamma=gamma, delta=dl, rot=rot, D=D, A=A, ceq=ceq, slopes=slopes, f0=f0,
                   steps=steps, phi0=phi0, mu0=mu0,
                   meta={"Delta": Delta, "R": R, "dtype": dtype_note})


def dendrite_2d() -> Problem:
    """2-D 128^2, 2 phases, binary, isotropic, obstacle, R=10 seed, FP64, 1000 steps."""
    return binary_problem("dendrite_2d128_n2_fp64", 128, delta=0.0, Delta=0.2, R=10.0,
                          potential="obstacle", dtype_note="f64", steps=1000)


def lamellae_x(nx: int, rng: PCG32, wmin: int = 8, wmax: int = 24) -> np.ndarray:
    """Phase label (0 = alpha, 1 = beta) per x column; widths uniform in [wmin, wmax]."""
    lab = np.zeros(nx, dtype=np.int64)
    x, ph = 0, 0
    while x < nx:
        w = rng.randint(wmin, wmax)
        lab[x:min(nx, x + w)] = ph
        x += w
        ph ^= 1
    return lab


def eutectic_3d(n: int = 256, steps: int = 2000, seed: int = BASE_SEED) -> Problem:
    """3-D n^3 directional eutectic: alpha/beta lamellae under liquid, ternary.

    Symmetric synthetic eutectic: c_eq^alpha = (0.75, 0.125),
    c_eq^beta = (0.125, 0.75), c_eq^l = (0.40, 0.40) at T_ref = 0, A = I,
    liquidus slopes s^l = (-0.05, -0.05) (read as dc/dT), frozen gradient
    T = G (z - z0 - V t), G = 1e-3, z0 = 24, V = 0.05; delta = 0.02 on the two
    solid-liquid pairs, solid-solid isotropic; no-flux in z, periodic in x/y.
    mu0 = 0.8 is the liquid's equilibrium potential A^l c^l at T_ref.
    """
    N, NM = 3, 2
    gamma, dl, rot, D, A = _default_material(N, NM)
    for s in (0, 1):
        dl[s, 2] = dl[2, s] = 0.02
    ceq = np.array([[0.75, 0.125], [0.125, 0.75], [0.40, 0.40]])
    slopes = np.zeros((N, NM))
    slopes[2] = [-0.05, -0.05]
    dt = 0.2 * dt_stab(3, 1.0, 1.0, 1.0, 0.02, 1.0)
    rng = PCG32(seed, seq=2)
    lab = lamellae_x(n, rng)
    phi0 = np.zeros((N, n, n, n))
    zc = _centres(n, 1.0)
    solid = zc < 20.0
    for ph in (0, 1):
        col = (lab == ph).astype(np.float64)  # [x]
        phi0[ph] = solid[:, None, None] * col[None, None, :]
    phi0[2] = 1.0 - phi0[0] - phi0[1]
    mu0 = np.full((NM, n, n, n), 0.8)
    return Problem(name=f"eutectic_3d{n}_n3k3_fp32", dim=3, nx=n, ny=n, nz=n, n_phases=N,
                   n_components=3, bc=[BC_PERIODIC, BC_PERIODIC, BC_NOFLUX], dt=dt,
                   gamma=gamma, delta=dl, rot=rot, D=D, A=A, ceq=ceq, slopes=slopes,
                   f0=np.zeros(N), T_ref=0.0, T0=0.0, G=1e-3, z0=24.0, V=0.05,
                   steps=steps, phi0=phi0, mu0=mu0, meta={"dtype": "f32"})


def batched_dendrites_2d(nsims: int = 512, steps: int = 500, seed: int = BASE_SEED) -> List[Problem]:
    """Batched 2-D dendrites: edge in {64,...,512}, Delta~U[0.1,0.4], delta~U[0.01,0.05]."""
    rng = PCG32(seed, seq=3)
    edges = list(range(64, 513, 32))
    sims = []
    for s in range(nsims):
        e = edges[rng.randint(0, len(edges) - 1)]
        Delta = 0.1 + 0.3 * rng.uniform()
        delta = 0.01 + 0.04 * rng.uniform()
        p = binary_problem(f"batched_dendrite{s}", e, delta=delta, Delta=Delta, R=6.0,
                           potential="obstacle", dtype_note="f32", steps=steps)
        sims.append(p)
    return sims


def adjoint_well_2d(n: int = 256, steps: int = 2000, delta: float = 0.03, mob: float = 1.0) -> Problem:
    """Adjoint case: 2-D n^2 binary, well potential; dt fixed from delta = 0.03."""
    dt = 0.2 * dt_stab(2, 1.0, 1.0, 1.0, 0.03, 1.0)
    p = binary_problem(f"adjoint_well_2d{n}_well", n, delta=delta, Delta=0.2, R=10.0,
                       potential="well", dtype_note="f32", steps=steps, dt=dt,
                       tau=1.0 / mob)
    p.meta.update({"ckpt_every": 100, "delta_eval": 0.02, "mob_eval": 0.8})
    return p


def shoemake_rotation(rng: PCG32) -> np.ndarray:
    """Uniform random rotation (Shoemake 1992, 'Uniform random rotations')."""
    u1, u2, u3 = rng.uniform(), rng.uniform(), rng.uniform()
    a = math.sqrt(1.0 - u1)
    b = math.sqrt(u1)
    w, x, y, z = (b * math.cos(2 * math.pi * u3), a * math.sin(2 * math.pi * u2),
                  a * math.cos(2 * math.pi * u2), b * math.sin(2 * math.pi * u3))
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def periodic_dist(a, b, n):
    d = np.abs(np.asarray(a) - np.asarray(b))
    d = np.minimum(d, n - d)
    return float(np.sqrt((d ** 2).sum()))


def multigrain_3d(n: int = 512, steps: int = 1000, grains: int = 7, R: float = 8.0,
         min_sep: float = 24.0, seed: int = BASE_SEED, make_fields: bool = True) -> Problem:
    """3-D n^3 multigrain: 7 rotated grains + liquid, binary, obstacle, periodic."""
    N, NM = grains + 1, 1
    rng = PCG32(seed, seq=5)
    gamma, dl, rot, D, A = _default_material(N, NM)
    L = N - 1
    for g in range(grains):
        dl[g, L] = dl[L, g] = 0.02
        Rg = shoemake_rotation(rng)
        rot[g, L] = Rg
        rot[L, g] = Rg
    centres = []
    while len(centres) < grains:
        c = [n * rng.uniform() for _ in range(3)]
        if all(periodic_dist(c, o, n) >= min_sep for o in centres):
            centres.append(c)
    ceq = np.array([[0.926]] * grains + [[0.817]])
    f0 = np.array([-0.2] * grains + [0.0])
    dt = 0.2 * dt_stab(3, 1.0, 1.0, 1.0, 0.02, 1.0)
    p = Problem(name=f"multigrain_3d{n}_n8_fp32", dim=3, nx=n, ny=n, nz=n, n_phases=N,
                n_components=2, bc=[BC_PERIODIC] * 3, dt=dt, gamma=gamma, delta=dl,
                rot=rot, D=D, A=A, ceq=ceq, slopes=np.zeros((N, NM)), f0=f0,
                steps=steps, meta={"dtype": "f32", "centres": centres, "R": R})
    if make_fields:
        p.phi0, p.mu0 = grain_fields(p, np.float64)
    return p


def uniform_gamma3(N: int, value: float) -> np.ndarray:
    """Gamma_abc = value for every triple of distinct phases, 0 otherwise."""
    G = np.full((N, N, N), float(value))
    for k in range(N):
        G[k, k, :] = 0.0
        G[k, :, k] = 0.0
        G[:, k, k] = 0.0
    return G


def sparse_grain_growth(n: int = 256, dim: int = 3, grains: int = 8, gamma3: float = 15.0,
                        seed: int = BASE_SEED, ny: int = None, nz: int = None, steps: int = 1000) -> Problem:
    """Grain growth for the sparse (locally active) path: the Voronoi grains
    of grain_growth with diffuse boundaries (diffuse_voronoi: a sharp start
    makes transient stencils of 10 and more grains), a uniform triple term
    Gamma_abc = gamma3 (above 96 gamma / pi^2, so that two-grain boundaries
    hold no third grain) and the projection over the locally active phases."""
    p = grain_growth(n=n, dim=dim, grains=grains, seed=seed, ny=ny, nz=nz, steps=steps)
    p = p.copy(gamma3=uniform_gamma3(grains, gamma3), active_set=1, name=p.name + "_sparse",
               meta={**p.meta, "gamma3": gamma3})
    p.phi0 = diffuse_voronoi(p)
    return p


def grain_growth(n: int = 256, dim: int = 3, grains: int = 8, seed: int = BASE_SEED, ny: int = None,
                 nz: int = None, steps: int = 1000) -> Problem:
    """Isotropic grain growth (GRAINGROWTH = 1): `grains` grains (one phase
    each, equal isotropic boundary energies) filling a periodic box as the
    Voronoi cells of seeded random centres (each cell pure in the grain of its
    nearest centre; the boundaries take their diffuse profile in the first
    steps).  The solute field (one, or two for 3 grains, to match the compiled
    (N, K) pairs) is held."""
    N = grains
    NM = 2 if N == 3 else 1
    ny = n if ny is None else ny
    nz = (n if dim == 3 else 1) if nz is None else nz
    rng = PCG32(seed, seq=7)
    gamma, dl, rot, D, A = _default_material(N, NM)
    D[:] = 0.0
    shape = (nz, ny, n) if dim == 3 else (1, ny, n)
    ext = [n, ny, nz][:dim]
    centres = [[e * rng.uniform() for e in ext] for _ in range(N)]
    # squared periodic distance of every cell centre to every grain centre
    grids = np.meshgrid(*[_centres(e, 1.0) for e in ext[::-1]], indexing="ij")   # z, y, x order
    d2 = np.zeros((N,) + grids[0].shape)
    for g, c in enumerate(centres):
        for k in range(dim):
            t = grids[dim - 1 - k] - c[k]
            t = t - ext[k] * np.round(t / ext[k])
            d2[g] += t * t
    nearest = np.argmin(d2, axis=0)
    phi = np.stack([(nearest == g).astype(np.float64) for g in range(N)]).reshape((N,) + shape)
    mu0 = np.zeros((NM,) + shape)
    dt = 0.2 * dt_stab(dim, 1.0, 1.0, 1.0, 0.0, 0.0)
    return Problem(name=f"gg_{dim}d{n}_n{N}", dim=dim, nx=n, ny=ny, nz=nz, n_phases=N, n_components=NM + 1,
                   bc=[BC_PERIODIC] * 3, dt=dt, gamma=gamma, delta=dl, rot=rot, D=D, A=A,
                   ceq=np.full((N, NM), 0.5), slopes=np.zeros((N, NM)), f0=np.zeros(N), steps=steps,
                   grain_growth=1, phi0=phi, mu0=mu0, meta={"dtype": "f32", "centres": centres})


def grain_fields(p: Problem, dtype=np.float64):
    """Initial phi/mu for a multigrain problem built from p.meta['centres']."""
    n, N = p.nx, p.n_phases
    R = p.meta["R"]
    phi = np.zeros((N, p.nz, p.ny, n), dtype=dtype)
    ax = _centres(n, 1.0)
    for g, c in enumerate(p.meta["centres"]):
        # periodic distance along each axis, evaluated on a bounding box only
        h = int(math.ceil(R + math.pi ** 2 * p.eps / 8.0)) + 2
        idx = [np.arange(int(math.floor(c[d])) - h, int(math.floor(c[d])) + h + 1) % n
               for d in range(3)]
        dz = ax[idx[2]] - c[2]
        dy = ax[idx[1]] - c[1]
        dxx = ax[idx[0]] - c[0]
        dz = np.minimum(np.abs(dz), n - np.abs(dz))
        dy = np.minimum(np.abs(dy), n - np.abs(dy))
        dxx = np.minimum(np.abs(dxx), n - np.abs(dxx))
        r = np.sqrt(dz[:, None, None] ** 2 + dy[None, :, None] ** 2 + dxx[None, None, :] ** 2)
        phi[g][np.ix_(idx[2], idx[1], idx[0])] = seed_profile((R - r) / p.eps, p.potential)
    tot = phi[:N - 1].sum(axis=0)
    over = tot > 1.0
    if over.any():
        phi[:N - 1][:, over] /= tot[over]
        tot = phi[:N - 1].sum(axis=0)
    phi[N - 1] = 1.0 - tot
    mu = np.full((1, p.nz, p.ny, n), 2.0 * 0.817, dtype=dtype)
    return phi, mu


def small_multiphase(n: int = 24, dim: int = 3, N: int = 3, NM: int = 2, seed: int = 7,
                     potential: str = "obstacle", aniso: bool = True, rotate: bool = False,
                     bc=None, nx: int = None, ny: int = None, nz: int = None,
                     gamma3: float = 0.0) -> Problem:
    """A small random-but-physical multiphase state for parity tests.

    Smooth random blobs of every phase (superposed seeded Gaussians) are
    normalised onto the simplex, so every pair of phases meets somewhere;
    mu is a seeded smooth perturbation around the liquid equilibrium value.
    """
    rng = PCG32(seed, seq=11)
    nx = n if nx is None else nx
    ny = n if ny is None else ny
    nz = 1 if dim == 2 else (n if nz is None else nz)
    gamma, dl, rot, D, A = _default_material(N, NM)
    for a in range(N):
        for b in range(a + 1, N):
            gamma[a, b] = gamma[b, a] = 0.8 + 0.4 * rng.uniform()
            if aniso:
                dl[a, b] = dl[b, a] = 0.01 + 0.04 * rng.uniform()
            if rotate:
                Rm = shoemake_rotation(rng)
                if dim == 2:
                    th = 2 * math.pi * rng.uniform()
                    Rm = np.array([[math.cos(th), -math.sin(th), 0.0],
                                   [math.sin(th), math.cos(th), 0.0], [0.0, 0.0, 1.0]])
                rot[a, b] = rot[b, a] = Rm
    ceq = np.zeros((N, NM))
    for a in range(N):
        for i in range(NM):
            ceq[a, i] = 0.1 + 0.8 * rng.uniform()
        A[a] = np.eye(NM) * (0.8 + 0.4 * rng.uniform())
        for i in range(NM):
            for j in range(i + 1, NM):
                A[a, i, j] = 0.1 * (rng.uniform() - 0.5)
    for a in range(N):
        D[a] = np.eye(NM) * (0.3 + 0.7 * rng.uniform()) if a == N - 1 else np.eye(NM) * 0.1 * rng.uniform()
    slopes = np.zeros((N, NM))
    slopes[N - 1] = -0.05
    g3 = None
    if gamma3:
        g3 = np.zeros((N, N, N))
        for a in range(N):
            for b in range(N):
                for c in range(N):
                    if len({a, b, c}) == 3:
                        g3[a, b, c] = gamma3
    # smooth random phase fields
    shape = (nz, ny, nx)
    grids = np.meshgrid(*[np.arange(s) + 0.5 for s in shape], indexing="ij")
    raw = np.zeros((N,) + shape)
    for a in range(N):
        for _ in range(3):
            c = [rng.uniform() * s for s in shape]
            w = 3.0 + 4.0 * rng.uniform()
            r2 = np.zeros(shape)
            for d, s in enumerate(shape):
                dd = np.abs(grids[d] - c[d])
                dd = np.minimum(dd, s - dd)
                r2 = r2 + dd ** 2
            raw[a] += np.exp(-r2 / (2 * w * w))
    raw = raw ** 3
    raw += 1e-3
    phi0 = raw / raw.sum(axis=0, keepdims=True)
    # sharpen: clip small values to exact zeros so bulk regions exist, renormalise
    phi0 = np.where(phi0 < 0.02, 0.0, phi0)
    phi0 = phi0 / phi0.sum(axis=0, keepdims=True)
    mu0 = np.zeros((NM,) + shape)
    for i in range(NM):
        mu0[i] = 2.0 * ceq[N - 1, i] * A[N - 1, i, i] + 0.02 * np.sin(
            2 * math.pi * (grids[2] / nx + (i + 1) * grids[1] / max(ny, 1)))
    dt = 0.2 * dt_stab(dim, 1.0, 1.0, float(gamma.max()), float(dl.max()), float(D.max()))
    return Problem(name=f"small_{dim}d_n{N}k{NM + 1}", dim=dim, nx=nx, ny=ny, nz=nz,
                   n_phases=N, n_components=NM + 1,
                   bc=bc or [BC_PERIODIC, BC_PERIODIC, BC_NOFLUX if dim == 3 else BC_PERIODIC],
                   dt=dt, potential=potential, gamma=gamma, delta=dl, rot=rot, gamma3=g3,
                   D=D, A=A, ceq=ceq, slopes=slopes, f0=np.zeros(N) - 0.05 * np.eye(N)[0],
                   T_ref=0.0, T0=0.0, G=2e-3, z0=(nz if dim == 3 else ny) / 2.0, V=0.05, steps=10,
                   phi0=phi0, mu0=mu0, meta={"seed": seed})


def diffuse_voronoi(p: Problem) -> np.ndarray:
    """Voronoi grains of p.meta['centres'] (periodic) with diffuse boundaries:
    each cell shares the obstacle profile S(s / eps) between its nearest and
    second-nearest grain, s the distance to their bisecting plane (pure in the
    nearest grain farther than pi^2 eps / 8 from it)."""
    n, ny, nz, N, dim = p.nx, p.ny, p.nz, p.n_phases, p.dim
    ext = np.array([n, ny, nz][:dim], dtype=np.float64)
    cen = np.array(p.meta["centres"], dtype=np.float64)
    grids = np.meshgrid(*[_centres(int(e), 1.0) for e in ext[::-1]], indexing="ij")
    pos = np.stack([grids[dim - 1 - k] for k in range(dim)], axis=-1)
    d2 = np.zeros((N,) + grids[0].shape)
    for g in range(N):
        t = pos - cen[g]
        t = t - ext * np.round(t / ext)
        d2[g] = (t * t).sum(-1)
    order = np.argsort(d2, axis=0)
    g1, g2 = order[0], order[1]
    d1 = np.take_along_axis(d2, g1[None], 0)[0]
    dd2 = np.take_along_axis(d2, g2[None], 0)[0]
    dc = cen[g2] - cen[g1]
    dc = dc - ext * np.round(dc / ext)
    s = (dd2 - d1) / (2.0 * np.sqrt((dc * dc).sum(-1)))
    f = seed_profile(s / p.eps, p.potential)
    phi = np.zeros((N,) + grids[0].shape)
    np.put_along_axis(phi, g1[None], f[None], 0)
    np.put_along_axis(phi, g2[None], (1.0 - f)[None], 0)
    return phi.reshape((N,) + p.phi0.shape[1:])
