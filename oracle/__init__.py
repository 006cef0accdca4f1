"""FP64 CPU oracle for the grand-potential phase-field step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA product path never does; the
two implementations share no code.  ``gp_oracle.cpp`` restates the paper's
equations as plain per-cell loops (see its header for the passages followed
and the readings taken where the paper is silent).

Parity status per function (pins live in ``tests/test_oracle_pins.py``):
  * pair_energy / its gradient, interpolation h, potentials, projection,
    thermodynamics (c(mu), psi, chi, Coeff_B/C), the isotropic Laplacian
    identity, planar sine / tanh profiles, Fourier-mode and Gaussian decay of
    mu, mass conservation, sum(phi)=1, flat-interface equilibrium,
    Gibbs-Thomson direction, anisotropic profile width, tangent vs finite
    differences: pinned.
  * The anti-trapping current (``tests/test_oracle_at.py``): closed-form face
    values, direction, inertness, flux-form conservation, symmetries: pinned.
  * Grain growth (``tests/test_oracle_gg.py``): frozen mu, stationary planar
    boundary, the curvature-driven area loss rate of a circular grain: pinned.
  * Elasticity (``tests/test_oracle_elastic.py``): closed-form laminate,
    Voigt shear factor, divergence-free stress: pinned.  With one stiffness
    per phase (elastic_fields_inhomogeneous): the homogeneous limit, the
    closed-form laminate of two stiffnesses, divergence-free stress, and the
    potentials as the phi-derivative of the equilibrium energy: pinned.
  * The chemical mobility inside interfaces, M = sum_a h_a D^a chi^a with
    phi^n (``tests/test_oracle_mobility.py``): exact one-step and frozen-phi
    mode decay, two-solute matrix order: pinned.
  * run_adjoint (the reverse sweep by a tape, ``tests/test_oracle_adjoint.py``):
    equal to the forward-mode tangent in a dot-product test: pinned.
  * count_flops (the op-counting scalar, ``tests/test_oracle_flops.py``):
    exact counts of hand-countable updates: pinned.
  * Grid refinement (``tests/test_oracle_refinement.py``): second-order
    convergence of a smooth three-phase anisotropic trajectory under dx ->
    dx/2 -> dx/4 with dt ~ dx^2, which pins the dx scaling of every term.
  * Gradient flow (``tests/test_oracle_variational.py``): at uniform mu and T,
    with isotropic pairs and three or four phases, one step's rate equals the
    projected variational derivative of the grand-potential functional.  That
    derivative is taken by finite differences of the functional, with spectral
    gradients, and the two agree at second order.  With rotated anisotropic
    pairs, the functional falls along the step's rate r at -tau eps |r|^2,
    also at second order: pinned.
  * Covariance (``tests/test_oracle_covariance.py``): the 3-D step with
    rotated anisotropic pairs commutes with the grid's axis permutations and
    mirrors when each rotation is composed with the inverse move: pinned.
  * The full multiphase (N >= 3) anisotropic dendrite / eutectic / multigrain
    trajectories: parity unpinned beyond the identities above and the
    convergence order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libgp_oracle.so")
_SRC = os.path.join(_HERE, "gp_oracle.cpp")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gp_oracle.cpp into oracle/_build/libgp_oracle.so (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("bc", ctypes.c_int * 3), ("N", ctypes.c_int), ("NM", ctypes.c_int),
        ("potential", ctypes.c_int),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("eps", ctypes.c_double),
        ("tau", ctypes.c_double),
        ("gamma", ctypes.c_void_p), ("delta", ctypes.c_void_p), ("rot", ctypes.c_void_p),
        ("gamma3", ctypes.c_void_p), ("D", ctypes.c_void_p), ("A", ctypes.c_void_p),
        ("ceq", ctypes.c_void_p), ("slopes", ctypes.c_void_p), ("f0", ctypes.c_void_p),
        ("T_ref", ctypes.c_double), ("T0", ctypes.c_double), ("G", ctypes.c_double),
        ("z0", ctypes.c_double), ("V", ctypes.c_double), ("t0", ctypes.c_double),
        ("z_origin", ctypes.c_int), ("noise_amp", ctypes.c_double), ("noise_seed", ctypes.c_ulonglong),
        ("step0", ctypes.c_longlong), ("anti_trapping", ctypes.c_int), ("grain_growth", ctypes.c_int),
        ("elw", ctypes.c_void_p), ("active_set", ctypes.c_int),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            dp = ctypes.POINTER(ctypes.c_double)
            P = ctypes.POINTER(_Problem)
            L.oracle_run.argtypes = [P, dp, dp, ctypes.c_int, dp, dp]
            L.oracle_run_tangent.argtypes = [P, dp, dp, dp, dp, dp, ctypes.c_double, dp,
                                             ctypes.c_int, dp, dp, dp, dp]
            L.oracle_rate_parts.argtypes = [P, dp, dp, dp, dp, dp, dp]
            L.oracle_diag.argtypes = [P, dp, dp, dp]
            L.oracle_count_flops.argtypes = [P, dp, dp, dp, dp]
            L.oracle_run_adjoint.argtypes = [P, dp, dp, ctypes.c_int, dp, dp, dp, dp, dp]
            L.oracle_pair_energy.argtypes = [P, ctypes.c_int, ctypes.c_int, dp]
            L.oracle_pair_energy.restype = ctypes.c_double
            L.oracle_pair_energy_grad.argtypes = [P, ctypes.c_int, ctypes.c_int, dp, dp]
            L.oracle_potential.argtypes = [P, dp, dp]
            L.oracle_potential.restype = ctypes.c_double
            L.oracle_interp.argtypes = [ctypes.c_int, dp, dp, dp]
            L.oracle_project.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
            L.oracle_thermo.argtypes = [P, ctypes.c_int, dp, ctypes.c_double, dp, dp, dp]
            L.oracle_at_face_flux.argtypes = [P, dp, dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_double, dp]
            L.oracle_noise.argtypes = [ctypes.c_ulonglong, ctypes.c_longlong, ctypes.c_ulonglong]
            L.oracle_noise.restype = ctypes.c_double
            L.oracle_num_threads.restype = ctypes.c_int
            L.oracle_set_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class OracleProblem:
    """Marshals a problem description (duck-typed workloads.Problem) for the C oracle."""

    def __init__(self, prob, t0: float = 0.0, step0: int = 0, **override):
        g = lambda k: override.get(k, getattr(prob, k))
        opt = lambda k, d: override.get(k, getattr(prob, k, d))
        self.N = int(g("n_phases"))
        self.NM = int(g("n_components")) - 1
        self.dim = int(g("dim"))
        self.nx, self.ny = int(g("nx")), int(g("ny"))
        self.nz = int(g("nz")) if self.dim == 3 else 1
        N, NM = self.N, self.NM
        self._keep = []

        def arr(x, shape):
            a = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(shape))
            self._keep.append(a)
            return a.ctypes.data

        s = _Problem()
        s.dim, s.nx, s.ny, s.nz = self.dim, self.nx, self.ny, self.nz
        bc = list(g("bc")) + [3] * 3
        s.bc = (ctypes.c_int * 3)(*bc[:3])
        s.N, s.NM = N, NM
        s.potential = 1 if g("potential") == "obstacle" else 2
        s.dx, s.dt, s.eps, s.tau = float(g("dx")), float(g("dt")), float(g("eps")), float(g("tau"))
        s.gamma = arr(g("gamma"), (N, N))
        s.delta = arr(g("delta"), (N, N))
        rot = g("rot")
        s.rot = arr(rot, (N, N, 3, 3)) if rot is not None else None
        g3 = g("gamma3")
        s.gamma3 = arr(g3, (N, N, N)) if g3 is not None else None
        s.D = arr(g("D"), (N, NM, NM))
        s.A = arr(g("A"), (N, NM, NM))
        s.ceq = arr(g("ceq"), (N, NM))
        s.slopes = arr(g("slopes"), (N, NM))
        f0 = g("f0")
        s.f0 = arr(f0, (N,)) if f0 is not None else None
        s.T_ref, s.T0, s.G = float(g("T_ref")), float(g("T0")), float(g("G"))
        s.z0, s.V = float(g("z0")), float(g("V"))
        s.t0 = float(t0)
        meta = getattr(prob, "meta", None) or {}
        s.z_origin = int(override.get("z_origin", meta.get("z_origin", 0)))
        s.noise_amp = float(opt("noise_amp", 0.0))
        s.noise_seed = int(opt("noise_seed", 0)) & 0xFFFFFFFFFFFFFFFF
        s.step0 = int(step0)
        s.anti_trapping = int(bool(opt("anti_trapping", 0)))
        s.grain_growth = int(bool(opt("grain_growth", 0)))
        elw = override.get("elw", None)
        s.elw = arr(elw, (N, self.nx * self.ny * self.nz)) if elw is not None else None
        s.active_set = int(bool(opt("active_set", 0)))
        self.s = s

    @property
    def cells(self):
        return self.nx * self.ny * self.nz

    def shape(self, nf):
        return (nf, self.nz, self.ny, self.nx)

    def ptr(self):
        return ctypes.byref(self.s)


# Voigt index of a symmetric pair (xx, yy, zz, yz, xz, xy)
_VOIGT = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (1, 2): 3, (2, 1): 3, (0, 2): 4, (2, 0): 4, (0, 1): 5, (1, 0): 5}


def stiffness_tensor(Cv, dim):
    """C_ijkl from the 6 x 6 Voigt matrix (sigma_v = C_v eps_v, engineering
    shear), restricted to the first `dim` axes (plane strain in 2-D)."""
    C = np.zeros((3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    C[i, j, k, l] = Cv[_VOIGT[i, j]][_VOIGT[k, l]]
    return C[:dim, :dim, :dim, :dim]


def interp_field(phi):
    """h_a(phi) of Eq. (hphi) over whole fields [N][...]: 3 phi_a^2 - 2 phi_a^3
    + 2 phi_a sum_{b<c; b, c != a} phi_b phi_c."""
    N = phi.shape[0]
    h = np.empty_like(phi)
    for a in range(N):
        pair = np.zeros_like(phi[0])
        for b in range(N):
            for c in range(b + 1, N):
                if b != a and c != a:
                    pair += phi[b] * phi[c]
        h[a] = 3.0 * phi[a] ** 2 - 2.0 * phi[a] ** 3 + 2.0 * phi[a] * pair
    return h


def _wavenumbers(n, dx):
    """2 pi m / (n dx) in FFT order, the Nyquist index of an even n taken as 0
    (its sign is ambiguous; a zero keeps the solution Hermitian)."""
    k = 2.0 * np.pi * np.fft.fftfreq(n, dx)
    if n % 2 == 0:
        k[n // 2] = 0.0
    return k


def elastic_fields(prob, phi):
    """Mechanical equilibrium with a homogeneous stiffness (Sec. 2 "Elasticity
    implementation": the homogeneous case of the Fourier-space solution, with
    the eigenstrain sum_a eps*^a h_a(phi) of its Eq. for e_kl and no
    homogeneous strain, i.e. a clamped periodic box).  In Fourier space
    t_i = C_ijmn k_j eps*_mn, G = (C_ijkl k_j k_l)^-1, the displacement is
    -i G t and the strain eps_kl = (k_k (G t)_l + k_l (G t)_k) / 2 (zero at
    k = 0); k_j = 2 pi m_j / (n_j dx) in FFT order (the Nyquist index of an
    even extent taken as 0).  Returns the stress
    sigma = C (eps - eps*) [dim][dim][nz][ny][nx] and, per phase, the elastic
    part of its potential w_b = -sigma : eps*^b [N][nz][ny][nx], whose
    contraction with dh_b/dphi_a is d f_el / d phi_a."""
    dim = prob.dim
    N = prob.n_phases
    nz = prob.nz if dim == 3 else 1
    shape = (nz, prob.ny, prob.nx)
    phi = np.asarray(phi, dtype=np.float64).reshape((N,) + shape)
    C = stiffness_tensor(np.asarray(prob.elastic_C, dtype=np.float64), dim)
    eig = np.asarray(prob.eigenstrain, dtype=np.float64).reshape(N, 3, 3)[:, :dim, :dim]
    h = interp_field(phi)
    E = np.einsum("amn,a...->mn...", eig, h)                      # eps*(x) [dim][dim][grid]
    axes = (0, 1, 2) if dim == 3 else (1, 2)
    Eh = np.fft.fftn(E, axes=tuple(a + 2 for a in axes))
    ks = [_wavenumbers(n, prob.dx) for n in (prob.nx, prob.ny, nz)[:dim]]
    K = np.zeros((dim,) + shape)
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")   # z, y, x
    for d in range(dim):
        K[d] = ks[d][grids[2 - d]]
    t = np.einsum("ijmn,j...,mn...->i...", C, K, Eh)
    Ginv = np.einsum("ijkl,j...,l...->ik...", C, K, K)
    Ginv = np.moveaxis(Ginv, (0, 1), (-2, -1))
    zero = (K ** 2).sum(axis=0) == 0.0
    Ginv[zero] = np.eye(dim)
    G = np.linalg.inv(Ginv)
    G[zero] = 0.0
    Gt = np.einsum("...ki,i...->k...", G, t)
    epsh = 0.5 * (np.einsum("k...,l...->kl...", K, Gt) + np.einsum("l...,k...->kl...", K, Gt))
    eps = np.real(np.fft.ifftn(epsh, axes=tuple(a + 2 for a in axes)))
    sigma = np.einsum("ijkl,kl...->ij...", C, eps - E)
    w = -np.einsum("ij...,bij->b...", sigma, eig)
    return sigma, w


def elastic_fields_inhomogeneous(prob, phi, C_phases, tol: float = 1e-13, max_iter: int = 5000):
    """Mechanical equilibrium with a stiffness that varies with the phases,
    C(x) = sum_a C^a h_a(phi) (Eqs. 43-44), in the Fourier-space form of
    Sec. 2 "Elastic equilibrium in a multiphase setting": the homogeneous part
    is the mean stiffness Cbar = (1/N) sum_a C^a (Eq. 47) and
    Delta C(x) = sum_a (C^a - Cbar) h_a (Eq. 48); Eqs. 51-55 are solved by
    their fixed point.  Each iteration applies the homogeneous operator of
    `elastic_fields` (same wavenumbers, clamped periodic box) for Cbar to the
    polarisation P = Cbar eps* - Delta C (eps - eps*) of the current strain,
    starting from eps = 0, until the strain changes by less than
    tol * max|eps*|.  C_phases: [N][6][6] Voigt matrices.

    Returns (sigma [dim][dim][grid], w [N][grid], iterations).
    w_b = 1/2 e : C^b : e - sigma : eps*^b with e = eps - eps*.  Contracted
    with dh_b/dphi_a it gives d f_el / d phi_a of
    f_el = 1/2 e : C(phi) : e at equilibrium.  With equal stiffnesses the
    first term cancels in that contraction (sum_b dh_b/dphi_a = 0), which
    leaves the homogeneous w_b."""
    dim = prob.dim
    N = prob.n_phases
    nz = prob.nz if dim == 3 else 1
    shape = (nz, prob.ny, prob.nx)
    phi = np.asarray(phi, dtype=np.float64).reshape((N,) + shape)
    Cs = [stiffness_tensor(np.asarray(C_phases[b], dtype=np.float64), dim) for b in range(N)]
    Cbar = sum(Cs) / N
    eig = np.asarray(prob.eigenstrain, dtype=np.float64).reshape(N, 3, 3)[:, :dim, :dim]
    h = interp_field(phi)
    E = np.einsum("amn,a...->mn...", eig, h)                      # eps*(x)
    dC = sum(np.einsum("ijkl,...->ijkl...", Cs[b] - Cbar, h[b]) for b in range(N))
    axes = tuple(a + 2 for a in ((0, 1, 2) if dim == 3 else (1, 2)))
    ks = [_wavenumbers(n, prob.dx) for n in (prob.nx, prob.ny, nz)[:dim]]
    K = np.zeros((dim,) + shape)
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")   # z, y, x
    for d in range(dim):
        K[d] = ks[d][grids[2 - d]]
    Ginv = np.moveaxis(np.einsum("ijkl,j...,l...->ik...", Cbar, K, K), (0, 1), (-2, -1))
    zero = (K ** 2).sum(axis=0) == 0.0
    Ginv[zero] = np.eye(dim)
    G = np.linalg.inv(Ginv)
    G[zero] = 0.0
    eps = np.zeros_like(E)
    scale = max(np.abs(E).max(), 1e-300)
    it = 0
    for it in range(1, max_iter + 1):
        P = np.einsum("ijkl,kl...->ij...", Cbar, E) - np.einsum("ijkl...,kl...->ij...", dC, eps - E)
        t = np.einsum("j...,ij...->i...", K, np.fft.fftn(P, axes=axes))
        Gt = np.einsum("...ki,i...->k...", G, t)
        epsh = 0.5 * (np.einsum("k...,l...->kl...", K, Gt) + np.einsum("l...,k...->kl...", K, Gt))
        new = np.real(np.fft.ifftn(epsh, axes=axes))
        change = np.abs(new - eps).max()
        eps = new
        if change <= tol * scale:
            break
    else:
        raise RuntimeError(f"inhomogeneous elasticity did not converge in {max_iter} iterations")
    e = eps - E
    sigma = np.einsum("ijkl,kl...->ij...", Cbar, e) + np.einsum("ijkl...,kl...->ij...", dC, e)
    w = np.stack([0.5 * np.einsum("ij...,ijkl,kl...->...", e, Cs[b], e)
                  - np.einsum("ij...,ij->...", sigma, eig[b]) for b in range(N)])
    return sigma, w, it


def _elastic(prob, override):
    C = override.get("elastic_C", getattr(prob, "elastic_C", None))
    return C is not None or override.get("elastic_C_phases") is not None


def run(prob, phi0, mu0, nsteps: int, t0: float = 0.0, step0: int = 0, **override):
    """nsteps explicit steps in FP64; returns (phi, mu) shaped [F][nz][ny][nx].
    step0 = step index of the input state (the counter of the phi noise).
    With a stiffness (`elastic_C`) the elastic potentials are solved from the
    state before every step; `elastic_C_phases` ([N][6][6]) takes one
    stiffness per phase instead (the inhomogeneous solve)."""
    if _elastic(prob, override) and "elw" not in override:
        phi, mu = phi0, mu0
        Cph = override.pop("elastic_C_phases", None)
        for n in range(int(nsteps)):
            if Cph is not None:
                _, w, _ = elastic_fields_inhomogeneous(prob, phi, Cph)
            else:
                _, w = elastic_fields(prob, phi)
            phi, mu = run(prob, phi, mu, 1, t0=t0 + n * prob.dt, step0=step0 + n, elw=w, **override)
        return phi, mu
    op = OracleProblem(prob, t0, step0, **override)
    phi0 = np.ascontiguousarray(phi0, dtype=np.float64).reshape(op.shape(op.N))
    mu0 = np.ascontiguousarray(mu0, dtype=np.float64).reshape(op.shape(op.NM))
    phi = np.empty_like(phi0)
    mu = np.empty_like(mu0)
    rc = lib().oracle_run(op.ptr(), _dp(phi0), _dp(mu0), int(nsteps), _dp(phi), _dp(mu))
    if rc:
        raise ValueError("oracle_run rejected the problem")
    return phi, mu


def at_face_flux(prob, phi, phin, mu, x: int, y: int, z: int, d: int, t0: float = 0.0, **override):
    """Normal component (along axis d) of the anti-trapping current j_at at the
    face between cell (x, y, z) and its +d neighbour, per solute; phi = phi^n,
    phin = phi^{n+1}, mu = mu^n at time t0 (Eq. jatr)."""
    op = OracleProblem(prob, t0, **override)
    phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(op.shape(op.N))
    phin = np.ascontiguousarray(phin, dtype=np.float64).reshape(op.shape(op.N))
    mu = np.ascontiguousarray(mu, dtype=np.float64).reshape(op.shape(op.NM))
    J = np.zeros(op.NM)
    if lib().oracle_at_face_flux(op.ptr(), _dp(phi), _dp(phin), _dp(mu), x, y, z, d, float(t0), _dp(J)):
        raise ValueError("oracle_at_face_flux rejected the problem")
    return J


def noise(seed: int, step: int, counter: int) -> float:
    """The phi-noise variate in [-1/2, 1/2) for (seed, step, counter), counter =
    lab cell index x + nx (y + ny z) times N plus the phase."""
    return lib().oracle_noise(int(seed) & 0xFFFFFFFFFFFFFFFF, int(step), int(counter) & 0xFFFFFFFFFFFFFFFF)


def shift(dim, phi, mu, planes: int, mu_fill):
    """Moving frame (the SHIFT key of Sec. 4, "moving camera"): drop the first
    `planes` cells along the last axis (z in 3-D, y in 2-D), move the rest
    down and fill the far end with pure liquid (the last phase) at the
    chemical potential mu_fill of the original alloy.  Fields [F][nz][ny][nx]."""
    ax = 1 if dim == 3 else 2
    n = phi.shape[ax]
    k = int(planes)
    out = []
    for f, fill in ((phi, None), (mu, mu_fill)):
        g = np.empty_like(f)
        src = [slice(None)] * 4
        dst = [slice(None)] * 4
        src[ax], dst[ax] = slice(k, n), slice(0, n - k)
        g[tuple(dst)] = f[tuple(src)]
        tail = [slice(None)] * 4
        tail[ax] = slice(n - k, n)
        if fill is None:
            g[tuple(tail)] = 0.0
            g[(-1,) + tuple(tail[1:])] = 1.0
        else:
            for i, v in enumerate(np.atleast_1d(fill)):
                g[(i,) + tuple(tail[1:])] = float(v)
        out.append(g)
    return out[0], out[1]


def run_tangent(prob, phi0, mu0, nsteps: int, dphi0=None, dmu0=None, ddelta=None,
                dmob: float = 0.0, dD=None, t0: float = 0.0, **override):
    """Forward-mode tangent: returns (phi, mu, dphi, dmu)."""
    op = OracleProblem(prob, t0, **override)
    N, NM = op.N, op.NM
    phi0 = np.ascontiguousarray(phi0, dtype=np.float64).reshape(op.shape(N))
    mu0 = np.ascontiguousarray(mu0, dtype=np.float64).reshape(op.shape(NM))
    z = lambda sh: np.zeros(sh)
    dphi0 = np.ascontiguousarray(z(phi0.shape) if dphi0 is None else dphi0, dtype=np.float64).reshape(phi0.shape)
    dmu0 = np.ascontiguousarray(z(mu0.shape) if dmu0 is None else dmu0, dtype=np.float64).reshape(mu0.shape)
    ddelta = np.ascontiguousarray(z((N, N)) if ddelta is None else ddelta, dtype=np.float64).reshape(N, N)
    dD = np.ascontiguousarray(z((N, NM, NM)) if dD is None else dD, dtype=np.float64).reshape(N, NM, NM)
    phi, mu = np.empty_like(phi0), np.empty_like(mu0)
    dphi, dmu = np.empty_like(phi0), np.empty_like(mu0)
    rc = lib().oracle_run_tangent(op.ptr(), _dp(phi0), _dp(mu0), _dp(dphi0), _dp(dmu0),
                                  _dp(ddelta), float(dmob), _dp(dD), int(nsteps),
                                  _dp(phi), _dp(mu), _dp(dphi), _dp(dmu))
    if rc:
        raise ValueError("oracle_run_tangent rejected the problem")
    return phi, mu, dphi, dmu


def rate_parts(prob, phi, mu, t0: float = 0.0, **override):
    op = OracleProblem(prob, t0, **override)
    phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(op.shape(op.N))
    mu = np.ascontiguousarray(mu, dtype=np.float64).reshape(op.shape(op.NM))
    outs = [np.empty_like(phi) for _ in range(4)]
    rc = lib().oracle_rate_parts(op.ptr(), _dp(phi), _dp(mu), *[_dp(o) for o in outs])
    if rc:
        raise ValueError("oracle_rate_parts rejected the problem")
    return tuple(outs)


def run_adjoint(prob, phi0, mu0, nsteps: int, lam_phi, lam_mu, t0: float = 0.0, step0: int = 0, **override):
    """Reverse adjoint of nsteps steps by the oracle's tape: for a loss with
    dL/dphi = lam_phi and dL/dmu = lam_mu at the final state, returns
    (dL/dphi0, dL/dmu0, dL/dtheta), theta = (delta_ab for pairs a < b, the
    phase mobility 1/tau, D^a_ij).  Single-threaded; small grids only."""
    op = OracleProblem(prob, t0, step0, **override)
    phi0 = np.ascontiguousarray(phi0, dtype=np.float64).reshape(op.shape(op.N))
    mu0 = np.ascontiguousarray(mu0, dtype=np.float64).reshape(op.shape(op.NM))
    lp = np.ascontiguousarray(lam_phi, dtype=np.float64).reshape(op.shape(op.N))
    lm = np.ascontiguousarray(lam_mu, dtype=np.float64).reshape(op.shape(op.NM))
    dphi0 = np.empty_like(phi0)
    dmu0 = np.empty_like(mu0)
    nprm = op.N * (op.N - 1) // 2 + 1 + op.N * op.NM * op.NM
    dtheta = np.zeros(nprm)
    if lib().oracle_run_adjoint(op.ptr(), _dp(phi0), _dp(mu0), int(nsteps), _dp(lp), _dp(lm), _dp(dphi0),
                                _dp(dmu0), _dp(dtheta)):
        raise ValueError("oracle_run_adjoint rejected the problem")
    return dphi0, dmu0, dtheta


def count_flops(prob, phi, mu, t0: float = 0.0, step0: int = 0, **override):
    """Arithmetic operations of one step per cell, counted by running the
    oracle's step with an op-counting scalar: (ops_phi, ops_mu), each
    [nz][ny][nx] (the phi sweep and the mu sweep).  Single-threaded."""
    op = OracleProblem(prob, t0, step0, **override)
    phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(op.shape(op.N))
    mu = np.ascontiguousarray(mu, dtype=np.float64).reshape(op.shape(op.NM))
    ops_phi = np.zeros(op.shape(1)[1:])
    ops_mu = np.zeros(op.shape(1)[1:])
    if lib().oracle_count_flops(op.ptr(), _dp(phi), _dp(mu), _dp(ops_phi), _dp(ops_mu)):
        raise ValueError("oracle_count_flops rejected the problem")
    return ops_phi, ops_mu


def diag(prob, phi, mu, t0: float = 0.0, **override):
    """[mass_1..mass_NM, max|sum phi - 1|, min phi, max phi] in FP64."""
    op = OracleProblem(prob, t0, **override)
    phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(op.shape(op.N))
    mu = np.ascontiguousarray(mu, dtype=np.float64).reshape(op.shape(op.NM))
    out = np.zeros(op.NM + 3)
    lib().oracle_diag(op.ptr(), _dp(phi), _dp(mu), _dp(out))
    return out


def pair_energy(prob, a, b, q, **override):
    op = OracleProblem(prob, **override)
    q = np.ascontiguousarray(q, dtype=np.float64)
    return lib().oracle_pair_energy(op.ptr(), a, b, _dp(q))


def pair_energy_grad(prob, a, b, q, **override):
    op = OracleProblem(prob, **override)
    q = np.ascontiguousarray(q, dtype=np.float64)
    g = np.zeros_like(q)
    lib().oracle_pair_energy_grad(op.ptr(), a, b, _dp(q), _dp(g))
    return g


def potential(prob, phi, **override):
    op = OracleProblem(prob, **override)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    dw = np.zeros_like(phi)
    w = lib().oracle_potential(op.ptr(), _dp(phi), _dp(dw))
    return w, dw


def interp(phi):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    N = phi.size
    h = np.zeros(N)
    dh = np.zeros((N, N))
    lib().oracle_interp(N, _dp(phi), _dp(h), _dp(dh))
    return h, dh


def project(v, potential_kind: str):
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros_like(v)
    lib().oracle_project(v.size, 1 if potential_kind == "obstacle" else 2, _dp(v), _dp(out))
    return out


def thermo(prob, a, mu, T, **override):
    """(c^a(mu,T), psi^a(mu,T), chi^a) for phase a."""
    op = OracleProblem(prob, **override)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    c = np.zeros(op.NM)
    psi = ctypes.c_double(0.0)
    chi = np.zeros((op.NM, op.NM))
    lib().oracle_thermo(op.ptr(), a, _dp(mu), float(T), _dp(c), ctypes.byref(psi), _dp(chi))
    return c, psi.value, chi


def num_threads() -> int:
    return lib().oracle_num_threads()


def set_threads(n: int):
    lib().oracle_set_threads(int(n))
