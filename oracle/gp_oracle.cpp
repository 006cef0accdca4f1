// Grand-potential multi-phase / multi-component explicit step: FP64 CPU oracle.
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference the CUDA
// library is checked against.  Only the test-suite, the package smoke check
// and the benchmark's CPU-baseline leg may load it; the product path never
// does.  It shares no code, header or table with the CUDA library.
//
// Every function restates one passage of the MICROSIM paper (arXiv 2404.01035,
// Sec. 2.1 "Grand-potential formulation" and Sec. 3 "Thermodynamic coupling"):
//   * Eq. (Eqn_a) / Eq. (aniso_eqn): gradient energy a = sum_{a<b} gamma_ab
//     a_c(R q_ab)^2 |q_ab|^2, q_ab = phi_a grad phi_b - phi_b grad phi_a, with the
//     four-fold a_c(q) = 1 - delta (3 - 4 sum_i q_i^4 / |q|^4).
//   * Eq. (Obstacle) / Eq. (Well): multi-obstacle / multi-well potential w(phi).
//   * Eq. (hphi): interpolation h_a; psi = sum_a h_a psi^a.
//   * Eq. (phi_eqn): tau eps dphi_a/dt = eps (div da/dgrad phi_a - da/dphi_a)
//     - (1/eps) dw/dphi_a - dpsi/dphi_a - lambda, lambda enforcing sum phi = 1.
//   * Eq. (Mu_explicit_temperature): dmu/dt = chi^-1 [div(M grad mu)
//     - sum_a c^a dh_a/dt - dT/dt sum_a (dc^a/dT)_mu h_a].
//   * Eq. (free_energy_density), Eqs. (Coeff_B), (Coeff_C): parabolic f^a.
//   * Eq. (jatr) and the obstacle / well forms of j^{at,alpha} below it: the
//     anti-trapping current, subtracted from M grad mu inside the divergence
//     of Eq. (Mu_explicit_temperature) when enabled.
//   * Sec. 4 "Grain-growth" (GRAINGROWTH = 1): isotropic grain growth, read as
//     the phi equation without the chemical term dpsi/dphi and with mu held.
//   * Sec. 2 "Elasticity implementation" (homogeneous stiffness): the elastic
//     driving force arrives as a per-phase field `elw` (computed by the Python
//     side of the oracle with an FFT) and is added to the phase potentials.
//
// Readings where the paper is silent or ambiguous (all listed in the design
// notes): unit-spacing finite differences with face fluxes (normal difference,
// 4-point averaged tangential differences, arithmetic face averages); centre
// terms with central differences; lambda realised as the Euclidean projection
// onto the simplex (obstacle) or the sum-one hyperplane (well); g = dA/dq := 0
// when |q|^2 < 1e-12 for an anisotropic pair, g = 2 gamma q for an isotropic
// pair (delta_ab == 0); the sum in Eq. (free_energy_density) taken over i <= j;
// the off-diagonal sum in Eq. (Coeff_B) with the sign its own equal-mu
// condition gives; "slopes" read as dc_eq/dT; chi evaluated with h(phi^{n+1}),
// c^a with mu^n; dh/dt and dT/dt as forward differences over one step; the
// face mobility the arithmetic mean of the two cell mobilities
// M = sum_a h_a D^a chi^a (matrix product); no-flux boundaries as mirror ghost
// cells (ghost = adjacent interior cell), periodic ones as index wrap; the
// temperature gradient along the last axis (z in 3-D, y in 2-D); the liquid
// (phase N-1) is the reference phase with B^l = C^l = 0; f0^a is a constant
// added to C^a (isothermal driving force).
//
// The step is templated on the scalar so that the same plain code, run with a
// forward-mode dual number, yields the exact tangent of the discrete step with
// respect to the initial fields, the anisotropy strengths, the phase-field
// mobility 1/tau and the diffusivities.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr int NMAX = 64;   // phases (the dense CUDA path takes at most 8; sparse grain growth more)
constexpr int KMAX = 3;   // independent solutes
constexpr double PI = 3.14159265358979323846;

// ---------------------------------------------------------------- dual number
struct Dual {
  double v = 0.0, d = 0.0;
  Dual() = default;
  Dual(double x) : v(x), d(0.0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
inline Dual operator-(Dual a) { return {-a.v, -a.d}; }
inline Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
inline Dual operator/(Dual a, Dual b) {
  return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)};
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
inline double sqrt_s(double x) { return std::sqrt(x); }
inline Dual sqrt_s(const Dual& x) {
  const double r = std::sqrt(x.v);
  return {r, x.d / (2.0 * r)};
}

// ------------------------------------------------------- op-counting scalar
// A double that counts the arithmetic done on it: every binary +, -, *, / and
// every square root with at least one counted operand adds one to g_ops
// (negation is a sign flip and counts nothing).  Arithmetic on parameters
// alone (plain doubles) is not counted: it does not depend on the state.
// Used only by oracle_count_flops, which runs single-threaded.
uint64_t g_ops = 0;
struct Cnt {
  double v = 0.0;
  Cnt() = default;
  Cnt(double x) : v(x) {}
};
inline Cnt operator+(Cnt a, Cnt b) { ++g_ops; return {a.v + b.v}; }
inline Cnt operator-(Cnt a, Cnt b) { ++g_ops; return {a.v - b.v}; }
inline Cnt operator-(Cnt a) { return {-a.v}; }
inline Cnt operator*(Cnt a, Cnt b) { ++g_ops; return {a.v * b.v}; }
inline Cnt operator/(Cnt a, Cnt b) { ++g_ops; return {a.v / b.v}; }
inline Cnt& operator+=(Cnt& a, Cnt b) { a = a + b; return a; }
inline Cnt& operator-=(Cnt& a, Cnt b) { a = a - b; return a; }
inline double val(const Cnt& x) { return x.v; }
inline Cnt sqrt_s(const Cnt& x) { ++g_ops; return {std::sqrt(x.v)}; }

// ------------------------------------------------------- reverse-mode tape
// A minimal tape for the reverse adjoint: every operation with a recorded
// operand appends a node holding its (at most two) operands and the partial
// derivatives with respect to them; a constant (no operand recorded) carries
// id -1.  The tape is global, so a step taped with Rev runs single-threaded
// (see taped<S> below).  Sweeping the nodes backwards accumulates adjoints.
struct TapeNode {
  int a, b;
  double da, db;
};
std::vector<TapeNode> g_tape;
struct Rev {
  double v = 0.0;
  int id = -1;
  Rev() = default;
  Rev(double x) : v(x), id(-1) {}
  Rev(double x, int i) : v(x), id(i) {}
};
inline Rev rev_node(double v, int a, double da, int b, double db) {
  if (a < 0 && b < 0) return Rev(v);
  g_tape.push_back({a, b, da, db});
  return Rev(v, (int)g_tape.size() - 1);
}
inline Rev rev_leaf(double v) {   // an independent input
  g_tape.push_back({-1, -1, 0.0, 0.0});
  return Rev(v, (int)g_tape.size() - 1);
}
inline Rev operator+(Rev x, Rev y) { return rev_node(x.v + y.v, x.id, 1.0, y.id, 1.0); }
inline Rev operator-(Rev x, Rev y) { return rev_node(x.v - y.v, x.id, 1.0, y.id, -1.0); }
inline Rev operator-(Rev x) { return rev_node(-x.v, x.id, -1.0, -1, 0.0); }
inline Rev operator*(Rev x, Rev y) { return rev_node(x.v * y.v, x.id, y.v, y.id, x.v); }
inline Rev operator/(Rev x, Rev y) {
  const double q = x.v / y.v;
  return rev_node(q, x.id, 1.0 / y.v, y.id, -q / y.v);
}
inline Rev& operator+=(Rev& x, Rev y) { x = x + y; return x; }
inline Rev& operator-=(Rev& x, Rev y) { x = x - y; return x; }
inline double val(const Rev& x) { return x.v; }
inline Rev sqrt_s(const Rev& x) {
  const double r = std::sqrt(x.v);
  return rev_node(r, x.id, 0.5 / r, -1, 0.0);
}

// A step may run its cell loops in parallel unless its scalar records onto
// the global tape.
template <class S>
constexpr bool taped() { return false; }
template <>
constexpr bool taped<Rev>() { return true; }

}  // namespace

extern "C" {

// Problem description handed in from Python (all arrays row-major, doubles).
typedef struct {
  int dim, nx, ny, nz;
  int bc[3];          // per axis: 3 = periodic, 1 = no-flux (paper codes)
  int N, NM;          // phases, independent solutes (components - 1)
  int potential;      // 1 = multi-obstacle, 2 = multi-well (Function_W)
  double dx, dt, eps, tau;
  const double* gamma;   // [N][N]
  const double* delta;   // [N][N]
  const double* rot;     // [N][N][3][3] or NULL (identity)
  const double* gamma3;  // [N][N][N] or NULL
  const double* D;       // [N][NM][NM]
  const double* A;       // [N][NM][NM], entries i <= j used
  const double* ceq;     // [N][NM] at T_ref
  const double* slopes;  // [N][NM]  dc_eq/dT
  const double* f0;      // [N] or NULL
  double T_ref, T0, G, z0, V;
  double t0;             // physical time of the input state
  int z_origin;          // lab index of the first cell along the last axis
  double noise_amp;      // phi noise amplitude (0 = off)
  unsigned long long noise_seed;
  long long step0;       // step index of the input state (noise counter)
  int anti_trapping;     // 1 = anti-trapping current j_at in the mu update
  int grain_growth;      // 1 = GRAINGROWTH: no chemical driving force, mu frozen
  const double* elw;     // [N][cells] elastic part of the potential of each phase, or NULL
  int active_set;        // 1 = the projection acts on the locally active phases only (see phi_cell)
} oracle_problem;

}  // extern "C"

namespace {

// Differentiable parameters (the rest of the problem stays double).
template <class S>
struct Prm {
  S delta[NMAX][NMAX];
  S mob;                     // phase-field mobility 1/tau
  S D[NMAX][KMAX][KMAX];
};

template <class S>
struct Ctx {
  const oracle_problem* p;
  Prm<S> q;
  int n[3];
  int64_t cells;
};

// ------------------------------------------------------------------- indexing
inline int map_axis(int i, int n, int bc) {
  if (i >= 0 && i < n) return i;
  if (bc == 3) return ((i % n) + n) % n;      // periodic: wrap
  return i < 0 ? 0 : n - 1;                    // no-flux: mirror ghost
}

template <class S>
inline int64_t cell_index(const Ctx<S>& c, int x, int y, int z) {
  x = map_axis(x, c.n[0], c.p->bc[0]);
  y = map_axis(y, c.n[1], c.p->bc[1]);
  z = map_axis(z, c.n[2], c.p->bc[2]);
  return (static_cast<int64_t>(z) * c.n[1] + y) * c.n[0] + x;
}

// ------------------------------------------------------ anisotropic energy A
// A_ab(q) = gamma_ab a_c(R q)^2 |q|^2 (Eq. aniso_eqn), a_c from the four-fold form.
template <class S>
S pair_energy(const Ctx<S>& c, int a, int b, const S* q) {
  const oracle_problem& p = *c.p;
  const int d = p.dim;
  const double gam = p.gamma[a * p.N + b];
  S Q = 0.0;
  for (int i = 0; i < d; ++i) Q += q[i] * q[i];
  S del = c.q.delta[a][b];
  if (val(del) == 0.0) return gam * Q;
  if (val(Q) < 1e-12) return S(0.0);
  S qr[3];
  for (int i = 0; i < d; ++i) {
    qr[i] = 0.0;
    for (int j = 0; j < d; ++j) {
      double R = p.rot ? p.rot[((a * p.N + b) * 3 + i) * 3 + j] : (i == j ? 1.0 : 0.0);
      qr[i] += R * q[j];
    }
  }
  S s4 = 0.0;
  for (int i = 0; i < d; ++i) s4 += qr[i] * qr[i] * qr[i] * qr[i];
  S ac = 1.0 - del * (3.0 - 4.0 * s4 / (Q * Q));
  return gam * ac * ac * Q;
}

// g = dA_ab/dq, derived by hand from pair_energy (checked against a finite
// difference of pair_energy in the tests).
template <class S>
void pair_energy_grad(const Ctx<S>& c, int a, int b, const S* q, S* g) {
  const oracle_problem& p = *c.p;
  const int d = p.dim;
  const double gam = p.gamma[a * p.N + b];
  S del = c.q.delta[a][b];
  if (val(del) == 0.0) {
    for (int i = 0; i < d; ++i) g[i] = 2.0 * gam * q[i];
    return;
  }
  S Q = 0.0;
  for (int i = 0; i < d; ++i) Q += q[i] * q[i];
  if (val(Q) < 1e-12) {
    for (int i = 0; i < d; ++i) g[i] = 0.0;
    return;
  }
  double R[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      R[i][j] = p.rot ? p.rot[((a * p.N + b) * 3 + i) * 3 + j] : (i == j ? 1.0 : 0.0);
  S qr[3];
  for (int i = 0; i < d; ++i) {
    qr[i] = 0.0;
    for (int j = 0; j < d; ++j) qr[i] += R[i][j] * q[j];
  }
  S s4 = 0.0;
  for (int i = 0; i < d; ++i) s4 += qr[i] * qr[i] * qr[i] * qr[i];
  S ac = 1.0 - del * (3.0 - 4.0 * s4 / (Q * Q));
  S gr[3];
  for (int i = 0; i < d; ++i)
    gr[i] = 2.0 * gam * ac *
            (ac * qr[i] + 16.0 * del * (qr[i] * qr[i] * qr[i] / Q - s4 * qr[i] / (Q * Q)));
  for (int j = 0; j < d; ++j) {   // back-rotate: g = R^T g'
    g[j] = 0.0;
    for (int i = 0; i < d; ++i) g[j] += R[i][j] * gr[i];
  }
}

// ---------------------------------------------------------- potential w(phi)
template <class S>
S potential_w(const oracle_problem& p, const S* phi) {
  S w = 0.0;
  for (int a = 0; a < p.N; ++a)
    for (int b = a + 1; b < p.N; ++b) {
      double gam = p.gamma[a * p.N + b];
      if (p.potential == 1)
        w += (16.0 / (PI * PI)) * gam * phi[a] * phi[b];
      else
        w += 9.0 * gam * phi[a] * phi[a] * phi[b] * phi[b];
    }
  if (p.gamma3)
    for (int a = 0; a < p.N; ++a)
      for (int b = a + 1; b < p.N; ++b)
        for (int e = b + 1; e < p.N; ++e)
          w += p.gamma3[(a * p.N + b) * p.N + e] * phi[a] * phi[b] * phi[e];
  return w;
}

// dw/dphi_a, written out term by term from potential_w.
template <class S>
void potential_dw(const oracle_problem& p, const S* phi, S* W) {
  for (int a = 0; a < p.N; ++a) {
    W[a] = 0.0;
    for (int b = 0; b < p.N; ++b) {
      if (b == a) continue;
      double gam = p.gamma[a * p.N + b];
      if (p.potential == 1)
        W[a] += (16.0 / (PI * PI)) * gam * phi[b];
      else
        W[a] += 18.0 * gam * phi[a] * phi[b] * phi[b];
    }
    if (p.gamma3)
      for (int b = 0; b < p.N; ++b)
        for (int e = b + 1; e < p.N; ++e)
          if (b != a && e != a) W[a] += p.gamma3[(a * p.N + b) * p.N + e] * phi[b] * phi[e];
  }
}

// ------------------------------------------------------ interpolation h(phi)
template <class S>
void interp_h(int N, const S* phi, S* h) {
  for (int a = 0; a < N; ++a) {
    S pair_sum = 0.0;
    for (int b = 0; b < N; ++b)
      for (int e = b + 1; e < N; ++e)
        if (b != a && e != a) pair_sum += phi[b] * phi[e];
    h[a] = 3.0 * phi[a] * phi[a] - 2.0 * phi[a] * phi[a] * phi[a] + 2.0 * phi[a] * pair_sum;
  }
}

// dh[b*N + a] = d h_b / d phi_a
template <class S>
void interp_dh(int N, const S* phi, S* dh) {
  for (int b = 0; b < N; ++b)
    for (int a = 0; a < N; ++a) {
      if (a == b) {
        S pair_sum = 0.0;
        for (int u = 0; u < N; ++u)
          for (int v = u + 1; v < N; ++v)
            if (u != a && v != a) pair_sum += phi[u] * phi[v];
        dh[b * N + a] = 6.0 * phi[a] - 6.0 * phi[a] * phi[a] + 2.0 * pair_sum;
      } else {
        S rest = 0.0;
        for (int u = 0; u < N; ++u)
          if (u != a && u != b) rest += phi[u];
        dh[b * N + a] = 2.0 * phi[b] * rest;
      }
    }
}

// ------------------------------------------------------------ thermodynamics
// Parabolic f^a(c) = sum_{i<=j} A_ij c_i c_j + sum_j B_j c_j + C (V_m = 1).
inline double A_entry(const oracle_problem& p, int a, int i, int j) {
  if (i > j) std::swap(i, j);
  return p.A[(a * p.NM + i) * p.NM + j];
}

void ceq_at(const oracle_problem& p, int a, double T, double* c) {
  for (int i = 0; i < p.NM; ++i)
    c[i] = p.ceq[a * p.NM + i] + p.slopes[a * p.NM + i] * (T - p.T_ref);
}

// Eq. (Coeff_B), off-diagonal sign from the equal-mu condition; liquid B = 0.
void coeff_B(const oracle_problem& p, int a, double T, double* B) {
  const int L = p.N - 1;
  if (a == L) {
    for (int j = 0; j < p.NM; ++j) B[j] = 0.0;
    return;
  }
  double ca[KMAX], cl[KMAX];
  ceq_at(p, a, T, ca);
  ceq_at(p, L, T, cl);
  for (int j = 0; j < p.NM; ++j) {
    B[j] = 2.0 * (A_entry(p, L, j, j) * cl[j] - A_entry(p, a, j, j) * ca[j]);
    for (int i = 0; i < p.NM; ++i)
      if (i != j) B[j] += A_entry(p, L, i, j) * cl[i] - A_entry(p, a, i, j) * ca[i];
  }
}

// Eq. (Coeff_C) plus the constant offset f0^a.
double coeff_C(const oracle_problem& p, int a, double T) {
  const int L = p.N - 1;
  double ca[KMAX], cl[KMAX];
  ceq_at(p, a, T, ca);
  ceq_at(p, L, T, cl);
  double C = 0.0;
  for (int i = 0; i < p.NM; ++i)
    for (int j = i; j < p.NM; ++j)
      C += A_entry(p, a, i, j) * ca[i] * ca[j] - A_entry(p, L, i, j) * cl[i] * cl[j];
  if (p.f0) C += p.f0[a];
  return C;
}

// Hessian of f^a: H_ii = 2 A_ii, H_ij = A_ij (i != j).
void hessian(const oracle_problem& p, int a, double* H) {
  for (int i = 0; i < p.NM; ++i)
    for (int j = 0; j < p.NM; ++j)
      H[i * p.NM + j] = (i == j ? 2.0 : 1.0) * A_entry(p, a, i, j);
}

// Dense inverse by Gauss-Jordan with partial pivoting (n <= KMAX).
template <class S>
void invert(int n, const S* M, S* out) {
  S a[KMAX][2 * KMAX];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) a[i][j] = j < n ? M[i * n + j] : S(i == j - n ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(val(a[r][c])) > std::fabs(val(a[piv][c]))) piv = r;
    if (piv != c)
      for (int j = 0; j < 2 * n; ++j) std::swap(a[c][j], a[piv][j]);
    S d = a[c][c];
    for (int j = 0; j < 2 * n; ++j) a[c][j] = a[c][j] / d;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      S f = a[r][c];
      for (int j = 0; j < 2 * n; ++j) a[r][j] = a[r][j] - f * a[c][j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) out[i * n + j] = a[i][j + n];
}

// chi^a = (d c^a / d mu) = H^-1.
void chi_phase(const oracle_problem& p, int a, double* chi) {
  double H[KMAX * KMAX];
  hessian(p, a, H);
  invert<double>(p.NM, H, chi);
}

// c^a(mu, T) solves d f^a / dc = mu, i.e. H c + B = mu.
template <class S>
void comp_of_mu(const oracle_problem& p, int a, const S* mu, double T, S* c) {
  double chi[KMAX * KMAX], B[KMAX];
  chi_phase(p, a, chi);
  coeff_B(p, a, T, B);
  for (int i = 0; i < p.NM; ++i) {
    c[i] = 0.0;
    for (int j = 0; j < p.NM; ++j) c[i] += chi[i * p.NM + j] * (mu[j] - B[j]);
  }
}

// psi^a(mu, T) = f^a(c^a(mu,T)) - mu . c^a(mu,T).
template <class S>
S grand_potential(const oracle_problem& p, int a, const S* mu, double T) {
  S c[KMAX];
  comp_of_mu(p, a, mu, T, c);
  double B[KMAX];
  coeff_B(p, a, T, B);
  S f = coeff_C(p, a, T);
  for (int i = 0; i < p.NM; ++i) {
    for (int j = i; j < p.NM; ++j) f += A_entry(p, a, i, j) * c[i] * c[j];
    f += B[i] * c[i];
  }
  S mc = 0.0;
  for (int i = 0; i < p.NM; ++i) mc += mu[i] * c[i];
  return f - mc;
}

// Temperature at a cell centre (frozen, pulled gradient along the last axis,
// in lab coordinates: the grid starts at lab index z_origin).
double temperature(const oracle_problem& p, int y, int z, double t) {
  int k = (p.dim == 3 ? z : y) + p.z_origin;
  double s = (k + 0.5) * p.dx;
  return p.T0 + p.G * (s - p.z0 - p.V * t);
}

// ------------------------------------------------------------------ noise
// Counter-based uniform variate in [-1/2, 1/2): the SplitMix64 finaliser
// (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
// OOPSLA 2014) applied in turn to the seed, the step index and the lab cell
// index times N plus the phase; the top 24 bits of the last value.
inline uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

inline double noise_variate(uint64_t seed, uint64_t step, uint64_t counter) {
  uint64_t h = splitmix64(seed);
  h = splitmix64(h ^ step);
  h = splitmix64(h ^ counter);
  return static_cast<double>(h >> 40) * (1.0 / 16777216.0) - 0.5;
}

// ------------------------------------------------------- simplex projection
// Euclidean projection onto {phi >= 0, sum phi = 1}: sort-based method
// (Held, Wolfe & Crowder 1974; Duchi et al. 2008).
template <class S>
void project_simplex(int N, const S* v, S* out) {
  S u[NMAX];
  for (int a = 0; a < N; ++a) u[a] = v[a];
  std::sort(u, u + N, [](const S& x, const S& y) { return val(x) > val(y); });
  S csum = 0.0, theta = 0.0;
  for (int j = 0; j < N; ++j) {
    csum += u[j];
    S t = (csum - 1.0) / double(j + 1);
    if (val(u[j]) - val(t) > 0.0) theta = t;
  }
  for (int a = 0; a < N; ++a) {
    S d = v[a] - theta;
    out[a] = val(d) > 0.0 ? d : S(0.0);
  }
}

template <class S>
void project_hyperplane(int N, const S* v, S* out) {
  S s = 0.0;
  for (int a = 0; a < N; ++a) s += v[a];
  S shift = (s - 1.0) / double(N);
  for (int a = 0; a < N; ++a) out[a] = v[a] - shift;
}

// --------------------------------------------------------------- face fluxes
// Normal component (along axis d) of J_a = da/dgrad phi_a at the face between
// cell (x,y,z) and its +d neighbour, for every phase a.
template <class S>
void face_flux(const Ctx<S>& c, const S* phi, int x, int y, int z, int d, S* Jn) {
  const oracle_problem& p = *c.p;
  const int N = p.N, dim = p.dim;
  int L[3] = {x, y, z}, Rr[3] = {x, y, z};
  Rr[d] += 1;
  auto at = [&](int a, const int* pos, int t, int s) {
    int q[3] = {pos[0], pos[1], pos[2]};
    if (t >= 0) q[t] += s;
    return phi[a * c.cells + cell_index(c, q[0], q[1], q[2])];
  };
  S pf[NMAX], gr[NMAX][3];
  for (int a = 0; a < N; ++a) {
    S vl = at(a, L, -1, 0), vr = at(a, Rr, -1, 0);
    pf[a] = 0.5 * (vl + vr);
    for (int t = 0; t < dim; ++t) {
      if (t == d)
        gr[a][t] = (vr - vl) / p.dx;
      else
        gr[a][t] = ((at(a, L, t, +1) + at(a, Rr, t, +1)) - (at(a, L, t, -1) + at(a, Rr, t, -1))) /
                   (4.0 * p.dx);
    }
  }
  for (int a = 0; a < N; ++a) Jn[a] = 0.0;
  for (int a = 0; a < N; ++a)
    for (int b = a + 1; b < N; ++b) {
      S q[3], g[3];
      for (int t = 0; t < dim; ++t) q[t] = pf[a] * gr[b][t] - pf[b] * gr[a][t];
      pair_energy_grad(c, a, b, q, g);
      Jn[a] -= pf[b] * g[d];   // da/dgrad phi_a = -sum_b phi_b g_ab(q_ab)
      Jn[b] += pf[a] * g[d];   // q_ba = -q_ab, g odd
    }
}

// Per-cell parts of the phi rate: divergence term, centre term, potential and
// driving force (before the projection that realises lambda).
template <class S>
void rate_parts(const Ctx<S>& c, const S* phi, const S* mu, int x, int y, int z, double t,
                S* divJ, S* Gc, S* W, S* P) {
  const oracle_problem& p = *c.p;
  const int N = p.N, dim = p.dim;
  const int64_t ic = cell_index(c, x, y, z);
  for (int a = 0; a < N; ++a) divJ[a] = 0.0;
  int pos[3] = {x, y, z};
  for (int d = 0; d < dim; ++d) {
    S Jp[NMAX], Jm[NMAX];
    face_flux(c, phi, x, y, z, d, Jp);
    int q[3] = {pos[0], pos[1], pos[2]};
    q[d] -= 1;
    face_flux(c, phi, q[0], q[1], q[2], d, Jm);
    for (int a = 0; a < N; ++a) divJ[a] += (Jp[a] - Jm[a]) / p.dx;
  }
  // centre term da/dphi_a = sum_b g_ab(q_ab) . grad phi_b, central differences
  S ph[NMAX], gc[NMAX][3];
  for (int a = 0; a < N; ++a) {
    ph[a] = phi[a * c.cells + ic];
    for (int d = 0; d < dim; ++d) {
      int u[3] = {x, y, z}, v[3] = {x, y, z};
      u[d] += 1;
      v[d] -= 1;
      gc[a][d] = (phi[a * c.cells + cell_index(c, u[0], u[1], u[2])] -
                  phi[a * c.cells + cell_index(c, v[0], v[1], v[2])]) / (2.0 * p.dx);
    }
  }
  for (int a = 0; a < N; ++a) Gc[a] = 0.0;
  for (int a = 0; a < N; ++a)
    for (int b = a + 1; b < N; ++b) {
      S q[3], g[3];
      for (int d = 0; d < dim; ++d) q[d] = ph[a] * gc[b][d] - ph[b] * gc[a][d];
      pair_energy_grad(c, a, b, q, g);
      for (int d = 0; d < dim; ++d) {
        Gc[a] += g[d] * gc[b][d];
        Gc[b] -= g[d] * gc[a][d];
      }
    }
  potential_dw(p, ph, W);
  const double T = temperature(p, y, z, t);
  S psi[NMAX], mloc[KMAX], dh[NMAX * NMAX];
  for (int i = 0; i < p.NM; ++i) mloc[i] = mu[i * c.cells + ic];
  // the elastic energy enters like a phase potential: d f_el / d phi_a =
  // sum_b (-sigma : eps*^b) dh_b / dphi_a (homogeneous stiffness, eigenstrain
  // interpolated with h; the field comes from the FFT equilibrium solve)
  for (int b = 0; b < N; ++b)
    psi[b] = grand_potential(p, b, mloc, T) + (p.elw ? p.elw[b * c.cells + ic] : 0.0);
  interp_dh(N, ph, dh);
  for (int a = 0; a < N; ++a) {
    P[a] = 0.0;
    for (int b = 0; b < N; ++b) P[a] += psi[b] * dh[b * N + a];
  }
}

// Mobility matrix of one cell: M = sum_a h_a(phi) D^a chi^a.
template <class S>
void cell_mobility(const Ctx<S>& c, const S* phi, int64_t ic, S* M) {
  const oracle_problem& p = *c.p;
  const int NM = p.NM;
  S ph[NMAX], h[NMAX];
  for (int a = 0; a < p.N; ++a) ph[a] = phi[a * c.cells + ic];
  interp_h(p.N, ph, h);
  for (int i = 0; i < NM * NM; ++i) M[i] = 0.0;
  for (int a = 0; a < p.N; ++a) {
    double chi[KMAX * KMAX];
    chi_phase(p, a, chi);
    for (int i = 0; i < NM; ++i)
      for (int j = 0; j < NM; ++j) {
        S dc = 0.0;
        for (int k = 0; k < NM; ++k) dc += c.q.D[a][i][k] * chi[k * NM + j];
        M[i * NM + j] += h[a] * dc;
      }
  }
}

// ------------------------------------------------------ anti-trapping current
// Coefficient of j^{at,alpha} (the two forms below Eq. jatr) at the local
// value phi0 of phi_alpha, read as the equilibrium 1-D profile value there:
// obstacle  pi eps phi0 (1 - h(phi0)) / (4 sqrt(phi0 (1 - phi0))), with h the
//           two-phase restriction phi0^2 (3 - 2 phi0) of Eq. (hphi) (the 1-D
//           profile holds two phases); 0 outside 0 < phi0 < 1;
// well      eps / (2 sqrt 2).
template <class S>
S at_coefficient(const oracle_problem& p, S phi0) {
  if (p.potential != 1) return S(p.eps / (2.0 * std::sqrt(2.0)));
  if (!(val(phi0) > 0.0 && val(phi0) < 1.0)) return S(0.0);
  const S h = phi0 * phi0 * (3.0 - 2.0 * phi0);
  const double pi = 3.14159265358979323846;
  return pi * p.eps * phi0 * (1.0 - h) / (4.0 * sqrt_s(phi0 * (1.0 - phi0)));
}

// Normal component (along axis d) of the anti-trapping current j_at_i
// (Eq. jatr) at the face between cell (x,y,z) and its +d neighbour, for every
// solute i.  phi = phi^n, phin = phi^{n+1}, mu = mu^n at time t.  Face values
// as for the gradient-energy fluxes: the arithmetic mean of the two cells for
// phi, mu and d phi/dt (each cell's forward difference over the step), the
// normal difference and 4-point averaged tangential differences for grad phi;
// the mean of the two cells' T.  The liquid is phase N-1; a phase whose face gradient
// has |grad phi|^2 < 1e-12 has no normal and contributes nothing.
template <class S>
void at_face_flux(const Ctx<S>& c, const S* phi, const S* phin, const S* mu, int x, int y, int z, int d,
                  double t, S* J) {
  const oracle_problem& p = *c.p;
  const int N = p.N, NM = p.NM, dim = p.dim, liq = N - 1;
  int L[3] = {x, y, z}, R[3] = {x, y, z};
  R[d] += 1;
  auto at = [&](const S* f, int a, const int* pos, int tt, int sgn) {
    int q[3] = {pos[0], pos[1], pos[2]};
    if (tt >= 0) q[tt] += sgn;
    return f[a * c.cells + cell_index(c, q[0], q[1], q[2])];
  };
  S pf[NMAX], rate[NMAX], nrm[NMAX][3];
  bool has_n[NMAX];
  for (int a = 0; a < N; ++a) {
    const S vl = at(phi, a, L, -1, 0), vr = at(phi, a, R, -1, 0);
    pf[a] = 0.5 * (vl + vr);
    rate[a] = 0.5 * ((at(phin, a, L, -1, 0) - vl) + (at(phin, a, R, -1, 0) - vr)) / p.dt;
    S gr[3] = {0.0, 0.0, 0.0}, g2 = 0.0;
    for (int tt = 0; tt < dim; ++tt) {
      if (tt == d)
        gr[tt] = (vr - vl) / p.dx;
      else
        gr[tt] = ((at(phi, a, L, tt, +1) + at(phi, a, R, tt, +1)) - (at(phi, a, L, tt, -1) + at(phi, a, R, tt, -1))) /
                 (4.0 * p.dx);
      g2 += gr[tt] * gr[tt];
    }
    has_n[a] = val(g2) >= 1e-12;
    const S inv = has_n[a] ? 1.0 / sqrt_s(g2) : S(0.0);
    for (int tt = 0; tt < 3; ++tt) nrm[a][tt] = gr[tt] * inv;
  }
  S mf[KMAX];
  for (int i = 0; i < NM; ++i) mf[i] = 0.5 * (at(mu, i, L, -1, 0) + at(mu, i, R, -1, 0));
  // T: the mean of the two cells' temperatures (cells taken after the
  // boundary mapping, so that a wrapped face has one value from either side)
  const int yl = map_axis(L[1], c.n[1], p.bc[1]), yr = map_axis(R[1], c.n[1], p.bc[1]);
  const int zl = map_axis(L[2], c.n[2], p.bc[2]), zr = map_axis(R[2], c.n[2], p.bc[2]);
  const double Tf = 0.5 * (temperature(p, yl, zl, t) + temperature(p, yr, zr, t));
  S cl[KMAX];
  comp_of_mu(p, liq, mf, Tf, cl);
  for (int i = 0; i < NM; ++i) J[i] = 0.0;
  if (!has_n[liq]) return;
  for (int al = 0; al < N - 1; ++al) {
    if (!has_n[al]) continue;
    S proj = 0.0;   // -n_alpha . n_liq
    for (int tt = 0; tt < dim; ++tt) proj -= nrm[al][tt] * nrm[liq][tt];
    S ca[KMAX];
    comp_of_mu(p, al, mf, Tf, ca);
    const S k = at_coefficient(p, pf[al]) * rate[al] * nrm[al][d] * proj;
    for (int i = 0; i < NM; ++i) J[i] += k * (ca[i] - cl[i]);
  }
}

// One explicit step phi^n, mu^n (time t) -> phi^{n+1}, mu^{n+1}.
// phi^{n+1} of cell (x, y, z): Eq. (phi_eqn) explicit Euler and the
// projection (first sweep of a step).
template <class S>
void phi_cell(const Ctx<S>& c, const S* phi, const S* mu, int x, int y, int z, double t, int64_t nstep,
              S* phi_out) {
  const oracle_problem& p = *c.p;
  const int N = p.N, dim = p.dim;
  const int64_t ic = cell_index(c, x, y, z);
  S divJ[NMAX], Gc[NMAX], W[NMAX], P[NMAX];
  rate_parts(c, phi, mu, x, y, z, t, divJ, Gc, W, P);
  S ph[NMAX], v[NMAX], pn[NMAX];
  for (int a = 0; a < N; ++a) {
    ph[a] = phi[a * c.cells + ic];
    // grain growth (GRAINGROWTH = 1, Sec. 4 "Grain-growth"): the
    // interfaces move by their curvature only, no dpsi/dphi term
    const S Pa = p.grain_growth ? S(0.0) : P[a];
    S r = c.q.mob * (p.eps * (divJ[a] - Gc[a]) - W[a] / p.eps - Pa) / p.eps;
    v[a] = ph[a] + p.dt * r;
    // phi noise on the cell's interface phases (0 < phi_a < 1): an
    // additive dt * amplitude * xi on the rate, before the projection
    if (p.noise_amp != 0.0 && val(ph[a]) > 0.0 && val(ph[a]) < 1.0) {
      const int64_t ylab = dim == 3 ? y : y + p.z_origin;
      const int64_t zlab = dim == 3 ? z + p.z_origin : 0;
      const uint64_t gcell = static_cast<uint64_t>(x + (int64_t)c.n[0] * (ylab + (int64_t)c.n[1] * zlab));
      v[a] += p.dt * p.noise_amp * noise_variate(p.noise_seed, (uint64_t)nstep, gcell * N + a);
    }
  }
  if (p.active_set) {
    // locally active phases (the multiphase-field form of the Lagrange
    // multiplier over the phases present at a point): those non-zero at the
    // cell or at one of its 2 dim face neighbours; the projection acts on
    // them alone and every other phase stays 0
    bool act[NMAX];
    for (int a = 0; a < N; ++a) act[a] = val(ph[a]) > 0.0;
    for (int d = 0; d < dim; ++d)
      for (int s = -1; s <= 1; s += 2) {
        int u[3] = {x, y, z};
        u[d] += s;
        const int64_t in = cell_index(c, u[0], u[1], u[2]);
        for (int a = 0; a < N; ++a) act[a] = act[a] || val(phi[a * c.cells + in]) > 0.0;
      }
    S va[NMAX], pa[NMAX];
    int na = 0;
    for (int a = 0; a < N; ++a)
      if (act[a]) va[na++] = v[a];
    if (p.potential == 1)
      project_simplex(na, va, pa);
    else
      project_hyperplane(na, va, pa);
    na = 0;
    for (int a = 0; a < N; ++a) pn[a] = act[a] ? pa[na++] : S(0.0);
  } else if (p.potential == 1) {
    project_simplex(N, v, pn);
  } else {
    project_hyperplane(N, v, pn);
  }
  for (int a = 0; a < N; ++a) phi_out[a * c.cells + ic] = pn[a];
}

// mu^{n+1} of cell (x, y, z): Eq. (Mu_explicit_temperature) with the
// mobility of Eq. (Mass_conservation) (second sweep of a step; phi_out holds
// phi^{n+1} of every cell, which the anti-trapping current reads).
template <class S>
void mu_cell(const Ctx<S>& c, const S* phi, const S* mu, const S* phi_out, int x, int y, int z, double t,
             S* mu_out) {
  const oracle_problem& p = *c.p;
  const int N = p.N, NM = p.NM, dim = p.dim;
  const int64_t ic = cell_index(c, x, y, z);
  S ph[NMAX], pn[NMAX];
  for (int a = 0; a < N; ++a) {
    ph[a] = phi[a * c.cells + ic];
    pn[a] = phi_out[a * c.cells + ic];
  }
  S h_old[NMAX], h_new[NMAX];
  interp_h(N, ph, h_old);
  interp_h(N, pn, h_new);
  S Mc[KMAX * KMAX], mc[KMAX];
  cell_mobility(c, phi, ic, Mc);
  for (int i = 0; i < NM; ++i) mc[i] = mu[i * c.cells + ic];
  S div[KMAX];
  for (int i = 0; i < NM; ++i) div[i] = 0.0;
  for (int d = 0; d < dim; ++d)
    for (int s = -1; s <= 1; s += 2) {
      int u[3] = {x, y, z};
      u[d] += s;
      const int64_t in = cell_index(c, u[0], u[1], u[2]);
      S Mn[KMAX * KMAX];
      cell_mobility(c, phi, in, Mn);
      for (int i = 0; i < NM; ++i)
        for (int j = 0; j < NM; ++j) {
          S Mf = 0.5 * (Mc[i * NM + j] + Mn[i * NM + j]);
          div[i] += Mf * (mu[j * c.cells + in] - mc[j]) / (p.dx * p.dx);
        }
    }
  if (p.anti_trapping) {   // - div j_at (Eq. Mu_explicit_temperature)
    for (int d = 0; d < dim; ++d) {
      S Jp[KMAX], Jm[KMAX];
      at_face_flux(c, phi, phi_out, mu, x, y, z, d, t, Jp);
      int q[3] = {x, y, z};
      q[d] -= 1;
      at_face_flux(c, phi, phi_out, mu, q[0], q[1], q[2], d, t, Jm);
      for (int i = 0; i < NM; ++i) div[i] -= (Jp[i] - Jm[i]) / p.dx;
    }
  }
  const double Tn = temperature(p, y, z, t);
  const double Tn1 = temperature(p, y, z, t + p.dt);
  S rhs[KMAX];
  for (int i = 0; i < NM; ++i) rhs[i] = p.dt * div[i];
  for (int a = 0; a < N; ++a) {
    S c_now[KMAX], c_next[KMAX];
    comp_of_mu(p, a, mc, Tn, c_now);
    comp_of_mu(p, a, mc, Tn1, c_next);
    for (int i = 0; i < NM; ++i) {
      rhs[i] -= c_now[i] * (h_new[a] - h_old[a]);
      rhs[i] -= h_new[a] * (c_next[i] - c_now[i]);
    }
  }
  S chi[KMAX * KMAX], chinv[KMAX * KMAX];
  for (int i = 0; i < NM * NM; ++i) chi[i] = 0.0;
  for (int a = 0; a < N; ++a) {
    double ca[KMAX * KMAX];
    chi_phase(p, a, ca);
    for (int i = 0; i < NM * NM; ++i) chi[i] += h_new[a] * ca[i];
  }
  invert<S>(NM, chi, chinv);
  for (int i = 0; i < NM; ++i) {
    S dmu = 0.0;
    for (int j = 0; j < NM; ++j) dmu += chinv[i * NM + j] * rhs[j];
    mu_out[i * c.cells + ic] = mc[i] + dmu;
  }
}

template <class S>
void step(const Ctx<S>& c, const S* phi, const S* mu, S* phi_out, S* mu_out, double t, int64_t nstep) {
  const oracle_problem& p = *c.p;
#pragma omp parallel for collapse(2) schedule(dynamic, 1) if (!taped<S>())
  for (int z = 0; z < c.n[2]; ++z)
    for (int y = 0; y < c.n[1]; ++y)
      for (int x = 0; x < c.n[0]; ++x) phi_cell(c, phi, mu, x, y, z, t, nstep, phi_out);
  // ---- chemical-potential update (a second sweep: the anti-trapping current
  // needs phi^{n+1} of the neighbours); grain growth keeps mu as it is
  if (p.grain_growth) {
    for (int64_t k = 0; k < (int64_t)p.NM * c.cells; ++k) mu_out[k] = mu[k];
    return;
  }
#pragma omp parallel for collapse(2) schedule(dynamic, 1) if (!taped<S>())
  for (int z = 0; z < c.n[2]; ++z)
    for (int y = 0; y < c.n[1]; ++y)
      for (int x = 0; x < c.n[0]; ++x) mu_cell(c, phi, mu, phi_out, x, y, z, t, mu_out);
}

template <class S>
void init_ctx(Ctx<S>& c, const oracle_problem* p) {
  c.p = p;
  c.n[0] = p->nx;
  c.n[1] = p->ny;
  c.n[2] = p->dim == 3 ? p->nz : 1;
  c.cells = static_cast<int64_t>(c.n[0]) * c.n[1] * c.n[2];
  for (int a = 0; a < NMAX; ++a)
    for (int b = 0; b < NMAX; ++b) c.q.delta[a][b] = 0.0;
  for (int a = 0; a < p->N; ++a)
    for (int b = 0; b < p->N; ++b) c.q.delta[a][b] = p->delta[a * p->N + b];
  c.q.mob = 1.0 / p->tau;
  for (int a = 0; a < p->N; ++a)
    for (int i = 0; i < p->NM; ++i)
      for (int j = 0; j < p->NM; ++j) c.q.D[a][i][j] = p->D[(a * p->NM + i) * p->NM + j];
}

int check(const oracle_problem* p) {
  if (!p || p->N < 2 || p->N > NMAX || p->NM < 1 || p->NM > KMAX) return 1;
  if (p->dim != 2 && p->dim != 3) return 1;
  if (p->nx < 1 || p->ny < 1 || (p->dim == 3 && p->nz < 1)) return 1;
  if (p->potential != 1 && p->potential != 2) return 1;
  return 0;
}

}  // namespace

extern "C" {

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

// Advance nsteps explicit steps in FP64.  Fields are [N][cells] and [NM][cells].
int oracle_run(const oracle_problem* p, const double* phi0, const double* mu0, int nsteps,
               double* phi, double* mu) {
  if (check(p)) return 1;
  Ctx<double> c;
  init_ctx(c, p);
  const int64_t cells = c.cells;
  std::vector<double> pa(phi0, phi0 + p->N * cells), pb(p->N * cells);
  std::vector<double> ma(mu0, mu0 + p->NM * cells), mb(p->NM * cells);
  for (int n = 0; n < nsteps; ++n) {
    step(c, pa.data(), ma.data(), pb.data(), mb.data(), p->t0 + n * p->dt, p->step0 + n);
    pa.swap(pb);
    ma.swap(mb);
  }
  std::memcpy(phi, pa.data(), sizeof(double) * p->N * cells);
  std::memcpy(mu, ma.data(), sizeof(double) * p->NM * cells);
  return 0;
}

// Forward-mode tangent of nsteps steps along the direction (dphi0, dmu0,
// ddelta [N][N], dmob, dD [N][NM][NM]); returns the state and its tangent.
int oracle_run_tangent(const oracle_problem* p, const double* phi0, const double* mu0,
                       const double* dphi0, const double* dmu0, const double* ddelta,
                       double dmob, const double* dD, int nsteps, double* phi, double* mu,
                       double* dphi, double* dmu) {
  if (check(p)) return 1;
  Ctx<Dual> c;
  init_ctx(c, p);
  for (int a = 0; a < p->N; ++a)
    for (int b = 0; b < p->N; ++b)
      if (ddelta) c.q.delta[a][b].d = ddelta[a * p->N + b];
  c.q.mob.d = dmob;
  for (int a = 0; a < p->N; ++a)
    for (int i = 0; i < p->NM; ++i)
      for (int j = 0; j < p->NM; ++j)
        if (dD) c.q.D[a][i][j].d = dD[(a * p->NM + i) * p->NM + j];
  const int64_t cells = c.cells;
  std::vector<Dual> pa(p->N * cells), pb(p->N * cells), ma(p->NM * cells), mb(p->NM * cells);
  for (int64_t i = 0; i < p->N * cells; ++i) pa[i] = Dual(phi0[i], dphi0 ? dphi0[i] : 0.0);
  for (int64_t i = 0; i < p->NM * cells; ++i) ma[i] = Dual(mu0[i], dmu0 ? dmu0[i] : 0.0);
  for (int n = 0; n < nsteps; ++n) {
    step(c, pa.data(), ma.data(), pb.data(), mb.data(), p->t0 + n * p->dt, p->step0 + n);
    pa.swap(pb);
    ma.swap(mb);
  }
  for (int64_t i = 0; i < p->N * cells; ++i) {
    phi[i] = pa[i].v;
    dphi[i] = pa[i].d;
  }
  for (int64_t i = 0; i < p->NM * cells; ++i) {
    mu[i] = ma[i].v;
    dmu[i] = ma[i].d;
  }
  return 0;
}

// Arithmetic operations of one step, per cell, counted with the op-counting
// scalar (single-threaded): ops_phi[cells] for the phi sweep (Eq. phi_eqn,
// the projection), ops_mu[cells] for the mu sweep (Eq.
// Mu_explicit_temperature); the state is advanced as by oracle_run with one
// step, the new state is discarded.
int oracle_count_flops(const oracle_problem* p, const double* phi, const double* mu, double* ops_phi,
                       double* ops_mu) {
  if (check(p)) return 1;
  Ctx<Cnt> c;
  init_ctx(c, p);
  const int64_t cells = c.cells;
  std::vector<Cnt> pa(p->N * cells), pb(p->N * cells), ma(p->NM * cells), mb(p->NM * cells);
  for (int64_t i = 0; i < p->N * cells; ++i) pa[i] = Cnt(phi[i]);
  for (int64_t i = 0; i < p->NM * cells; ++i) ma[i] = Cnt(mu[i]);
  for (int z = 0; z < c.n[2]; ++z)
    for (int y = 0; y < c.n[1]; ++y)
      for (int x = 0; x < c.n[0]; ++x) {
        const uint64_t before = g_ops;
        phi_cell(c, pa.data(), ma.data(), x, y, z, p->t0, p->step0, pb.data());
        ops_phi[cell_index(c, x, y, z)] = static_cast<double>(g_ops - before);
      }
  for (int z = 0; z < c.n[2]; ++z)
    for (int y = 0; y < c.n[1]; ++y)
      for (int x = 0; x < c.n[0]; ++x) {
        const uint64_t before = g_ops;
        if (!p->grain_growth) mu_cell(c, pa.data(), ma.data(), pb.data(), x, y, z, p->t0, mb.data());
        ops_mu[cell_index(c, x, y, z)] = static_cast<double>(g_ops - before);
      }
  return 0;
}

// Reverse (adjoint) sweep of nsteps steps by the tape: given lam_phi / lam_mu
// = dL/dphi, dL/dmu of the final state, returns dL/dphi0, dL/dmu0 of the
// initial state and dL/dtheta for theta = (delta_ab for pairs a < b in
// row-major order, the phase mobility 1/tau, the entries D^a_ij), accumulated
// over the steps.  The forward states are kept; each step is taped from its
// own input (recorded leaves) and swept back on its own.
int oracle_run_adjoint(const oracle_problem* p, const double* phi0, const double* mu0, int nsteps,
                       const double* lam_phi, const double* lam_mu, double* dphi0, double* dmu0, double* dtheta) {
  if (check(p)) return 1;
  Ctx<double> c;
  init_ctx(c, p);
  const int64_t cells = c.cells;
  const int N = p->N, NM = p->NM;
  const int64_t nphi = N * cells, nmu = NM * cells;
  std::vector<double> st((int64_t)(nsteps + 1) * (nphi + nmu));
  std::memcpy(st.data(), phi0, sizeof(double) * nphi);
  std::memcpy(st.data() + nphi, mu0, sizeof(double) * nmu);
  for (int n = 0; n < nsteps; ++n) {
    double* a = st.data() + (int64_t)n * (nphi + nmu);
    double* b = a + (nphi + nmu);
    step(c, a, a + nphi, b, b + nphi, p->t0 + n * p->dt, p->step0 + n);
  }
  const int P = N * (N - 1) / 2;
  const int NPRM = P + 1 + N * NM * NM;
  for (int k = 0; k < NPRM; ++k) dtheta[k] = 0.0;
  std::vector<double> lp(lam_phi, lam_phi + nphi), lm(lam_mu, lam_mu + nmu);
  for (int n = nsteps - 1; n >= 0; --n) {
    g_tape.clear();
    Ctx<Rev> r;
    init_ctx(r, p);
    // the differentiable parameters as recorded leaves
    int pid[NMAX * NMAX], mid, did[NMAX * KMAX * KMAX];
    for (int a = 0, k = 0; a < N; ++a)
      for (int b = a + 1; b < N; ++b, ++k) {
        r.q.delta[a][b] = rev_leaf(p->delta[a * N + b]);
        r.q.delta[b][a] = r.q.delta[a][b];
        pid[k] = r.q.delta[a][b].id;
      }
    r.q.mob = rev_leaf(1.0 / p->tau);
    mid = r.q.mob.id;
    for (int a = 0; a < N; ++a)
      for (int i = 0; i < NM; ++i)
        for (int j = 0; j < NM; ++j) {
          r.q.D[a][i][j] = rev_leaf(p->D[(a * NM + i) * NM + j]);
          did[(a * NM + i) * NM + j] = r.q.D[a][i][j].id;
        }
    const double* in = st.data() + (int64_t)n * (nphi + nmu);
    std::vector<Rev> pa(nphi), ma(nmu), pb(nphi), mb(nmu);
    for (int64_t i = 0; i < nphi; ++i) pa[i] = rev_leaf(in[i]);
    for (int64_t i = 0; i < nmu; ++i) ma[i] = rev_leaf(in[nphi + i]);
    step(r, pa.data(), ma.data(), pb.data(), mb.data(), p->t0 + n * p->dt, p->step0 + n);
    std::vector<double> adj(g_tape.size(), 0.0);
    for (int64_t i = 0; i < nphi; ++i)
      if (pb[i].id >= 0) adj[pb[i].id] += lp[i];
    for (int64_t i = 0; i < nmu; ++i)
      if (mb[i].id >= 0) adj[mb[i].id] += lm[i];
    for (int64_t k = (int64_t)g_tape.size() - 1; k >= 0; --k) {
      const TapeNode& t = g_tape[k];
      if (adj[k] == 0.0) continue;
      if (t.a >= 0) adj[t.a] += t.da * adj[k];
      if (t.b >= 0) adj[t.b] += t.db * adj[k];
    }
    for (int64_t i = 0; i < nphi; ++i) lp[i] = adj[pa[i].id];
    for (int64_t i = 0; i < nmu; ++i) lm[i] = adj[ma[i].id];
    for (int k = 0; k < P; ++k) dtheta[k] += adj[pid[k]];
    dtheta[P] += adj[mid];
    for (int k = 0; k < N * NM * NM; ++k) dtheta[P + 1 + k] += adj[did[k]];
  }
  g_tape.clear();
  g_tape.shrink_to_fit();
  std::memcpy(dphi0, lp.data(), sizeof(double) * nphi);
  std::memcpy(dmu0, lm.data(), sizeof(double) * nmu);
  return 0;
}

// Rate parts at every cell: divJ, centre term, dw/dphi, dpsi/dphi ([N][cells] each).
int oracle_rate_parts(const oracle_problem* p, const double* phi, const double* mu,
                      double* divJ, double* Gc, double* W, double* P) {
  if (check(p)) return 1;
  Ctx<double> c;
  init_ctx(c, p);
  for (int z = 0; z < c.n[2]; ++z)
    for (int y = 0; y < c.n[1]; ++y)
      for (int x = 0; x < c.n[0]; ++x) {
        const int64_t ic = cell_index(c, x, y, z);
        double a1[NMAX], a2[NMAX], a3[NMAX], a4[NMAX];
        rate_parts(c, phi, mu, x, y, z, p->t0, a1, a2, a3, a4);
        for (int a = 0; a < p->N; ++a) {
          divJ[a * c.cells + ic] = a1[a];
          Gc[a * c.cells + ic] = a2[a];
          W[a * c.cells + ic] = a3[a];
          P[a * c.cells + ic] = a4[a];
        }
      }
  return 0;
}

// FP64 diagnostics: out[0..NM) = sum over cells of c_i = sum_a h_a c^a_i(mu,T);
// out[NM] = max |sum phi - 1|; out[NM+1] = min phi; out[NM+2] = max phi.
int oracle_diag(const oracle_problem* p, const double* phi, const double* mu, double* out) {
  if (check(p)) return 1;
  Ctx<double> c;
  init_ctx(c, p);
  for (int i = 0; i < p->NM + 3; ++i) out[i] = 0.0;
  out[p->NM + 1] = 1e300;
  out[p->NM + 2] = -1e300;
  for (int z = 0; z < c.n[2]; ++z)
    for (int y = 0; y < c.n[1]; ++y)
      for (int x = 0; x < c.n[0]; ++x) {
        const int64_t ic = cell_index(c, x, y, z);
        double ph[NMAX], h[NMAX], m[KMAX], s = 0.0;
        for (int a = 0; a < p->N; ++a) {
          ph[a] = phi[a * c.cells + ic];
          s += ph[a];
          out[p->NM + 1] = std::min(out[p->NM + 1], ph[a]);
          out[p->NM + 2] = std::max(out[p->NM + 2], ph[a]);
        }
        out[p->NM] = std::max(out[p->NM], std::fabs(s - 1.0));
        interp_h(p->N, ph, h);
        for (int i = 0; i < p->NM; ++i) m[i] = mu[i * c.cells + ic];
        const double T = temperature(*p, y, z, p->t0);
        for (int a = 0; a < p->N; ++a) {
          double ca[KMAX];
          comp_of_mu(*p, a, m, T, ca);
          for (int i = 0; i < p->NM; ++i) out[i] += h[a] * ca[i];
        }
      }
  return 0;
}

// ---- single-formula probes used by the pin tests
// The anti-trapping current's normal component at the +d face of cell
// (x, y, z): J[NM] (see at_face_flux); phi, phin [N][cells], mu [NM][cells].
int oracle_at_face_flux(const oracle_problem* p, const double* phi, const double* phin, const double* mu, int x,
                        int y, int z, int d, double t, double* J) {
  if (check(p)) return 1;
  Ctx<double> c;
  init_ctx(c, p);
  at_face_flux(c, phi, phin, mu, x, y, z, d, t, J);
  return 0;
}

// The phi-noise variate for (seed, step, counter) (see noise_variate).
double oracle_noise(unsigned long long seed, long long step, unsigned long long counter) {
  return noise_variate(seed, (uint64_t)step, counter);
}

double oracle_pair_energy(const oracle_problem* p, int a, int b, const double* q) {
  Ctx<double> c;
  init_ctx(c, p);
  return pair_energy(c, a, b, q);
}

void oracle_pair_energy_grad(const oracle_problem* p, int a, int b, const double* q, double* g) {
  Ctx<double> c;
  init_ctx(c, p);
  pair_energy_grad(c, a, b, q, g);
}

double oracle_potential(const oracle_problem* p, const double* phi, double* dw) {
  potential_dw(*p, phi, dw);
  return potential_w(*p, phi);
}

void oracle_interp(int N, const double* phi, double* h, double* dh) {
  interp_h(N, phi, h);
  interp_dh(N, phi, dh);
}

void oracle_project(int N, int potential, const double* v, double* out) {
  if (potential == 1)
    project_simplex(N, v, out);
  else
    project_hyperplane(N, v, out);
}

// c^a(mu,T), psi^a(mu,T), chi^a for one phase.
void oracle_thermo(const oracle_problem* p, int a, const double* mu, double T, double* c,
                   double* psi, double* chi) {
  comp_of_mu(*p, a, mu, T, c);
  *psi = grand_potential(*p, a, mu, T);
  chi_phase(*p, a, chi);
}

}  // extern "C"
