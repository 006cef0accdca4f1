// Sparse grain growth: many grains (up to 64), each cell storing only the
// grains non-zero there (MICROSIM paper, arXiv 2404.01035, Sec. 4
// "Grain-growth": the phi equation of Sec. 2.1 without the chemical driving
// force; isotropic boundary energies, multi-obstacle potential with the
// triple term Gamma_abc).
//
// Reading (locally active phases): the Lagrange multiplier acts on the grains
// present at the cell or at one of its face neighbours -- the projection onto
// the simplex runs over them alone and every other grain stays 0 -- so a grain
// can only appear next to where it already is, and a cell holds few grains.
// With isotropic pairs (g = 2 gamma q) the update of a cell reads only its
// 7-point stencil (face fluxes need the normal differences alone).
//
// State per buffer: for every cell the number of stored grains, up to kSlots
// (grain index, value) pairs sorted by grain index (slot-major arrays), and a
// code byte (grain + 1 when the cell is that grain alone with value 1, else 0).
// One step = two launches:
//   k_ggs_classify: one thread per cell; a cell whose 7 codes name one grain
//     keeps it (written only when the destination buffer, which holds the
//     state one step back, does not already hold it); the others are appended
//     to a work list (warp-aggregated).
//   k_ggs_update: grid-stride over the list (a build for unions of up to 4
//     grains, which defers larger ones to a second list and build); the grains of the 7 stencil cells
//     (a 64-bit union mask), their values gathered into per-thread shared
//     memory, the face fluxes, centre term, potential derivative and rate over
//     that union in increasing grain order (the order of the dense sums, whose
//     other terms are exact zeros), the projection over the union, and the
//     non-zero results stored.
// A cell that would need more than kSlots grains (or a stencil union above
// kUnion) sets the sticky status MS_ERR_BOUNDS instead of losing a grain.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/microsim_gb.h"
#include "ms_device.cuh"
#include "ms_rt.h"
#include "ms_trace.h"

namespace msgb {
ms_status build_model(ms_ctx* c, const ms_grid* g, int N, int K, const ms_params* p, HostModel& m);
}

using namespace msgb;

namespace {

constexpr int kSlots = 8;        // grains stored per cell
constexpr int kUnion = 8;        // grains in a 7-point stencil at most
constexpr int kUnionSmall = 4;   // the union size of the first update build
constexpr int kMaxGrains = 64;   // union masks are 64-bit
constexpr int kStatusOverflow = 8;

template <class Real>
struct GgsArgs {
  int nx, ny, nz, dim, N;
  int bc[3];
  long long cells;
  Real dt, eps, inv_eps, mob, inv_dx, half_inv_dx, g3;
  int has_g3;
  const Real* gam2;   // [N][N] 2 gamma_ab
  const Real* cw;     // [N][N] 16 gamma_ab / pi^2
  // input / output state
  const uint8_t* cnt_in;
  const uint8_t* code_in;
  const uint8_t* idx_in;   // [kSlots][cells]
  const Real* val_in;      // [kSlots][cells]
  uint8_t* cnt_out;
  uint8_t* code_out;
  uint8_t* idx_out;
  Real* val_out;
  unsigned int* list;      // [0] count, [1..] cell indices
  unsigned int* list2;     // the cells whose stencil holds more than kUnionSmall grains
  unsigned int list_cap;
  int* status;
};

__device__ __forceinline__ int wrap_axis(int i, int n, int bc) {
  if (i >= 0 && i < n) return i;
  if (bc == 3) return i < 0 ? i + n : i - n;
  return i < 0 ? 0 : n - 1;   // no-flux: mirror ghost = adjacent interior cell
}

// Linear index of the cell at (x, y, z) + unit step s along axis d (boundary mapped).
template <class Real>
__device__ __forceinline__ long long nb_index(const GgsArgs<Real>& g, int x, int y, int z, int d, int s) {
  if (d == 0) x = wrap_axis(x + s, g.nx, g.bc[0]);
  if (d == 1) y = wrap_axis(y + s, g.ny, g.bc[1]);
  if (d == 2) z = wrap_axis(z + s, g.nz, g.bc[2]);
  return ((long long)z * g.ny + y) * g.nx + x;
}

template <class Real>
__global__ void __launch_bounds__(256) k_ggs_classify(const GgsArgs<Real> g) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  bool listed = false;
  if (i < g.cells) {
    const int x = (int)(i % g.nx), y = (int)((i / g.nx) % g.ny), z = (int)(i / ((long long)g.nx * g.ny));
    const uint8_t c0 = g.code_in[i];
    bool bulk = c0 != 0;
    for (int d = 0; d < g.dim && bulk; ++d)
      for (int s = -1; s <= 1 && bulk; s += 2) bulk = g.code_in[nb_index(g, x, y, z, d, s)] == c0;
    if (bulk) {
      // the destination holds the state one step back: rewrite only when it differs
      if (g.code_out[i] != c0 || g.cnt_out[i] != 1) {
        g.cnt_out[i] = 1;
        g.idx_out[i] = (uint8_t)(c0 - 1);
        g.val_out[i] = Real(1);
      }
      g.code_out[i] = c0;
    } else {
      listed = true;
    }
  }
  const unsigned int need = __ballot_sync(0xffffffffu, listed);
  if (need) {
    const int first = __ffs(need) - 1;
    unsigned int base = 0;
    if (lane == first) base = atomicAdd(&g.list[0], (unsigned int)__popc(need));
    base = __shfl_sync(0xffffffffu, base, first);
    if (listed) {
      const unsigned int k = base + __popc(need & ((1u << lane) - 1u));
      if (k < g.list_cap) g.list[1 + k] = (unsigned int)i;
    }
  }
}

// Simplex projection (Held-Wolfe-Crowder 1974; Duchi et al. 2008) of the
// first n <= kUnion values: the threshold theta (phi = max(v - theta, 0)).
template <class Real, int K>
__device__ __forceinline__ Real simplex_theta(const Real* v, int n) {
  Real u[K];
#pragma unroll
  for (int a = 0; a < K; ++a) u[a] = a < n ? v[a] : Real(-INFINITY);
  // insertion sort, descending (a fixed network over K entries)
#pragma unroll
  for (int i = 1; i < K; ++i)
#pragma unroll
    for (int j = i; j > 0; --j)
      if (u[j] > u[j - 1]) {
        const Real t = u[j];
        u[j] = u[j - 1];
        u[j - 1] = t;
      }
  Real csum = Real(0), theta = Real(0);
#pragma unroll
  for (int j = 0; j < K; ++j) {
    if (j >= n) break;
    csum += u[j];
    const Real t = (csum - Real(1)) / Real(j + 1);
    if (u[j] - t > Real(0)) theta = t;
  }
  return theta;
}

// Threads per block of the update kernel: its shared memory holds 7 x KU
// values per thread.
template <class Real, int KU>
struct UpdShape {
  static constexpr int THREADS = sizeof(Real) * KU > 16 ? 64 : 128;
  static constexpr int MIN_BLOCKS = sizeof(Real) * KU > 16 ? 4 : 4;   // registers for 16 warps per SM (8 for the large builds)
};

// Two builds: KU = kUnionSmall takes the cells of the first list whose
// stencil holds at most that many grains (nearly all) and moves the others to
// the second list, which the KU = kUnion build then updates (each build's
// registers fit its own union size).
template <class Real, int KU>
__global__ void __launch_bounds__(UpdShape<Real, KU>::THREADS, UpdShape<Real, KU>::MIN_BLOCKS)
    k_ggs_update(const GgsArgs<Real> g) {
  constexpr int T = UpdShape<Real, KU>::THREADS;
  constexpr bool kFirst = KU < kUnion;
  const unsigned int* list = kFirst ? g.list : g.list2;
  // per thread: the union's values at the 7 stencil cells ([cell][grain]) and
  // the union's grain ids (increasing)
  __shared__ Real s_val[T][7][KU];
  __shared__ uint8_t s_uid[T][KU];
  Real (*sv)[KU] = s_val[threadIdx.x];
  uint8_t* uid = s_uid[threadIdx.x];
  const unsigned int count = min(*(volatile const unsigned int*)&list[0], g.list_cap);
  const int nst = 2 * g.dim + 1;   // stencil cells: 0 the centre, 1 + 2d the -d and 2 + 2d the +d neighbour
  for (unsigned int w = blockIdx.x * blockDim.x + threadIdx.x; w < count; w += gridDim.x * blockDim.x) {
    const long long i = list[1 + w];
    const int x = (int)(i % g.nx), y = (int)((i / g.nx) % g.ny), z = (int)(i / ((long long)g.nx * g.ny));
    long long ci[7];
    ci[0] = i;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (d >= g.dim) break;
      ci[1 + 2 * d] = nb_index(g, x, y, z, d, -1);
      ci[2 + 2 * d] = nb_index(g, x, y, z, d, 1);
    }
    // union of the grains present on the stencil (every load independent:
    // the counts first, then all slots, predicated)
    int cntc[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) cntc[c] = c < nst ? (int)g.cnt_in[ci[c]] : 0;
    unsigned long long mask = 0ull;
#pragma unroll
    for (int c = 0; c < 7; ++c)
#pragma unroll
      for (int k = 0; k < kSlots; ++k)
        if (k < cntc[c]) mask |= 1ull << g.idx_in[k * g.cells + ci[c]];
    const int nu = __popcll(mask);
    if (nu > KU) {
      if constexpr (kFirst) {
        const unsigned int k2 = atomicAdd(&g.list2[0], 1u);
        if (k2 < g.list_cap) g.list2[1 + k2] = (unsigned int)i;
      } else {
        atomicOr(g.status, kStatusOverflow);
      }
      continue;
    }
    {
      unsigned long long m = mask;
#pragma unroll
      for (int u = 0; u < KU; ++u) {
        uid[u] = m ? (uint8_t)(__ffsll((long long)m) - 1) : (uint8_t)0;
        m &= m - 1ull;
      }
    }
#pragma unroll
    for (int c = 0; c < 7; ++c)
#pragma unroll
      for (int u = 0; u < KU; ++u) sv[c][u] = Real(0);
#pragma unroll
    for (int c = 0; c < 7; ++c)
#pragma unroll
      for (int k = 0; k < kSlots; ++k)
        if (k < cntc[c]) {
          const int a = g.idx_in[k * g.cells + ci[c]];
          sv[c][__popcll(mask & ((1ull << a) - 1ull))] = g.val_in[k * g.cells + ci[c]];
        }
    // S1-S3: divergence of the face fluxes (isotropic: the normal component
    // of g = 2 gamma q needs the normal differences only), in the order of
    // the dense sums restricted to the present grains
    Real divJ[KU], Gc[KU];
#pragma unroll
    for (int u = 0; u < KU; ++u) {
      divJ[u] = Real(0);
      Gc[u] = Real(0);
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (d >= g.dim) break;
      Real Jm[KU], Jp[KU];
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        // side 0: the face with the -d neighbour (left = it, right = the
        // cell); side 1: with the +d neighbour (left = the cell)
        const int cl = side ? 0 : 1 + 2 * d, cr = side ? 2 + 2 * d : 0;
        Real* J = side ? Jp : Jm;
        Real pf[KU], gr[KU];
#pragma unroll
        for (int a = 0; a < KU; ++a) {
          J[a] = Real(0);
          if (a >= nu) continue;
          const Real vl = sv[cl][a], vr = sv[cr][a];
          pf[a] = Real(0.5) * (vl + vr);
          gr[a] = (vr - vl) * g.inv_dx;
        }
#pragma unroll
        for (int a = 0; a < KU; ++a) {
          if (a >= nu) break;
#pragma unroll
          for (int b = a + 1; b < KU; ++b) {
            if (b >= nu) break;
            const Real q = pf[a] * gr[b] - pf[b] * gr[a];
            const Real gq = g.gam2[uid[a] * g.N + uid[b]] * q;
            J[a] -= pf[b] * gq;
            J[b] += pf[a] * gq;
          }
        }
      }
#pragma unroll
      for (int a = 0; a < KU; ++a)
        if (a < nu) divJ[a] += (Jp[a] - Jm[a]) * g.inv_dx;
    }
    // centre term, central differences
    Real gc[KU][3];
#pragma unroll
    for (int a = 0; a < KU; ++a)
#pragma unroll
      for (int d = 0; d < 3; ++d) gc[a][d] = d < g.dim ? (sv[2 + 2 * d][a] - sv[1 + 2 * d][a]) * g.half_inv_dx : Real(0);
#pragma unroll
    for (int a = 0; a < KU; ++a) {
      if (a >= nu) break;
#pragma unroll
      for (int b = a + 1; b < KU; ++b) {
        if (b >= nu) break;
        const Real gm = g.gam2[uid[a] * g.N + uid[b]];
        Real gq[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) gq[d] = gm * (sv[0][a] * gc[b][d] - sv[0][b] * gc[a][d]);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          if (d >= g.dim) break;
          Gc[a] += gq[d] * gc[b][d];
          Gc[b] -= gq[d] * gc[a][d];
        }
      }
    }
    // S4 potential derivative (obstacle, with the triple term), S5 rate and
    // explicit Euler (no chemical driving force in grain growth)
    Real v[KU];
#pragma unroll
    for (int a = 0; a < KU; ++a) {
      v[a] = Real(0);
      if (a >= nu) continue;
      Real W = Real(0);
#pragma unroll
      for (int b = 0; b < KU; ++b)
        if (b < nu && b != a) W += g.cw[uid[a] * g.N + uid[b]] * sv[0][b];
      if (g.has_g3) {
#pragma unroll
        for (int b = 0; b < KU; ++b)
#pragma unroll
          for (int e = b + 1; e < KU; ++e)
            if (e < nu && b != a && e != a) W += g.g3 * sv[0][b] * sv[0][e];
      }
      const Real r = g.mob * (g.eps * (divJ[a] - Gc[a]) - W * g.inv_eps) * g.inv_eps;
      v[a] = sv[0][a] + g.dt * r;
    }
    // projection over the locally active grains (the union)
    const Real theta = simplex_theta<Real, KU>(v, nu);
    int n_out = 0;
    uint8_t code = 0;
#pragma unroll
    for (int a = 0; a < KU; ++a) {
      if (a >= nu) break;
      const Real dd = v[a] - theta;
      const Real pn = dd > Real(0) ? dd : Real(0);
      if (pn > Real(0)) {
        if (n_out < kSlots) {
          g.idx_out[n_out * g.cells + i] = uid[a];
          g.val_out[n_out * g.cells + i] = pn;
          if (pn == Real(1)) code = (uint8_t)(uid[a] + 1);
        }
        ++n_out;
      }
    }
    if (n_out > kSlots) {
      atomicOr(g.status, kStatusOverflow);
      n_out = kSlots;
    }
    g.cnt_out[i] = (uint8_t)n_out;
    g.code_out[i] = n_out == 1 ? code : 0;
  }
}

// dense [N][cells] -> slots (sorted by grain), codes; overflow -> status
template <class Real>
__global__ void k_ggs_pack(const Real* __restrict__ dense, int N, long long cells, uint8_t* cnt, uint8_t* code,
                           uint8_t* idx, Real* val, int* status) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= cells) return;
  int n = 0;
  uint8_t c = 0;
  for (int a = 0; a < N; ++a) {
    const Real v = dense[a * cells + i];
    if (v > Real(0)) {
      if (n < kSlots) {
        idx[n * cells + i] = (uint8_t)a;
        val[n * cells + i] = v;
        if (v == Real(1)) c = (uint8_t)(a + 1);
      }
      ++n;
    } else if (!(v == Real(0))) {
      atomicOr(status, kStatusOverflow);   // negative or non-finite input
    }
  }
  if (n > kSlots) {
    atomicOr(status, kStatusOverflow);
    n = kSlots;
  }
  cnt[i] = (uint8_t)n;
  code[i] = n == 1 ? c : 0;
}

template <class Real>
__global__ void k_ggs_unpack(Real* __restrict__ dense, long long cells, const uint8_t* cnt, const uint8_t* idx,
                             const Real* val) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= cells) return;
  const int n = cnt[i];
  for (int k = 0; k < n; ++k) dense[idx[k * cells + i] * cells + i] = val[k * cells + i];
}

}  // namespace

struct ms_ggs {
  HostModel m;
  int N = 0;
  long long cells = 0;
  size_t s = 4;
  void* buf[2] = {nullptr, nullptr};   // cnt | code | idx | val per buffer
  void* tables = nullptr;              // gam2 [N][N], cw [N][N]
  unsigned int* list = nullptr;
  unsigned int* list2 = nullptr;
  int* status = nullptr;
  int cur = 0;
  int64_t step = 0;
  int upd_blocks = 0;
  double g3 = 0.0;
  int has_g3 = 0;
  cudaStream_t stream = nullptr;
  AllocHook hook;
  std::string err;
};

namespace {

ms_status gfail(ms_ggs* s, ms_status st, const std::string& m) {
  if (s) s->err = m;
  return fail(nullptr, st, m);
}

size_t buf_bytes(const ms_ggs* s) {
  const size_t c = (size_t)s->cells;
  const size_t head = (2 * c + (size_t)kSlots * c + 255) / 256 * 256;
  return head + (size_t)kSlots * c * s->s;
}
uint8_t* cnt_of(const ms_ggs* s, int b) { return static_cast<uint8_t*>(s->buf[b]); }
uint8_t* code_of(const ms_ggs* s, int b) { return cnt_of(s, b) + s->cells; }
uint8_t* idx_of(const ms_ggs* s, int b) { return cnt_of(s, b) + 2 * s->cells; }
void* val_of(const ms_ggs* s, int b) {
  const size_t c = (size_t)s->cells;
  return cnt_of(s, b) + (2 * c + (size_t)kSlots * c + 255) / 256 * 256;
}

template <class Real>
GgsArgs<Real> make_args(const ms_ggs* s, int src) {
  GgsArgs<Real> g;
  std::memset(&g, 0, sizeof(g));
  const HostModel& m = s->m;
  g.nx = m.nx;
  g.ny = m.ny;
  g.nz = m.dim == 3 ? m.nz : 1;
  g.dim = m.dim;
  g.N = s->N;
  for (int d = 0; d < 3; ++d) g.bc[d] = m.bc[d];
  g.cells = s->cells;
  g.dt = (Real)m.dt;
  g.eps = (Real)m.eps;
  g.inv_eps = (Real)(1.0 / m.eps);
  g.mob = (Real)(1.0 / m.tau);
  g.inv_dx = (Real)(1.0 / m.dx);
  g.half_inv_dx = (Real)(0.5 / m.dx);
  g.g3 = (Real)s->g3;
  g.has_g3 = s->has_g3;
  g.gam2 = static_cast<const Real*>(s->tables);
  g.cw = static_cast<const Real*>(s->tables) + s->N * s->N;
  g.cnt_in = cnt_of(s, src);
  g.code_in = code_of(s, src);
  g.idx_in = idx_of(s, src);
  g.val_in = static_cast<const Real*>(val_of(s, src));
  g.cnt_out = cnt_of(s, 1 - src);
  g.code_out = code_of(s, 1 - src);
  g.idx_out = idx_of(s, 1 - src);
  g.val_out = static_cast<Real*>(val_of(s, 1 - src));
  g.list = s->list;
  g.list2 = s->list2;
  g.list_cap = (unsigned int)s->cells;
  g.status = s->status;
  return g;
}

template <class Real>
cudaError_t step_once(ms_ggs* s) {
  const GgsArgs<Real> g = make_args<Real>(s, s->cur);
  cudaError_t e = cudaMemsetAsync(s->list, 0, sizeof(unsigned int), s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->list2, 0, sizeof(unsigned int), s->stream);
  if (e != cudaSuccess) return e;
  k_ggs_classify<Real><<<(unsigned int)((s->cells + 255) / 256), 256, 0, s->stream>>>(g);
  k_ggs_update<Real, kUnionSmall><<<s->upd_blocks, UpdShape<Real, kUnionSmall>::THREADS, 0, s->stream>>>(g);
  k_ggs_update<Real, kUnion><<<s->upd_blocks, UpdShape<Real, kUnion>::THREADS, 0, s->stream>>>(g);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

ms_status ms_ggs_create(const ms_grid* grid, int n_grains, const ms_params* p, void* stream,
                        const ms_allocator* alloc, ms_ggs** out) {
  if (!out || !grid || !p) return gfail(nullptr, MS_ERR_ARG, "grid, params and out are required");
  *out = nullptr;
  if (n_grains < 2 || n_grains > kMaxGrains)
    return gfail(nullptr, MS_ERR_ARG, "sparse grain growth takes 2 to 64 grains");
  if (p->potential != MS_POT_OBSTACLE)
    return gfail(nullptr, MS_ERR_UNSUPPORTED, "sparse grain growth needs the obstacle potential");
  if (p->noise_amp != 0.0 || p->anti_trapping || p->elastic_C)
    return gfail(nullptr, MS_ERR_UNSUPPORTED, "sparse grain growth takes no noise, anti-trapping or elasticity");
  const int N = n_grains;
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b)
      if (a != b && p->delta && p->delta[a * N + b] != 0.0)
        return gfail(nullptr, MS_ERR_UNSUPPORTED, "sparse grain growth is isotropic (delta = 0 for every pair)");
  double g3 = 0.0;
  int has_g3 = 0;
  if (p->gamma3) {
    // a uniform triple term over distinct triples (the only form stored)
    bool first = true;
    for (int a = 0; a < N; ++a)
      for (int b = 0; b < N; ++b)
        for (int c = 0; c < N; ++c) {
          const double v = p->gamma3[(a * N + b) * N + c];
          if (a == b || b == c || a == c) {
            if (v != 0.0) return gfail(nullptr, MS_ERR_ARG, "gamma3 must vanish unless the three phases differ");
            continue;
          }
          if (first) {
            g3 = v;
            first = false;
          } else if (v != g3) {
            return gfail(nullptr, MS_ERR_UNSUPPORTED, "sparse grain growth takes a uniform gamma3");
          }
        }
    has_g3 = g3 != 0.0;
  }
  if (grid->dim == 3 && grid->bc[2] == MS_BC_HALO)
    return gfail(nullptr, MS_ERR_UNSUPPORTED, "sparse grain growth runs on the whole domain");
  ensure_registered();
  ms_ggs* s = new ms_ggs();
  // the model checks of a context (grid, boundaries, dt bound, gamma): one
  // solute field stands in for the held mu, with the values build_model needs
  ms_params q = *p;
  std::vector<double> D(N, 0.0), A(N, 1.0), ceq(N, 0.5), sl(N, 0.0);
  q.D = D.data();
  q.A = A.data();
  q.ceq = ceq.data();
  q.slopes = sl.data();
  q.f0 = nullptr;
  q.gamma3 = nullptr;
  q.grain_growth = 1;
  q.rot = nullptr;
  q.delta = nullptr;
  std::vector<double> zero(N * N, 0.0);
  q.delta = zero.data();
  if (N > kNMax) {
    // build_model checks at most kNMax phases: check the shape here
    if (grid->dim != 2 && grid->dim != 3) {
      delete s;
      return gfail(nullptr, MS_ERR_ARG, "dim must be 2 or 3");
    }
    if (grid->nx < 1 || grid->ny < 1 || (grid->dim == 3 && grid->nz < 1) || !(grid->dx > 0.0)) {
      delete s;
      return gfail(nullptr, MS_ERR_ARG, "bad grid");
    }
    for (int d = 0; d < grid->dim; ++d)
      if (grid->bc[d] != MS_BC_PERIODIC && grid->bc[d] != MS_BC_NOFLUX) {
        delete s;
        return gfail(nullptr, MS_ERR_ARG, "boundaries must be periodic or no-flux");
      }
    if (!(p->eps > 0.0) || !(p->tau > 0.0) || !(p->dt > 0.0) || !p->gamma) {
      delete s;
      return gfail(nullptr, MS_ERR_ARG, "eps, tau, dt and gamma are required");
    }
    s->m.dim = grid->dim;
    s->m.nx = grid->nx;
    s->m.ny = grid->ny;
    s->m.nz = grid->dim == 3 ? grid->nz : 1;
    s->m.dx = grid->dx;
    for (int d = 0; d < 3; ++d) s->m.bc[d] = d < grid->dim ? grid->bc[d] : 3;
    s->m.dtype = p->dtype;
    s->m.eps = p->eps;
    s->m.tau = p->tau;
    s->m.dt = p->dt;
  } else {
    ms_status st = build_model(nullptr, grid, N, 2, &q, s->m);
    if (st != MS_OK) {
      std::string msg = ms_last_error(nullptr);
      delete s;
      return gfail(nullptr, st, msg);
    }
  }
  // explicit stability of the phase equation (isotropic): dt <= (dx^2 / 2d) tau / gamma_max
  double gmax = 0.0;
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b)
      if (a != b) {
        const double v = p->gamma[a * N + b];
        if (!(v >= 0.0) || v != p->gamma[b * N + a]) {
          delete s;
          return gfail(nullptr, MS_ERR_ARG, "gamma must be symmetric and non-negative");
        }
        gmax = std::max(gmax, v);
      }
  const double bound = grid->dx * grid->dx / (2.0 * grid->dim) * p->tau / (gmax > 0 ? gmax : 1.0);
  if (p->dt > bound) {
    delete s;
    return gfail(nullptr, MS_ERR_DT_UNSTABLE, "dt above the explicit stability bound");
  }
  s->N = N;
  s->g3 = g3;
  s->has_g3 = has_g3;
  s->cells = (long long)grid->nx * grid->ny * (grid->dim == 3 ? grid->nz : 1);
  if (s->cells >= 0xFFFFFFFFll) {
    delete s;
    return gfail(nullptr, MS_ERR_BOUNDS, "grid too large for the work list");
  }
  s->s = p->dtype == MS_F64 ? 8 : 4;
  s->stream = static_cast<cudaStream_t>(stream);
  if (alloc) s->hook = AllocHook{alloc->alloc, alloc->release, alloc->user};
  for (int b = 0; b < 2; ++b) s->buf[b] = dev_alloc(s->hook, buf_bytes(s));
  s->tables = dev_alloc(s->hook, 2 * (size_t)N * N * s->s);
  s->list = static_cast<unsigned int*>(dev_alloc(s->hook, 2 * (size_t)(s->cells + 1) * sizeof(unsigned int) + 256));
  if (!s->buf[0] || !s->buf[1] || !s->tables || !s->list) {
    ms_ggs_destroy(s);
    return gfail(nullptr, MS_ERR_OOM, "sparse grain-growth allocation failed");
  }
  s->list2 = s->list + (s->cells + 1);
  s->status = reinterpret_cast<int*>(s->list2 + (s->cells + 1));
  const double PI = 3.14159265358979323846;
  std::vector<double> tab(2 * (size_t)N * N);
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) {
      tab[a * N + b] = 2.0 * p->gamma[a * N + b];
      tab[N * N + a * N + b] = (16.0 / (PI * PI)) * p->gamma[a * N + b];   // as the obstacle term forms it
    }
  cudaError_t e = cudaSuccess;
  if (s->s == 8) {
    e = cudaMemcpyAsync(s->tables, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, s->stream);
  } else {
    std::vector<float> tf(tab.begin(), tab.end());
    e = cudaMemcpyAsync(s->tables, tf.data(), tf.size() * 4, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  }
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMemsetAsync(s->buf[b], 0, buf_bytes(s), s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->status, 0, sizeof(int), s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  s->upd_blocks = 8 * sms;
  if (e != cudaSuccess) {
    std::string m = std::string("sparse grain growth set-up: ") + cudaGetErrorString(e);
    ms_ggs_destroy(s);
    return gfail(nullptr, MS_ERR_CUDA, m);
  }
  *out = s;
  return MS_OK;
}

void ms_ggs_destroy(ms_ggs* s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  for (int b = 0; b < 2; ++b) dev_free(s->hook, s->buf[b]);
  dev_free(s->hook, s->tables);
  dev_free(s->hook, s->list);
  delete s;
}

const char* ms_ggs_last_error(const ms_ggs* s) { return s ? s->err.c_str() : ms_last_error(nullptr); }

ms_status ms_ggs_set_fields(ms_ggs* s, const void* phi, int on_device) {
  if (!s || !phi) return gfail(s, MS_ERR_ARG, "ctx and phi are required");
  const size_t bytes = (size_t)s->N * s->cells * s->s;
  void* dense = const_cast<void*>(phi);
  void* tmp = nullptr;
  cudaError_t e = cudaSuccess;
  if (!on_device) {
    tmp = dev_alloc(s->hook, bytes);
    if (!tmp) return gfail(s, MS_ERR_OOM, "staging allocation failed");
    e = cudaMemcpyAsync(tmp, phi, bytes, cudaMemcpyHostToDevice, s->stream);
    dense = tmp;
  }
  const unsigned int blocks = (unsigned int)((s->cells + 255) / 256);
  if (e == cudaSuccess) {
    if (s->s == 8)
      k_ggs_pack<double><<<blocks, 256, 0, s->stream>>>(static_cast<const double*>(dense), s->N, s->cells,
                                                         cnt_of(s, s->cur), code_of(s, s->cur), idx_of(s, s->cur),
                                                         static_cast<double*>(val_of(s, s->cur)), s->status);
    else
      k_ggs_pack<float><<<blocks, 256, 0, s->stream>>>(static_cast<const float*>(dense), s->N, s->cells,
                                                        cnt_of(s, s->cur), code_of(s, s->cur), idx_of(s, s->cur),
                                                        static_cast<float*>(val_of(s, s->cur)), s->status);
    e = cudaGetLastError();
  }
  // the other buffer holds nothing of this state
  if (e == cudaSuccess) e = cudaMemsetAsync(s->buf[1 - s->cur], 0, 2 * (size_t)s->cells, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  dev_free(s->hook, tmp);
  if (e != cudaSuccess) return gfail(s, MS_ERR_CUDA, std::string("sparse set fields: ") + cudaGetErrorString(e));
  s->step = 0;
  return ms_ggs_sync(s);
}

ms_status ms_ggs_get_fields(ms_ggs* s, void* phi, int on_device) {
  if (!s || !phi) return gfail(s, MS_ERR_ARG, "ctx and phi are required");
  const size_t bytes = (size_t)s->N * s->cells * s->s;
  void* dense = phi;
  void* tmp = nullptr;
  if (!on_device) {
    tmp = dev_alloc(s->hook, bytes);
    if (!tmp) return gfail(s, MS_ERR_OOM, "staging allocation failed");
    dense = tmp;
  }
  cudaError_t e = cudaMemsetAsync(dense, 0, bytes, s->stream);
  const unsigned int blocks = (unsigned int)((s->cells + 255) / 256);
  if (e == cudaSuccess) {
    if (s->s == 8)
      k_ggs_unpack<double><<<blocks, 256, 0, s->stream>>>(static_cast<double*>(dense), s->cells, cnt_of(s, s->cur),
                                                           idx_of(s, s->cur), static_cast<double*>(val_of(s, s->cur)));
    else
      k_ggs_unpack<float><<<blocks, 256, 0, s->stream>>>(static_cast<float*>(dense), s->cells, cnt_of(s, s->cur),
                                                          idx_of(s, s->cur), static_cast<float*>(val_of(s, s->cur)));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(phi, dense, bytes, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  dev_free(s->hook, tmp);
  if (e != cudaSuccess) return gfail(s, MS_ERR_CUDA, std::string("sparse get fields: ") + cudaGetErrorString(e));
  return MS_OK;
}

ms_status ms_ggs_step(ms_ggs* s, int64_t n) {
  TraceRange trace("ms_ggs_step");
  if (!s || n < 0) return gfail(s, MS_ERR_ARG, "bad argument");
  for (int64_t k = 0; k < n; ++k) {
    cudaError_t e = s->s == 8 ? step_once<double>(s) : step_once<float>(s);
    if (e != cudaSuccess) return gfail(s, MS_ERR_CUDA, std::string("sparse step: ") + cudaGetErrorString(e));
    s->cur = 1 - s->cur;
    s->step += 1;
  }
  return MS_OK;
}

ms_status ms_ggs_sync(ms_ggs* s) {
  if (!s) return gfail(nullptr, MS_ERR_ARG, "ctx is NULL");
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, s->status, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return gfail(s, MS_ERR_CUDA, std::string("sparse sync: ") + cudaGetErrorString(e));
  if (st & kStatusOverflow)
    return gfail(s, MS_ERR_BOUNDS, "a cell needed more than 8 grains (or its stencil more than 8), or the input "
                                   "held a negative or non-finite value");
  return MS_OK;
}

ms_status ms_ggs_stats(ms_ggs* s, int64_t* listed_cells, int64_t* step) {
  if (!s) return gfail(nullptr, MS_ERR_ARG, "ctx is NULL");
  unsigned int cnt = 0;
  cudaError_t e = cudaMemcpyAsync(&cnt, s->list, sizeof(unsigned int), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return gfail(s, MS_ERR_CUDA, std::string("sparse stats: ") + cudaGetErrorString(e));
  if (listed_cells) *listed_cells = s->step > 0 ? (int64_t)cnt : 0;
  if (step) *step = s->step;
  return MS_OK;
}

}  // extern "C"
