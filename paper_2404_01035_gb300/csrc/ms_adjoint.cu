// Discrete adjoint of the explicit grand-potential step (reverse mode over
// time, checkpointed), plus the snapshot bookkeeping it needs.
//
// One reverse step maps lambda^{n+1} = dL/d(phi^{n+1}, mu^{n+1}) to
// lambda^n = J_n^T lambda^{n+1}, J_n the Jacobian of the step at state n, and
// adds lambda^{n+1} . d(step)/d(theta) to the parameter gradients, theta =
// (delta_ab per pair, phase mobility 1/tau, D^a entries).
//
// J_n^T is applied as a gather, one thread per input cell j, with no atomics:
// cell j's value is read by every cell i whose stencil covers one of j's
// positions p (j itself, or a ghost image of j across a periodic / no-flux
// face).  For each such (p, i) the thread re-evaluates cell i's update with
// forward-mode dual numbers seeded on all fields at position p, and contracts
// the result with lambda_i^{n+1}.  Each (i, p) pair is evaluated once over the
// grid, so the cost is (stencil size) dual evaluations per cell.  The
// parameter derivative is one more dual evaluation per cell, seeded on theta,
// reduced per block in FP64 and summed in a fixed order (deterministic).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/microsim_gb.h"
#include "ms_launch.cuh"
#include "ms_rt.h"

namespace msgb {

template <int NP, int NM>
struct ParamCount {
  static constexpr int P = NP * (NP - 1) / 2;
  static constexpr int value = P + 1 + NP * NM * NM;   // delta pairs, mobility, D entries
};

template <class Real, int NP, int NM>
struct AdjExtra {
  Real D[NP][NM * NM];
};

// Stencil accessor over the padded state in global memory, yielding duals.
// SEED: derivative slot a (phase) / NP + i (solute) is 1 at padded index
// `seed`; otherwise all derivatives are zero.
template <int DIM, int NP, int NM, class R, int W, bool SEED, class DXT>
struct GAcc {
  using D = Dual<R, W>;
  const R* st;
  long long fstride, plane, base, seed;
  int pitch;
  const DXT* DX;

  __device__ __forceinline__ D load(int f, int dx, int dy, int dz) const {
    const long long idx = base + dz * plane + (long long)dy * pitch + dx;
    D v(st[f * fstride + idx]);
    if constexpr (SEED) {
      if (idx == seed) v.d[f] = R(1);
    }
    return v;
  }
  __device__ __forceinline__ D phi(int a, int dx, int dy, int dz) const { return load(a, dx, dy, dz); }
  __device__ __forceinline__ D mu(int i, int dx, int dy, int dz) const { return load(NP + i, dx, dy, dz); }
  __device__ __forceinline__ uint32_t mask() const { return (1u << NP) - 1u; }
  __device__ __forceinline__ void mobility(int dx, int dy, int dz, D* M) const {
    D ph[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) ph[a] = phi(a, dx, dy, dz);
    cell_mobility<NP, NM>(ph, *DX, M);
  }
};

template <int DIM, int NP, int NM, class Real>
__global__ void __launch_bounds__(128) k_adjoint(const Real* __restrict__ st, const Real* __restrict__ lam_in,
                                                 Real* __restrict__ lam_out,
                                                 const __grid_constant__ StepArgs<Real, NP, NM> g,
                                                 const __grid_constant__ AdjExtra<Real, NP, NM> ex,
                                                 double* __restrict__ partials) {
  constexpr int NF = NP + NM;
  constexpr int P = NP * (NP - 1) / 2;
  constexpr int NPRM = ParamCount<NP, NM>::value;
  using DF = Dual<Real, NF>;
  using DPm = Dual<Real, NPRM>;
  const long long cells = (long long)g.nx * g.ny * g.nz;
  const long long plane = (long long)g.nyp * g.pitch;
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const bool live = j < cells;
  double gpar[NPRM];
#pragma unroll
  for (int k = 0; k < NPRM; ++k) gpar[k] = 0.0;
  if (live) {
    const int x = (int)(j % g.nx), y = (int)((j / g.nx) % g.ny), z = (int)(j / ((long long)g.nx * g.ny));
    auto padded = [&](int px, int py, int pz) {
      return (long long)(pz + g.zoff) * plane + (long long)(py + 1) * g.pitch + px + g.xoff;
    };
    auto dense = [&](int px, int py, int pz) { return ((long long)pz * g.ny + py) * g.nx + px; };
    // positions holding cell j's value: itself and its ghost images
    int xs[3], ys[3], zs[3], nxs = 1, nys = 1, nzs = 1;
    xs[0] = x;
    ys[0] = y;
    zs[0] = z;
    if (x == 0) xs[nxs++] = g.bc[0] == 3 ? g.nx : -1;
    if (x == g.nx - 1) xs[nxs++] = g.bc[0] == 3 ? -1 : g.nx;
    if (y == 0) ys[nys++] = g.bc[1] == 3 ? g.ny : -1;
    if (y == g.ny - 1) ys[nys++] = g.bc[1] == 3 ? -1 : g.ny;
    if (DIM == 3) {
      if (z == 0) zs[nzs++] = g.bc[2] == 3 ? g.nz : -1;
      if (z == g.nz - 1) zs[nzs++] = g.bc[2] == 3 ? -1 : g.nz;
    }
    DiffPrm<DF, P> dpf;
    dpf.mob = DF(g.mob);
#pragma unroll
    for (int p = 0; p < P; ++p) dpf.delta[p] = DF(g.delta[p]);
    Real acc[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) acc[f] = Real(0);
#pragma unroll 1
    for (int iz = 0; iz < nzs; ++iz)
#pragma unroll 1
      for (int iy = 0; iy < nys; ++iy)
#pragma unroll 1
        for (int ix = 0; ix < nxs; ++ix) {
          const int px = xs[ix], py = ys[iy], pz = zs[iz];
          const long long seed = padded(px, py, pz);
#pragma unroll 1
          for (int o = 0; o < (DIM == 3 ? 27 : 9); ++o) {
            const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = DIM == 3 ? o / 9 - 1 : 0;
            if (DIM == 3 && dx != 0 && dy != 0 && dz != 0) continue;   // corners: not in the stencil
            const int rx = px - dx, ry = py - dy, rz = pz - dz;       // reader cell
            if (rx < 0 || rx >= g.nx || ry < 0 || ry >= g.ny || rz < 0 || rz >= (DIM == 3 ? g.nz : 1))
              continue;
            GAcc<DIM, NP, NM, Real, NF, true, Real[NP][NM * NM]> A;
            A.st = st;
            A.fstride = g.fstride;
            A.plane = plane;
            A.pitch = g.pitch;
            A.base = padded(rx, ry, rz);
            A.seed = seed;
            A.DX = &g.DX;
            DF pn[NP], mn[NM];
            gp_cell<DIM, NP, NM, Real, DF>(A, g, dpf, (DIM == 3 ? rz : ry) + g.zorg, lab_cell<DIM>(g, rx, ry, rz), pn,
                                           mn);
            const long long ri = dense(rx, ry, rz);
#pragma unroll
            for (int a = 0; a < NP; ++a) {
              const Real l = lam_in[a * cells + ri];
#pragma unroll
              for (int f = 0; f < NF; ++f) acc[f] += l * pn[a].d[f];
            }
#pragma unroll
            for (int i = 0; i < NM; ++i) {
              const Real l = lam_in[(NP + i) * cells + ri];
#pragma unroll
              for (int f = 0; f < NF; ++f) acc[f] += l * mn[i].d[f];
            }
          }
        }
#pragma unroll
    for (int f = 0; f < NF; ++f) lam_out[f * cells + j] = acc[f];

    if (partials) {
      // parameter derivative of cell j's own update
      DiffPrm<DPm, P> dpp;
      dpp.mob = DPm(g.mob);
      dpp.mob.d[P] = Real(1);
#pragma unroll
      for (int p = 0; p < P; ++p) {
        dpp.delta[p] = DPm(g.delta[p]);
        dpp.delta[p].d[p] = Real(1);
      }
      DPm DXd[NP][NM * NM];
#pragma unroll
      for (int a = 0; a < NP; ++a)
#pragma unroll
        for (int r = 0; r < NM; ++r)
#pragma unroll
          for (int c = 0; c < NM; ++c) {
            DPm s(Real(0));
#pragma unroll
            for (int m = 0; m < NM; ++m) {
              DPm Dm(ex.D[a][r * NM + m]);
              Dm.d[P + 1 + (a * NM + r) * NM + m] = Real(1);
              s += Dm * DPm(g.chi[a][m * NM + c]);
            }
            DXd[a][r * NM + c] = s;
          }
      GAcc<DIM, NP, NM, Real, NPRM, false, DPm[NP][NM * NM]> A;
      A.st = st;
      A.fstride = g.fstride;
      A.plane = plane;
      A.pitch = g.pitch;
      A.base = padded(x, y, z);
      A.seed = -1;
      A.DX = &DXd;
      DPm pn[NP], mn[NM];
      gp_cell<DIM, NP, NM, Real, DPm>(A, g, dpp, (DIM == 3 ? z : y) + g.zorg, lab_cell<DIM>(g, x, y, z), pn, mn);
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        const Real l = lam_in[a * cells + j];
#pragma unroll
        for (int k = 0; k < NPRM; ++k) gpar[k] += (double)(l * pn[a].d[k]);
      }
#pragma unroll
      for (int i = 0; i < NM; ++i) {
        const Real l = lam_in[(NP + i) * cells + j];
#pragma unroll
        for (int k = 0; k < NPRM; ++k) gpar[k] += (double)(l * mn[i].d[k]);
      }
    }
  }
  if (partials) {
    __shared__ double red[128];
    for (int k = 0; k < NPRM; ++k) {
      red[threadIdx.x] = gpar[k];
      __syncthreads();
      for (int w = 64; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
      }
      if (threadIdx.x == 0) partials[blockIdx.x * NPRM + k] = red[0];
      __syncthreads();
    }
  }
}

// gsum[k] += sum over blocks of partials[b][k], in block order (deterministic).
__global__ void k_accumulate_params(const double* __restrict__ partials, int nblocks, int nprm,
                                    double* __restrict__ gsum) {
  const int k = threadIdx.x;
  if (k >= nprm) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partials[b * nprm + k];
  gsum[k] += s;
}

struct AdjKernel {
  int dim, np, nm, dtype, nprm;
  cudaError_t (*launch)(const void* state, const void* lam_in, void* lam_out, const void* blob,
                        const HostModel& m, double t, double* partials, cudaStream_t st);
};

template <int DIM, int NP, int NM, class Real>
cudaError_t launch_adjoint(const void* state, const void* lam_in, void* lam_out, const void* blob,
                           const HostModel& m, double t, double* partials, cudaStream_t st) {
  StepArgs<Real, NP, NM> g = *reinterpret_cast<const StepArgs<Real, NP, NM>*>(blob);
  g.tz0 = (Real)temp_offset(m, t);
  AdjExtra<Real, NP, NM> ex;
  for (int a = 0; a < NP; ++a)
    for (int k = 0; k < NM * NM; ++k) ex.D[a][k] = (Real)m.D[a][k];
  const long long cells = (long long)m.nx * m.ny * m.nz;
  const int blocks = (int)((cells + 127) / 128);
  k_adjoint<DIM, NP, NM, Real><<<blocks, 128, 0, st>>>(
      reinterpret_cast<const Real*>(state), reinterpret_cast<const Real*>(lam_in),
      reinterpret_cast<Real*>(lam_out), g, ex, partials);
  return cudaGetLastError();
}

template <int DIM, int NP, int NM, class Real>
AdjKernel make_adjoint() {
  return AdjKernel{DIM, NP, NM, sizeof(Real) == 8 ? 1 : 0, ParamCount<NP, NM>::value,
                   &launch_adjoint<DIM, NP, NM, Real>};
}

const std::vector<AdjKernel>& adjoint_registry() {
  static const std::vector<AdjKernel> r = {
      make_adjoint<2, 2, 1, float>(),
      make_adjoint<2, 2, 1, double>(),
      make_adjoint<2, 3, 2, double>(),
      make_adjoint<3, 2, 1, double>(),
  };
  return r;
}

const AdjKernel* find_adjoint(const HostModel& m) {
  for (auto& k : adjoint_registry())
    if (k.dim == m.dim && k.np == m.N && k.nm == m.NM && k.dtype == m.dtype) return &k;
  return nullptr;
}

void free_adjoint(ms_ctx* c) {
  AdjointStore& a = c->adj;
  for (void* p : a.snaps) dev_free(c->hook, p);
  a.snaps.clear();
  dev_free(c->hook, a.seg);
  a.seg = nullptr;
  a.seg_bytes = 0;
  for (int b = 0; b < 2; ++b) {
    dev_free(c->hook, a.adj[b]);
    a.adj[b] = nullptr;
  }
  dev_free(c->hook, a.gpart);
  a.gpart = nullptr;
  dev_free(c->hook, a.gsum);
  a.gsum = nullptr;
}

}  // namespace msgb

using namespace msgb;

ms_status ms_before_step(ms_ctx* c) {
  AdjointStore& a = c->adj;
  if (a.every <= 0) return MS_OK;
  const int64_t rel = c->step - a.first_step;
  if (rel < 0 || rel % a.every != 0) return MS_OK;
  const size_t idx = (size_t)(rel / a.every);
  if (idx < a.snaps.size()) return MS_OK;
  void* p = dev_alloc(c->hook, c->state_bytes);
  if (!p) return fail(c, MS_ERR_OOM, "adjoint snapshot allocation failed");
  a.snaps.push_back(p);
  cudaError_t e = cudaMemcpyAsync(p, c->buf[c->cur], c->state_bytes, cudaMemcpyDeviceToDevice, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint snapshot");
  return MS_OK;
}

void ms_reset_extra(ms_ctx* c) {
  cudaStreamSynchronize(c->stream);
  for (void* p : c->adj.snaps) dev_free(c->hook, p);
  c->adj.snaps.clear();
  c->adj.first_step = c->step;
}

void ms_release_extra(ms_ctx* c) { free_adjoint(c); }

extern "C" {

ms_status ms_enable_checkpoints(ms_ctx* c, int every) {
  if (!c || every < 0) return fail(c, MS_ERR_ARG, "bad argument");
  if (every > 0 && !find_adjoint(c->m))
    return fail(c, MS_ERR_UNSUPPORTED, "no compiled adjoint kernel for this (dim, N, K, dtype)");
  if (every > 0 && c->m.noise_amp != 0.0)
    return fail(c, MS_ERR_UNSUPPORTED, "the adjoint does not support phi noise (noise_amp != 0)");
  if (every > 0 && (c->m.at || c->m.gg || c->m.el))
    return fail(c, MS_ERR_UNSUPPORTED,
                "the adjoint does not support the anti-trapping current, grain growth or elasticity");
  ms_reset_extra(c);
  c->adj.every = every;
  return MS_OK;
}

int ms_grad_param_count(const ms_ctx* c) {
  if (!c) return 0;
  const int P = c->m.N * (c->m.N - 1) / 2;
  return P + 1 + c->m.N * c->m.NM * c->m.NM;
}

ms_status ms_grad(ms_ctx* c, const void* dphi_T, const void* dmu_T, double* dparams, void* dphi0,
                  void* dmu0) {
  if (!c || !dphi_T) return fail(c, MS_ERR_ARG, "ctx and dphi_T are required");
  AdjointStore& A = c->adj;
  if (A.every <= 0) return fail(c, MS_ERR_STATE, "checkpoints are not enabled (ms_enable_checkpoints)");
  if (c->m.noise_amp != 0.0) return fail(c, MS_ERR_UNSUPPORTED, "the adjoint does not support phi noise (noise_amp != 0)");
  if (c->m.at || c->m.gg || c->m.el)
    return fail(c, MS_ERR_UNSUPPORTED,
                "the adjoint does not support the anti-trapping current, grain growth or elasticity");
  const AdjKernel* ak = find_adjoint(c->m);
  if (!ak) return fail(c, MS_ERR_UNSUPPORTED, "no compiled adjoint kernel for this (dim, N, K, dtype)");
  const int64_t nsteps = c->step - A.first_step;
  const int64_t nseg = (nsteps + A.every - 1) / A.every;
  if ((int64_t)A.snaps.size() < nseg) return fail(c, MS_ERR_STATE, "missing adjoint snapshots");
  const HostModel& m = c->m;
  const size_t s = m.dtype == MS_F64 ? 8 : 4;
  const int NF = m.N + m.NM;
  const long long cells = (long long)m.nx * m.ny * m.nz;
  const size_t lam_bytes = (size_t)NF * cells * s;
  const int nprm = ak->nprm;
  const int blocks = (int)((cells + 127) / 128);
  // lazily sized work buffers
  if (!A.adj[0]) {
    for (int b = 0; b < 2; ++b) {
      A.adj[b] = dev_alloc(c->hook, lam_bytes);
      if (!A.adj[b]) return fail(c, MS_ERR_OOM, "adjoint state allocation failed");
    }
  }
  if (!A.gpart) {
    A.gpart = static_cast<double*>(dev_alloc(c->hook, sizeof(double) * (size_t)blocks * nprm));
    A.gsum = static_cast<double*>(dev_alloc(c->hook, sizeof(double) * 64));
    if (!A.gpart || !A.gsum) return fail(c, MS_ERR_OOM, "gradient scratch allocation failed");
  }
  const size_t seg_need = (size_t)A.every * c->state_bytes;
  if (A.seg_bytes < seg_need) {
    dev_free(c->hook, A.seg);
    A.seg = dev_alloc(c->hook, seg_need);
    if (!A.seg) return fail(c, MS_ERR_OOM, "adjoint segment allocation failed");
    A.seg_bytes = seg_need;
  }
  cudaStream_t st = c->stream;
  cudaError_t e = cudaMemcpyAsync(A.adj[0], dphi_T, (size_t)m.N * cells * s, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) {
    char* mu_part = static_cast<char*>(A.adj[0]) + (size_t)m.N * cells * s;
    e = dmu_T ? cudaMemcpyAsync(mu_part, dmu_T, (size_t)m.NM * cells * s, cudaMemcpyDeviceToDevice, st)
              : cudaMemsetAsync(mu_part, 0, (size_t)m.NM * cells * s, st);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(A.gsum, 0, sizeof(double) * 64, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint seeding");
  int cur = 0;
  const int cur_state = c->cur;
  for (int64_t seg = nseg - 1; seg >= 0; --seg) {
    const int64_t s0 = A.first_step + seg * A.every;
    const int len = (int)std::min<int64_t>(A.every, c->step - s0);
    char* slots = static_cast<char*>(A.seg);
    e = cudaMemcpyAsync(slots, A.snaps[seg], c->state_bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "segment restore");
    if (len > 1) {
      e = c->kern->codes(slots, m, c->codes[1 - cur_state], st);
      if (e != cudaSuccess) return cuda_fail(c, e, "segment codes");
    }
    // the recompute writes into fresh slots: nothing to keep from them
    LaunchGeom lg = c->lg;
    lg.reuse_prev = 0;
    int cs = 1 - cur_state;
    for (int k = 1; k < len; ++k) {
      CUtensorMap tm, tmi;
      char* src = slots + (size_t)(k - 1) * c->state_bytes;
      if (!encode_step_maps(*c->kern, &tm, &tmi, src, m)) return fail(c, MS_ERR_CUDA, "cuTensorMapEncodeTiled failed");
      const double t = m.t0 + (double)(s0 + k - 1) * m.dt;
      e = c->kern->launch(&tm, &tmi, c->args.data(), m, t,
                          slots + (size_t)k * c->state_bytes, c->codes[cs],
                          c->codes[1 - cs], lg, st);
      if (e != cudaSuccess) return cuda_fail(c, e, "segment recompute");
      cs = 1 - cs;
    }
    for (int k = len - 1; k >= 0; --k) {
      const double t = m.t0 + (double)(s0 + k) * m.dt;
      e = ak->launch(slots + (size_t)k * c->state_bytes, A.adj[cur], A.adj[1 - cur], c->args.data(), m, t,
                     A.gpart, st);
      if (e != cudaSuccess) return cuda_fail(c, e, "adjoint step");
      k_accumulate_params<<<1, 64, 0, st>>>(A.gpart, blocks, nprm, A.gsum);
      cur = 1 - cur;
    }
  }
  // the recompute used both code buffers: restore the current state's codes
  {
    ms_status rs = refresh_codes(c);
    if (rs != MS_OK) return rs;
  }
  if (dphi0) {
    e = cudaMemcpyAsync(dphi0, A.adj[cur], (size_t)m.N * cells * s, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "dphi0 copy");
  }
  if (dmu0) {
    e = cudaMemcpyAsync(dmu0, static_cast<char*>(A.adj[cur]) + (size_t)m.N * cells * s, (size_t)m.NM * cells * s,
                        cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "dmu0 copy");
  }
  if (dparams) {
    e = cudaMemcpyAsync(dparams, A.gsum, sizeof(double) * nprm, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "gradient copy");
  }
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(c, e, "adjoint");
  return MS_OK;
}

}  // extern "C"
