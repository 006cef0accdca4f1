// Allocation-free diagnostics: ms_diag_noalloc.
//
// Some callers cannot allocate device memory while they run: a solver that
// embeds this library inside its own memory pool with a fixed budget, code
// running under a CUDA stream capture (where cudaMalloc would break or
// serialise the capture), and real-time loops that must not stall on the
// allocator.  They still want the solute-mass / stability diagnostics of a
// state they hold themselves.  This entry point computes exactly the
// quantities of ms_diag from dense device fields the caller passes in, and
// writes them to a device buffer the caller also passes in.  Its only working
// memory is the file-scope array below, which exists once per device for the
// lifetime of the process.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/microsim_gb.h"
#include "ms_diag.cuh"
#include "ms_rt.h"

namespace msgb {

ms_status build_model(ms_ctx* c, const ms_grid* g, int N, int K, const ms_params* p, HostModel& m);

namespace {

constexpr int kNaThreads = 256;
constexpr long long kNaCellsPerBlock = 256ll * 128;   // fixed: reduction order is size-only
constexpr int kNaMaxBlocks = 8192;                    // => at most 268,435,456 cells
constexpr int kNaMaxValues = kKMax + 5;               // per-block partials

// Per-block FP64 partial sums of the last call.  Every block of a call
// overwrites its own slots before the final reduction reads them, so nothing
// has to be cleared between calls.
static __device__ __align__(256) double g_noalloc_partials[kNaMaxBlocks * kNaMaxValues];

__device__ __forceinline__ int na_map(int i, int n, int bc) {
  if (i >= 0 && i < n) return i;
  if (bc == 3) return ((i % n) + n) % n;
  return i < 0 ? 0 : n - 1;
}

// Dense-layout twin of k_diag: same per-cell arithmetic, neighbours found by
// the boundary mapping instead of ghost cells.
template <int DIM, int NP, int NM, class Real>
__global__ void __launch_bounds__(kNaThreads) k_diag_dense(
    const Real* __restrict__ phi, const Real* __restrict__ mu, int nx, int ny, int nz, int bcx, int bcy,
    int bcz, int zorg, double tz0, double tzg, double dt, double inv_dx2,
    const __grid_constant__ DiagConsts<Real, NP, NM> c, double* __restrict__ partials) {
  constexpr int NV = NM + 5;
  double acc[NV];
#pragma unroll
  for (int i = 0; i < NM; ++i) acc[i] = 0.0;
  acc[NM] = 0.0;
  acc[NM + 1] = 1e300;
  acc[NM + 2] = -1e300;
  acc[NM + 3] = 0.0;
  acc[NM + 4] = 0.0;
  DiagRun<Real> run;
  const long long cells = (long long)nx * ny * nz;
  auto idx = [&](int x, int y, int z) { return ((long long)z * ny + y) * nx + x; };
  auto mob_at = [&](long long i0, Real* M) {
    Real ph[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) ph[a] = phi[a * cells + i0];
    cell_mobility<NP, NM>(ph, c.DX, M);
  };
  const long long first = blockIdx.x * kNaCellsPerBlock;
  const long long last = min(cells, first + kNaCellsPerBlock);
  for (long long cidx = first + threadIdx.x; cidx < last; cidx += kNaThreads) {
    const int x = (int)(cidx % nx);
    const int y = (int)((cidx / nx) % ny);
    const int z = (int)(cidx / ((long long)nx * ny));
    Real ph[NP], m[NM];
    bool finite = true;
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      ph[a] = phi[a * cells + cidx];
      finite = finite && isfinite(ph[a]);
      run.phase(ph[a]);
    }
#pragma unroll
    for (int i = 0; i < NM; ++i) {
      m[i] = mu[i * cells + cidx];
      finite = finite && isfinite(m[i]);
    }
    if (!finite) {
      acc[NM + 3] += 1.0;
      continue;
    }
    run.template sum_dev<NP>(ph);
    Real h[NP];
    interp_h<NP>(ph, h);
    const Real s = (Real)(tz0 + tzg * ((DIM == 3 ? z : y) + zorg + 0.5));
#pragma unroll
    for (int i = 0; i < NM; ++i) {
      Real ci = Real(0);
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        Real ca = Real(0);
#pragma unroll
        for (int j = 0; j < NM; ++j) ca += c.chi[a][i * NM + j] * (m[j] - (c.B0[a][j] + c.B1[a][j] * s));
        ci += h[a] * ca;
      }
      acc[i] += (double)ci;
    }
    Real chi[NM * NM], chinv[NM * NM], Mc[NM * NM];
#pragma unroll
    for (int k = 0; k < NM * NM; ++k) {
      chi[k] = Real(0);
#pragma unroll
      for (int a = 0; a < NP; ++a) chi[k] += h[a] * c.chi[a][k];
    }
    inv_small<NM>(chi, chinv);
    mob_at(cidx, Mc);
    Real num = Real(0);
#pragma unroll
    for (int d = 0; d < DIM; ++d)
#pragma unroll
      for (int sd = -1; sd <= 1; sd += 2) {
        const int xn = d == 0 ? na_map(x + sd, nx, bcx) : x;
        const int yn = d == 1 ? na_map(y + sd, ny, bcy) : y;
        const int zn = d == 2 ? na_map(z + sd, nz, bcz) : z;
        Real Mn[NM * NM];
        mob_at(idx(xn, yn, zn), Mn);
        Real rmax = Real(0);
#pragma unroll
        for (int i = 0; i < NM; ++i) {
          Real r = Real(0);
#pragma unroll
          for (int j = 0; j < NM; ++j) {
            Real e = Real(0);
#pragma unroll
            for (int k = 0; k < NM; ++k) e += chinv[i * NM + k] * (Real(0.5) * (Mc[k * NM + j] + Mn[k * NM + j]));
            r += fabs(e);
          }
          rmax = fmax(rmax, r);
        }
        num += rmax;
      }
    run.diffusion(num, dt, inv_dx2);
  }
  run.finish(dt, inv_dx2, acc, NM);
  __shared__ double red[kNaThreads];
  for (int v = 0; v < NV; ++v) {
    red[threadIdx.x] = acc[v];
    __syncthreads();
    for (int w = kNaThreads / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) {
        const double o = red[threadIdx.x + w];
        double& r = red[threadIdx.x];
        if (v < NM || v == NM + 3) r += o;
        else if (v == NM + 1) r = fmin(r, o);
        else r = fmax(r, o);
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x * NV + v] = red[0];
    __syncthreads();
  }
}

// Final fixed-order reduction of the per-block partials into the caller's buffer.
template <int NM>
__global__ void __launch_bounds__(kNaThreads) k_diag_dense_final(const double* __restrict__ partials,
                                                                 int nblocks, double* __restrict__ out) {
  constexpr int NV = NM + 5;
  __shared__ double red[kNaThreads];
  for (int v = 0; v < NV; ++v) {
    const bool is_sum = v < NM || v == NM + 3;
    const bool is_min = v == NM + 1;
    double r = is_sum ? 0.0 : (is_min ? 1e300 : -1e300);
    for (int b = threadIdx.x; b < nblocks; b += kNaThreads) {
      const double o = partials[b * NV + v];
      r = is_sum ? r + o : (is_min ? fmin(r, o) : fmax(r, o));
    }
    red[threadIdx.x] = r;
    __syncthreads();
    for (int w = kNaThreads / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) {
        const double o = red[threadIdx.x + w];
        double& q = red[threadIdx.x];
        q = is_sum ? q + o : (is_min ? fmin(q, o) : fmax(q, o));
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) out[v] = red[0];
    __syncthreads();
  }
}

template <int DIM, int NP, int NM, class Real>
cudaError_t na_launch(const HostModel& m, double t, const void* phi, const void* mu, double* partials,
                      int nblocks, double* out, cudaStream_t st) {
  DiagConsts<Real, NP, NM> c;
  for (int a = 0; a < NP; ++a) {
    for (int k = 0; k < NM * NM; ++k) {
      c.chi[a][k] = (Real)m.chi[a][k];
      c.DX[a][k] = (Real)m.DX[a][k];
    }
    for (int i = 0; i < NM; ++i) {
      c.B0[a][i] = (Real)m.B0[a][i];
      c.B1[a][i] = (Real)m.B1[a][i];
    }
  }
  const double tz0 = m.T0 - m.T_ref - m.G * (m.z0 + m.V * t);
  k_diag_dense<DIM, NP, NM, Real><<<nblocks, kNaThreads, 0, st>>>(
      static_cast<const Real*>(phi), static_cast<const Real*>(mu), m.nx, m.ny, DIM == 3 ? m.nz : 1, m.bc[0],
      m.bc[1], m.bc[2], m.zorg, tz0, m.G * m.dx, m.dt, 1.0 / (m.dx * m.dx), c, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_diag_dense_final<NM><<<1, kNaThreads, 0, st>>>(partials, nblocks, out);
  return cudaGetLastError();
}

typedef cudaError_t (*NaFn)(const HostModel&, double, const void*, const void*, double*, int, double*,
                            cudaStream_t);

NaFn na_find(int dim, int np, int nm, int dtype) {
#define MS_NA(D, P, M)                                                            \
  if (dim == D && np == P && nm == M) return dtype ? &na_launch<D, P, M, double> \
                                                   : &na_launch<D, P, M, float>;
  MS_NA(2, 2, 1)
  MS_NA(2, 3, 2)
  MS_NA(3, 2, 1)
  MS_NA(3, 3, 2)
  MS_NA(3, 8, 1)
#undef MS_NA
  return nullptr;
}

// Device address of g_noalloc_partials, looked up once per device.
constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
double* g_na_ptr[kNaMaxDevices] = {};

}  // namespace
}  // namespace msgb

using namespace msgb;

extern "C" ms_status ms_diag_noalloc(const ms_grid* grid, int n_phases, int n_components,
                                     const ms_params* params, double t, const void* phi_dev,
                                     const void* mu_dev, double* out_dev, void* stream) {
  if (!phi_dev || !mu_dev || !out_dev) return fail(nullptr, MS_ERR_ARG, "phi, mu and out are required");
  HostModel m;
  ms_status s = build_model(nullptr, grid, n_phases, n_components, params, m);
  if (s != MS_OK) return s;
  NaFn fn = na_find(m.dim, m.N, m.NM, m.dtype);
  if (!fn) return fail(nullptr, MS_ERR_UNSUPPORTED, "no compiled diagnostics for this (dim, N, K)");
  const long long cells = (long long)m.nx * m.ny * m.nz;
  const long long nblocks = (cells + kNaCellsPerBlock - 1) / kNaCellsPerBlock;
  if (nblocks > kNaMaxBlocks)
    return fail(nullptr, MS_ERR_BOUNDS,
                "grid of " + std::to_string(cells) + " cells exceeds the allocation-free diagnostics limit of " +
                    std::to_string((long long)kNaMaxBlocks * kNaCellsPerBlock) + " cells");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
  if (dev < 0 || dev >= kNaMaxDevices) return fail(nullptr, MS_ERR_BOUNDS, "device index out of range");
  double* partials = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
      // first call on this device: resolve the device address of the
      // file-scope scratch array with this device current
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_partials);
      if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetSymbolAddress(g_noalloc_partials)");
      g_na_ptr[dev] = static_cast<double*>(p);
    }
    partials = g_na_ptr[dev];
  }
  e = fn(m, t, phi_dev, mu_dev, partials, (int)nblocks, out_dev, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "allocation-free diagnostics launch");
  return MS_OK;
}
