// Diagnostics of one state with FP64 reductions: solute mass sum_cells c_i
// with c = sum_a h_a c^a(mu, T) (the composition constraint under Eq.
// Mu_explicit_temperature), max |sum phi - 1|, min/max phi, the count of
// non-finite values, and the largest explicit mu-diffusion number
// dt sum_faces ||chi(phi)^-1 M_f||_inf / dx^2 (the device-side dt check).
// Per-cell values are evaluated in the state's precision and accumulated in
// FP64; the two-stage reduction runs in a fixed order (deterministic).
#pragma once

#include "ms_internal.h"
#include "ms_step.cuh"

namespace msgb {

constexpr int kDiagThreads = 256;

template <int NM, class R>
__device__ __forceinline__ void inv_small(const R* A, R* X) {
  if constexpr (NM == 1) {
    X[0] = R(1) / A[0];
  } else if constexpr (NM == 2) {
    R det = A[0] * A[3] - A[1] * A[2];
    X[0] = A[3] / det;
    X[1] = -A[1] / det;
    X[2] = -A[2] / det;
    X[3] = A[0] / det;
  } else {
    R c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8];
    R c02 = A[3] * A[7] - A[4] * A[6];
    R det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    X[0] = c00 / det;
    X[3] = c01 / det;
    X[6] = c02 / det;
    X[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    X[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    X[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    X[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    X[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    X[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  }
}

// Per-thread running values of the diagnostics other than the solute sums:
// min / max phi, max |sum phi - 1|, max of the per-cell diffusion sum.  FP64
// states keep them in FP64.  FP32 states keep them in FP32 and convert once
// at the end (FP64 is a slow pipe): min and max are exact in either, the
// diffusion number dt num / dx^2 is monotone in num (its FP64 rounding
// commutes with the max), and |sum phi - 1| comes from an error-free FP32
// summation (TwoSum), so the result is the deviation rounded once to FP32.
template <class Real>
struct DiagRun {
  double lo = 1e300, hi = -1e300, dev = 0.0, num = 0.0;
  __device__ __forceinline__ void phase(Real v) {
    lo = fmin(lo, (double)v);
    hi = fmax(hi, (double)v);
  }
  template <int NP>
  __device__ __forceinline__ void sum_dev(const Real* ph) {
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < NP; ++a) s += (double)ph[a];
    dev = fmax(dev, fabs(s - 1.0));
  }
  __device__ __forceinline__ void diffusion(Real n, double dt, double inv_dx2) {
    num = fmax(num, dt * (double)n * inv_dx2);
  }
  __device__ __forceinline__ void finish(double dt, double inv_dx2, double* acc, int NM) {
    acc[NM] = dev;
    acc[NM + 1] = lo;
    acc[NM + 2] = hi;
    acc[NM + 4] = num;
  }
};

template <>
struct DiagRun<float> {
  float lo = INFINITY, hi = -INFINITY, dev = 0.0f, num = 0.0f;
  __device__ __forceinline__ void phase(float v) {
    lo = fminf(lo, v);
    hi = fmaxf(hi, v);
  }
  template <int NP>
  __device__ __forceinline__ void sum_dev(const float* ph) {
    float s = ph[0], e = 0.0f;
#pragma unroll
    for (int a = 1; a < NP; ++a) {   // TwoSum (Knuth): s + e is the exact sum
      const float t = __fadd_rn(s, ph[a]);
      const float bp = __fsub_rn(t, s);
      e = __fadd_rn(e, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(ph[a], bp)));
      s = t;
    }
    dev = fmaxf(dev, fabsf(__fadd_rn(__fsub_rn(s, 1.0f), e)));
  }
  __device__ __forceinline__ void diffusion(float n, double, double) { num = fmaxf(num, n); }
  __device__ __forceinline__ void finish(double dt, double inv_dx2, double* acc, int NM) {
    acc[NM] = (double)dev;
    acc[NM + 1] = lo == INFINITY ? 1e300 : (double)lo;
    acc[NM + 2] = hi == -INFINITY ? -1e300 : (double)hi;
    acc[NM + 4] = dt * (double)num * inv_dx2;
  }
};

template <class Real, int NP, int NM>
struct DiagConsts {
  Real chi[NP][NM * NM];
  Real DX[NP][NM * NM];
  Real B0[NP][NM], B1[NP][NM];
};

template <int DIM, int NP, int NM, class Real>
__global__ void __launch_bounds__(kDiagThreads) k_diag(const Real* __restrict__ st, int nx, int ny,
                                                       int nz, int pitch, int nyp, long long fstride,
                                                       int xoff, int zoff, int zorg, double tz0, double tzg,
                                                       double dt, double inv_dx2,
                                                       const __grid_constant__ DiagConsts<Real, NP, NM> c,
                                                       double* __restrict__ partials) {
  constexpr int NV = NM + 5;
  double acc[NV];
#pragma unroll
  for (int i = 0; i < NM; ++i) acc[i] = 0.0;
  acc[NM] = 0.0;          // max |sum phi - 1|
  acc[NM + 1] = 1e300;    // min phi
  acc[NM + 2] = -1e300;   // max phi
  acc[NM + 3] = 0.0;      // non-finite count
  acc[NM + 4] = 0.0;      // max diffusion number
  DiagRun<Real> run;
  const long long cells = (long long)nx * ny * nz;
  const long long plane = (long long)nyp * pitch;
  auto idx = [&](int x, int y, int z) {
    return (long long)(z + zoff) * plane + (long long)(y + 1) * pitch + x + xoff;
  };
  auto mob_at = [&](long long i0, Real* M) {
    Real ph[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) ph[a] = st[a * fstride + i0];
    cell_mobility<NP, NM>(ph, c.DX, M);
  };
  for (long long cidx = blockIdx.x * (long long)blockDim.x + threadIdx.x; cidx < cells;
       cidx += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(cidx % nx);
    const int y = (int)((cidx / nx) % ny);
    const int z = (int)(cidx / ((long long)nx * ny));
    const long long i0 = idx(x, y, z);
    Real ph[NP], mu[NM];
    bool finite = true;
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      ph[a] = st[a * fstride + i0];
      finite = finite && isfinite(ph[a]);
      run.phase(ph[a]);
    }
#pragma unroll
    for (int i = 0; i < NM; ++i) {
      mu[i] = st[(NP + i) * fstride + i0];
      finite = finite && isfinite(mu[i]);
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
        for (int j = 0; j < NM; ++j) ca += c.chi[a][i * NM + j] * (mu[j] - (c.B0[a][j] + c.B1[a][j] * s));
        ci += h[a] * ca;
      }
      acc[i] += (double)ci;
    }
    // explicit diffusion number of the mu update at this cell
    Real chi[NM * NM], chinv[NM * NM], Mc[NM * NM];
#pragma unroll
    for (int k = 0; k < NM * NM; ++k) {
      chi[k] = Real(0);
#pragma unroll
      for (int a = 0; a < NP; ++a) chi[k] += h[a] * c.chi[a][k];
    }
    inv_small<NM>(chi, chinv);
    mob_at(i0, Mc);
    Real num = Real(0);
#pragma unroll
    for (int d = 0; d < DIM; ++d)
#pragma unroll
      for (int sd = -1; sd <= 1; sd += 2) {
        const long long inb = idx(x + (d == 0 ? sd : 0), y + (d == 1 ? sd : 0), z + (d == 2 ? sd : 0));
        Real Mn[NM * NM];
        mob_at(inb, Mn);
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
  __shared__ double red[kDiagThreads];
  for (int v = 0; v < NV; ++v) {
    red[threadIdx.x] = acc[v];
    __syncthreads();
    for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
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

template <int NM>
__global__ void __launch_bounds__(kDiagThreads) k_diag_final(const double* __restrict__ partials,
                                                             int nblocks, double* __restrict__ out,
                                                             int* status) {
  constexpr int NV = NM + 5;
  __shared__ double red[kDiagThreads];
  for (int v = 0; v < NV; ++v) {
    const bool is_sum = v < NM || v == NM + 3;
    const bool is_min = v == NM + 1;
    double r = is_sum ? 0.0 : (is_min ? 1e300 : -1e300);
    for (int b = threadIdx.x; b < nblocks; b += kDiagThreads) {
      const double o = partials[b * NV + v];
      r = is_sum ? r + o : (is_min ? fmin(r, o) : fmax(r, o));
    }
    red[threadIdx.x] = r;
    __syncthreads();
    for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
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
  if (threadIdx.x == 0 && out[NM + 3] > 0.0) atomicOr(status, kStatusNonFinite);
}

template <int DIM, int NP, int NM, class Real>
cudaError_t launch_diag(const void* state, const HostModel& m, double t, double* partials,
                        int nblocks, double* out, int* status, cudaStream_t st) {
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
  k_diag<DIM, NP, NM, Real><<<nblocks, kDiagThreads, 0, st>>>(
      reinterpret_cast<const Real*>(state), m.nx, m.ny, DIM == 3 ? m.nz : 1, m.pitch, m.nyp,
      m.fstride, m.xoff, m.zoff, m.zorg, tz0, m.G * m.dx, m.dt, 1.0 / (m.dx * m.dx), c, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_diag_final<NM><<<1, kDiagThreads, 0, st>>>(partials, nblocks, out, status);
  return cudaGetLastError();
}

}  // namespace msgb
