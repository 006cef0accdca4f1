// Device building blocks of the grand-potential step: launch arguments,
// PTX wrappers (TMA tile loads, mbarriers, bounded waits), a forward-mode
// dual number for the adjoint, and the per-cell model arithmetic.
//
// Model: MICROSIM paper (arXiv 2404.01035) Sec. 2.1 and Sec. 3.  Each helper
// names the equation it evaluates.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ms_internal.h"

namespace msgb {

constexpr int kMaxPhases = 8;
constexpr int kMaxSolutes = 3;

// Bounded wait: give up after this many nanoseconds of %globaltimer.
constexpr unsigned long long kWaitLimitNs = 1000ull * 1000ull * 1000ull;

template <int NP>
struct PairCount {
  static constexpr int value = NP * (NP - 1) / 2;
};

// Everything one step launch needs, passed by value (grid constant).
template <class Real, int NP, int NM>
struct StepArgs {
  static constexpr int P = NP * (NP - 1) / 2;
  // geometry (elements)
  int nx, ny, nz;
  int pitch, nyp, nzp;      // padded extents: x pitch, rows incl. 2 ghosts, planes
  long long fstride;        // elements per field
  int xoff, zoff;           // index of interior x = 0 inside a row; of z = 0
  int zchunk;               // planes marched per CTA (3-D)
  int zorg;                 // global index of z-plane 0 (temperature position)
  int bc[3];
  Real* out;                // destination state (padded, NP + NM fields)
  int* status;              // sticky device status word
  // Segment codes: one byte per 32-cell x-segment of every row of every
  // plane, [nz][ny][segs]; the low bits (kCodePhase) hold l + 1 when all its
  // cells are exactly pure phase l, else 0; bit kCodeReuse is set by the
  // split step when the state one step earlier held the same pure phase there
  // (writers that do not know that state leave it clear).  Read for the input
  // state, written for the output state.
  const uint8_t* codes_in;
  uint8_t* codes_out;
  int segs;
  // Interface work list of the split 3-D step: [0] = number of listed warp
  // rows, [1] = completion ticket of the interface kernel, [2..] = the rows
  // that are not bulk, each (z << (seg_bits + y_bits)) | (y << seg_bits) |
  // segment (bit fields: decoding needs no division).
  unsigned int* iface;
  int seg_bits, y_bits;   // widths of the segment and y fields of a list entry
  unsigned int iface_cap;
  unsigned int* iface2;   // second list, same layout (rows left for the full update)
  // anti-trapping work list: [0] count, [1] ticket, [2..] row segments
  // (z ny + y) segs + segment whose block of segments is not one pure phase
  unsigned int* at_list;
  unsigned int at_cap;
  // phi noise: amplitude, seed, step index of the input state
  Real noise_amp;
  unsigned long long noise_seed, step;
  // 1 when the output buffer holds the state one step before the input
  // (ping-pong stepping): bulk rows whose pure phase is unchanged over the
  // two steps then skip phi (fused step: codes_out still describe that state
  // before they are overwritten; split step: the reuse bit of codes_in).
  int reuse_prev;
  // scalars
  Real dt, eps, inv_eps, mob, inv_dx, half_inv_dx, quarter_inv_dx, inv_dx2;
  int potential;            // 1 obstacle, 2 well
  int gg;                   // grain growth: no chemical driving force, mu held
  // elastic part of each phase potential, -sigma : eps*^b, dense
  // [NP][nz][ny][nx] (grid cell index), or NULL without elasticity
  const Real* elw;
  int has_g3;
  // pairs (a < b, row-major order)
  Real gam2[P];             // 2 gamma_ab
  Real delta[P];
  unsigned char aniso[P];   // delta_ab != 0
  unsigned char rotated[P]; // rotation differs from identity
  Real rot[P][9];
  Real cw[NP][NP];          // obstacle: 16 gamma/pi^2, well: 18 gamma
  Real g3[NP][NP][NP];      // third-order coefficients (only if has_g3)
  // thermodynamics (parabolic, Sec. 3)
  Real chi[NP][NM * NM];    // chi^a = (Hessian f^a)^-1
  Real DX[NP][NM * NM];     // D^a chi^a
  Real B0[NP][NM], B1[NP][NM];  // B^a(T) = B0 + B1 (T - T_ref)
  Real C0[NP], C1[NP], C2[NP];  // C^a(T) = C0 + C1 s + C2 s^2, s = T - T_ref
  Real dcT[NP][NM];         // c^a(mu, T^{n+1}) - c^a(mu, T^n) = chi B1 G V dt
  // single-phase (bulk) mu update: mu += Kb (sum_nb mu_nb - 2d mu) - eb
  Real Kb[NP][NM * NM];     // dt / dx^2 (chi^a)^-1 D^a chi^a
  Real eb[NP][NM];          // (chi^a)^-1 dcT^a
  // temperature along the last axis: T = tz0 + tzg * (k + 1/2), tref subtracted
  Real tz0, tzg;
};

// --------------------------------------------------------------------- dual
template <class R, int W>
struct Dual {
  R v;
  R d[W];
  __device__ __forceinline__ Dual() {}
  __device__ __forceinline__ Dual(R x) : v(x) {
#pragma unroll
    for (int i = 0; i < W; ++i) d[i] = R(0);
  }
};
template <class R, int W>
__device__ __forceinline__ Dual<R, W> operator+(const Dual<R, W>& a, const Dual<R, W>& b) {
  Dual<R, W> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < W; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <class R, int W>
__device__ __forceinline__ Dual<R, W> operator-(const Dual<R, W>& a, const Dual<R, W>& b) {
  Dual<R, W> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < W; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <class R, int W>
__device__ __forceinline__ Dual<R, W> operator-(const Dual<R, W>& a) {
  Dual<R, W> r;
  r.v = -a.v;
#pragma unroll
  for (int i = 0; i < W; ++i) r.d[i] = -a.d[i];
  return r;
}
template <class R, int W>
__device__ __forceinline__ Dual<R, W> operator*(const Dual<R, W>& a, const Dual<R, W>& b) {
  Dual<R, W> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < W; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <class R, int W>
__device__ __forceinline__ Dual<R, W> operator/(const Dual<R, W>& a, const Dual<R, W>& b) {
  Dual<R, W> r;
  R inv = R(1) / b.v;
  r.v = a.v * inv;
#pragma unroll
  for (int i = 0; i < W; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * inv;
  return r;
}
template <class R, int W>
__device__ __forceinline__ Dual<R, W> operator*(R s, const Dual<R, W>& a) {
  Dual<R, W> r;
  r.v = s * a.v;
#pragma unroll
  for (int i = 0; i < W; ++i) r.d[i] = s * a.d[i];
  return r;
}
template <class R, int W>
__device__ __forceinline__ Dual<R, W> operator*(const Dual<R, W>& a, R s) { return s * a; }
template <class R, int W>
__device__ __forceinline__ Dual<R, W> operator/(R s, const Dual<R, W>& b) {
  Dual<R, W> r;
  const R inv = R(1) / b.v;
  r.v = s * inv;
#pragma unroll
  for (int i = 0; i < W; ++i) r.d[i] = -r.v * b.d[i] * inv;
  return r;
}
template <class R, int W>
__device__ __forceinline__ Dual<R, W> operator+(const Dual<R, W>& a, R s) {
  Dual<R, W> r = a;
  r.v += s;
  return r;
}
template <class R, int W>
__device__ __forceinline__ Dual<R, W> operator+(R s, const Dual<R, W>& a) { return a + s; }
template <class R, int W>
__device__ __forceinline__ Dual<R, W> operator-(const Dual<R, W>& a, R s) {
  Dual<R, W> r = a;
  r.v -= s;
  return r;
}
template <class R, int W>
__device__ __forceinline__ Dual<R, W> operator-(R s, const Dual<R, W>& a) {
  Dual<R, W> r = -a;
  r.v += s;
  return r;
}
template <class R, int W>
__device__ __forceinline__ Dual<R, W>& operator+=(Dual<R, W>& a, const Dual<R, W>& b) {
  a = a + b;
  return a;
}
template <class R, int W>
__device__ __forceinline__ Dual<R, W>& operator-=(Dual<R, W>& a, const Dual<R, W>& b) {
  a = a - b;
  return a;
}

__device__ __forceinline__ float val(float x) { return x; }
__device__ __forceinline__ double val(double x) { return x; }
template <class R, int W>
__device__ __forceinline__ R val(const Dual<R, W>& x) { return x.v; }

// ----------------------------------------------------------- PTX wrappers
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Adds expected transaction bytes to the current phase without arriving.
__device__ __forceinline__ void mbar_expect_tx_only(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// As mbar_try_wait, but the thread may stay suspended (not issuing) for up
// to `hint_ns` while the phase is incomplete; it resumes when the phase
// completes.
__device__ __forceinline__ bool mbar_try_wait_suspend(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of the barrier, giving up after kWaitLimitNs.
// Retries suspend the waiting warp so that it leaves the issue slots to the
// warps that have work.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  unsigned long long limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (;;) {
#pragma unroll 1
    for (int i = 0; i < 8; ++i)
      if (mbar_try_wait_suspend(bar, parity, 20000u)) return true;
    if (globaltimer() - t0 > limit_ns) return false;
  }
}

// 4-D tiled TMA load of one box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Orders this thread's generic-proxy shared-memory accesses before later
// async-proxy (TMA) accesses to the same memory.
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ------------------------------------------------------------ model pieces
// Index of pair (a, b), a < b, in row-major upper-triangle order.
template <int NP>
__host__ __device__ constexpr int pair_index(int a, int b) {
  return a * NP - a * (a + 1) / 2 + (b - a - 1);
}

// g = dA/dq for A(q) = gamma a_c(R q)^2 |q|^2 with the four-fold
// Two FP32 values in one 64-bit register with the paired FP32 arithmetic of
// sm_100-class GPUs (one add / sub / mul / fma instruction for both halves,
// each rounded as the scalar operation).
struct F2 {
  unsigned long long v;
};
__device__ __forceinline__ F2 f2(float lo, float hi) {
  F2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ F2 f2s(float x) { return f2(x, x); }
__device__ __forceinline__ float f2lo(F2 a) {
  float l, h;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(l), "=f"(h) : "l"(a.v));
  return l;
}
__device__ __forceinline__ float f2hi(F2 a) {
  float l, h;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(l), "=f"(h) : "l"(a.v));
  return h;
}
__device__ __forceinline__ F2 operator+(F2 a, F2 b) {
  F2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
  F2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b) {
  F2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) {   // a * b + c
  F2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}

// ------------------------------------------------------------- phi noise
// Counter-based uniform variate in [-1/2, 1/2): the SplitMix64 finaliser
// (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
// OOPSLA 2014) applied in turn to the seed, the step index and the counter;
// the top 24 bits of the last value (exact in FP32 and FP64).
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  unsigned long long z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <class Real>
__device__ __forceinline__ Real noise_variate(unsigned long long seed, unsigned long long step,
                                              unsigned long long counter) {
  unsigned long long h = splitmix64(seed);
  h = splitmix64(h ^ step);
  h = splitmix64(h ^ counter);
  return Real(h >> 40) * Real(1.0 / 16777216.0) - Real(0.5);
}

// Lab index of cell (x, y, z): x + nx (y_lab + ny z_lab), the last axis
// offset by the grid's origin (z in 3-D, y in 2-D).
template <int DIM, class Real, int NP, int NM>
__device__ __forceinline__ unsigned long long lab_cell(const StepArgs<Real, NP, NM>& g, int x, int y, int z) {
  const long long yl = DIM == 3 ? y : y + g.zorg;
  const long long zl = DIM == 3 ? z + g.zorg : 0;
  return (unsigned long long)(x + (long long)g.nx * (yl + (long long)g.ny * zl));
}

// 1 / x: the hardware approximate reciprocal in FP32 (relative error of a
// few ulp, far below the FP32 path's tolerance), an exact division otherwise.
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
template <class R, int W>
__device__ __forceinline__ Dual<R, W> recip(const Dual<R, W>& x) {
  return R(1) / x;
}

// a_c(q) = 1 - delta (3 - 4 sum q_i^4 / |q|^4) (Eqs. Eqn_a, aniso_eqn);
// g = 2 gamma q for an isotropic pair; g = 0 when |q|^2 < 1e-12 (anisotropic).
template <int DIM, class S, class Real>
__device__ __forceinline__ void pair_grad(const S* q, Real gam2, const S& del, bool aniso,
                                          bool rotated, const Real* R, S* g) {
  if (!aniso) {
#pragma unroll
    for (int i = 0; i < DIM; ++i) g[i] = gam2 * q[i];
    return;
  }
  S Q = q[0] * q[0];
#pragma unroll
  for (int i = 1; i < DIM; ++i) Q += q[i] * q[i];
  if (val(Q) < Real(1e-12)) {
#pragma unroll
    for (int i = 0; i < DIM; ++i) g[i] = S(Real(0));
    return;
  }
  S qr[DIM];
  if (rotated) {
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      qr[i] = R[i * 3 + 0] * q[0];
#pragma unroll
      for (int j = 1; j < DIM; ++j) qr[i] += R[i * 3 + j] * q[j];
    }
  } else {
#pragma unroll
    for (int i = 0; i < DIM; ++i) qr[i] = q[i];
  }
  S invQ = recip(Q);
  S q2[DIM];
  S s4 = S(Real(0));
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    q2[i] = qr[i] * qr[i];
    s4 += q2[i] * q2[i];
  }
  S r = s4 * invQ * invQ;
  S ac = Real(1) - del * (Real(3) - Real(4) * r);
  S k16 = Real(16) * del;
  S gr[DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
    gr[i] = gam2 * ac * (ac * qr[i] + k16 * (q2[i] * qr[i] * invQ - r * qr[i]));
  if (rotated) {
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      g[j] = R[0 * 3 + j] * gr[0];
#pragma unroll
      for (int i = 1; i < DIM; ++i) g[j] += R[i * 3 + j] * gr[i];
    }
  } else {
#pragma unroll
    for (int i = 0; i < DIM; ++i) g[i] = gr[i];
  }
}

// Interpolation h_a (Eq. hphi) through e1 = sum phi, e2 = sum_{b<c} phi_b phi_c:
// sum_{b<c; b,c != a} phi_b phi_c = e2 - phi_a (e1 - phi_a).
template <int NP, class S>
__device__ __forceinline__ void interp_h(const S* ph, S* h) {
  S e1 = ph[0];
#pragma unroll
  for (int a = 1; a < NP; ++a) e1 += ph[a];
  S e2 = S(0.0f * val(e1));
  {
    S run = ph[0];
#pragma unroll
    for (int a = 1; a < NP; ++a) {
      e2 += ph[a] * run;
      run += ph[a];
    }
  }
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    S rest = e2 - ph[a] * (e1 - ph[a]);
    S p2 = ph[a] * ph[a];
    h[a] = decltype(val(e1))(3) * p2 - decltype(val(e1))(2) * p2 * ph[a] +
           decltype(val(e1))(2) * ph[a] * rest;
  }
}

// Cell mobility M = sum_a h_a(phi) D^a chi^a (Eq. Mass_conservation).
template <int NP, int NM, class S, class DXT>
__device__ __forceinline__ void cell_mobility(const S* ph, const DXT& DX, S* M) {
  S h[NP];
  interp_h<NP>(ph, h);
#pragma unroll
  for (int k = 0; k < NM * NM; ++k) {
    M[k] = h[0] * DX[0][k];
#pragma unroll
    for (int a = 1; a < NP; ++a) M[k] += h[a] * DX[a][k];
  }
}

// Small dense solve x = A^-1 b for n <= 3 by cofactors.
template <int NM, class S>
__device__ __forceinline__ void solve_small(const S* A, const S* b, S* x) {
  if constexpr (NM == 1) {
    x[0] = b[0] * recip(A[0]);
  } else if constexpr (NM == 2) {
    S det = A[0] * A[3] - A[1] * A[2];
    S inv = recip(det);
    x[0] = (A[3] * b[0] - A[1] * b[1]) * inv;
    x[1] = (A[0] * b[1] - A[2] * b[0]) * inv;
  } else {
    S c00 = A[4] * A[8] - A[5] * A[7];
    S c01 = A[5] * A[6] - A[3] * A[8];
    S c02 = A[3] * A[7] - A[4] * A[6];
    S det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    S inv = recip(det);
    S c10 = A[2] * A[7] - A[1] * A[8];
    S c11 = A[0] * A[8] - A[2] * A[6];
    S c12 = A[1] * A[6] - A[0] * A[7];
    S c20 = A[1] * A[5] - A[2] * A[4];
    S c21 = A[2] * A[3] - A[0] * A[5];
    S c22 = A[0] * A[4] - A[1] * A[3];
    x[0] = (c00 * b[0] + c10 * b[1] + c20 * b[2]) * inv;
    x[1] = (c01 * b[0] + c11 * b[1] + c21 * b[2]) * inv;
    x[2] = (c02 * b[0] + c12 * b[1] + c22 * b[2]) * inv;
  }
}

// Euclidean projection onto the simplex (sort-based; Held-Wolfe-Crowder 1974,
// Duchi et al. 2008) or onto the sum-one hyperplane: the Lagrange multiplier of
// Eq. (phi_eqn) together with the obstacle's infinite walls.
template <int NP, class S>
__device__ __forceinline__ void project(int potential, const S* v, S* out) {
  using R = decltype(val(v[0]));
  if (potential == 1) {
    S u[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) u[a] = v[a];
    // insertion sort, descending by value
#pragma unroll
    for (int i = 1; i < NP; ++i) {
#pragma unroll
      for (int j = i; j > 0; --j) {
        if (val(u[j]) > val(u[j - 1])) {
          S t = u[j];
          u[j] = u[j - 1];
          u[j - 1] = t;
        }
      }
    }
    S csum = u[0];
    S theta = u[0] - R(1);
#pragma unroll
    for (int j = 1; j < NP; ++j) {
      csum += u[j];
      S t = (csum - R(1)) * R(1.0 / (j + 1));
      if (val(u[j]) - val(t) > R(0)) theta = t;
    }
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      S d = v[a] - theta;
      out[a] = val(d) > R(0) ? d : S(R(0));
    }
  } else {
    S s = v[0];
#pragma unroll
    for (int a = 1; a < NP; ++a) s += v[a];
    S shift = (s - R(1)) * R(1.0 / NP);
#pragma unroll
    for (int a = 0; a < NP; ++a) out[a] = v[a] - shift;
  }
}

}  // namespace msgb
