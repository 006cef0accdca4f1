// Elasticity with a homogeneous stiffness (MICROSIM paper, arXiv 2404.01035,
// Sec. 2 "Elasticity implementation": the homogeneous case of its
// Fourier-space equilibrium).  Before a step, from phi^n:
//   1. k_el_eig:   eps*(x) = sum_a eps*^a h_a(phi)          (dense components)
//   2. cuFFT R2C of every component
//   3. k_el_spec:  t_i = C_ijmn k_j eps*_mn, G = (C_ijkl k_j k_l)^-1,
//                  eps_kl = (k_k (G t)_l + k_l (G t)_k) / 2, zero at k = 0
//                  (no homogeneous strain), Nyquist wavenumbers taken as 0
//   4. cuFFT C2R back to the periodic strain
//   5. k_el_force: sigma = C (eps - eps*), w_b = -sigma : eps*^b per phase,
// and the step adds w_b to each phase potential psi_b, so that the phase rate
// sees d f_el / d phi_a = sum_b w_b dh_b / dphi_a.  cuFFT is opened at run
// time, so the library loads (and everything else runs) without it.
#include <cuda_runtime.h>
#include <cufft.h>
#include <dlfcn.h>

#include <cmath>
#include <mutex>

#include "ms_device.cuh"
#include "ms_rt.h"

namespace msgb {

// ------------------------------------------------------------------ cuFFT
namespace {

struct FftApi {
  decltype(&cufftPlanMany) plan_many = nullptr;
  decltype(&cufftSetStream) set_stream = nullptr;
  decltype(&cufftExecR2C) r2c = nullptr;
  decltype(&cufftExecC2R) c2r = nullptr;
  decltype(&cufftExecD2Z) d2z = nullptr;
  decltype(&cufftExecZ2D) z2d = nullptr;
  decltype(&cufftDestroy) destroy = nullptr;
  bool ok = false;
};

const FftApi& fft_api() {
  static FftApi api;
  static std::once_flag once;
  std::call_once(once, [] {
    const char* names[] = {"libcufft.so.12", "libcufft.so", "/usr/local/cuda/lib64/libcufft.so.12"};
    void* h = nullptr;
    for (const char* n : names)
      if ((h = dlopen(n, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
    if (!h) return;
    api.plan_many = reinterpret_cast<decltype(api.plan_many)>(dlsym(h, "cufftPlanMany"));
    api.set_stream = reinterpret_cast<decltype(api.set_stream)>(dlsym(h, "cufftSetStream"));
    api.r2c = reinterpret_cast<decltype(api.r2c)>(dlsym(h, "cufftExecR2C"));
    api.c2r = reinterpret_cast<decltype(api.c2r)>(dlsym(h, "cufftExecC2R"));
    api.d2z = reinterpret_cast<decltype(api.d2z)>(dlsym(h, "cufftExecD2Z"));
    api.z2d = reinterpret_cast<decltype(api.z2d)>(dlsym(h, "cufftExecZ2D"));
    api.destroy = reinterpret_cast<decltype(api.destroy)>(dlsym(h, "cufftDestroy"));
    api.ok = api.plan_many && api.set_stream && api.r2c && api.c2r && api.d2z && api.z2d && api.destroy;
  });
  return api;
}

// Symmetric components: 3-D (xx, yy, zz, yz, xz, xy), 2-D (xx, yy, xy).
template <int DIM>
struct Comp {
  static constexpr int N = DIM == 3 ? 6 : 3;
  __host__ __device__ static int index(int i, int j) {
    if (i == j) return i;
    if (DIM == 2) return 2;
    const int s = i + j;   // (1,2) -> 3, (0,2) -> 4, (0,1) -> 5
    return s == 3 ? 3 : (s == 2 ? 4 : 5);
  }
};

template <class Real>
struct ElConst {
  Real C[3][3][3][3];
  Real eig[kNMax][6];   // per phase, tensor components in Comp order
  Real kstep[3];        // 2 pi / (n dx) per axis
  int nx, ny, nz, nxh, pitch, nyp, xoff, zoff;
  long long fstride, cells, ncplx;
};

template <int DIM, int NP, class Real>
__global__ void k_el_eig(const ElConst<Real> q, const Real* __restrict__ st, Real* __restrict__ E) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= q.cells) return;
  const int x = (int)(idx % q.nx), y = (int)((idx / q.nx) % q.ny), z = (int)(idx / ((long long)q.nx * q.ny));
  const long long o = (long long)(DIM == 3 ? z + q.zoff : 0) * q.nyp * q.pitch + (long long)(y + 1) * q.pitch + x + q.xoff;
  Real ph[NP], h[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) ph[a] = st[a * q.fstride + o];
  interp_h<NP>(ph, h);
#pragma unroll
  for (int c = 0; c < Comp<DIM>::N; ++c) {
    Real e = Real(0);
#pragma unroll
    for (int a = 0; a < NP; ++a) e += h[a] * q.eig[a][c];
    E[c * q.cells + idx] = e;
  }
}

template <class Real>
struct Cplx {
  Real re, im;
};

// Wavenumber of FFT index i of an extent n (the Nyquist index of an even n -> 0).
template <class Real>
__device__ __forceinline__ Real wavenumber(int i, int n, Real step) {
  if (2 * i == n) return Real(0);
  return step * Real(2 * i < n ? i : i - n);
}

template <int DIM, class Real>
__global__ void k_el_spec(const ElConst<Real> q, Cplx<Real>* __restrict__ S) {
  using Cp = Comp<DIM>;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= q.ncplx) return;
  const int mx = (int)(idx % q.nxh), my = (int)((idx / q.nxh) % q.ny), mz = (int)(idx / ((long long)q.nxh * q.ny));
  Real k[3] = {wavenumber<Real>(mx, q.nx, q.kstep[0]), wavenumber<Real>(my, q.ny, q.kstep[1]),
               DIM == 3 ? wavenumber<Real>(mz, q.nz, q.kstep[2]) : Real(0)};
  Real k2 = Real(0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) k2 += k[d] * k[d];
  if (k2 == Real(0)) {
#pragma unroll
    for (int c = 0; c < Cp::N; ++c) S[c * q.ncplx + idx] = Cplx<Real>{Real(0), Real(0)};
    return;
  }
  Cplx<Real> e[Cp::N];
#pragma unroll
  for (int c = 0; c < Cp::N; ++c) e[c] = S[c * q.ncplx + idx];
  // t_i = C_ijmn k_j e_mn; A_ik = C_ijkl k_j k_l
  Cplx<Real> t[DIM];
  Real A[DIM][DIM];
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    t[i] = Cplx<Real>{Real(0), Real(0)};
#pragma unroll
    for (int j = 0; j < DIM; ++j)
#pragma unroll
      for (int m = 0; m < DIM; ++m)
#pragma unroll
        for (int n = 0; n < DIM; ++n) {
          const Real ck = q.C[i][j][m][n] * k[j];
          const Cplx<Real> v = e[Cp::index(m, n)];
          t[i].re += ck * v.re;
          t[i].im += ck * v.im;
        }
#pragma unroll
    for (int kk = 0; kk < DIM; ++kk) {
      Real a = Real(0);
#pragma unroll
      for (int j = 0; j < DIM; ++j)
#pragma unroll
        for (int l = 0; l < DIM; ++l) a += q.C[i][j][kk][l] * k[j] * k[l];
      A[i][kk] = a;
    }
  }
  // G = A^-1 (adjugate over the determinant)
  Real G[DIM][DIM];
  if constexpr (DIM == 2) {
    const Real det = A[0][0] * A[1][1] - A[0][1] * A[1][0];
    G[0][0] = A[1][1] / det;
    G[0][1] = -A[0][1] / det;
    G[1][0] = -A[1][0] / det;
    G[1][1] = A[0][0] / det;
  } else {
    const Real c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1], c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
    const Real c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
    const Real det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
    G[0][0] = c00 / det;
    G[1][0] = c01 / det;
    G[2][0] = c02 / det;
    G[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
    G[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
    G[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
    G[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
    G[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
    G[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
  }
  Cplx<Real> gt[DIM];
#pragma unroll
  for (int kk = 0; kk < DIM; ++kk) {
    gt[kk] = Cplx<Real>{Real(0), Real(0)};
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      gt[kk].re += G[kk][i] * t[i].re;
      gt[kk].im += G[kk][i] * t[i].im;
    }
  }
  const Real scale = Real(1) / Real(q.cells);   // the inverse transform is unnormalised
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = i; j < DIM; ++j) {
      const Real re = Real(0.5) * (k[i] * gt[j].re + k[j] * gt[i].re);
      const Real im = Real(0.5) * (k[i] * gt[j].im + k[j] * gt[i].im);
      S[Cp::index(i, j) * q.ncplx + idx] = Cplx<Real>{re * scale, im * scale};
    }
}

template <int DIM, int NP, class Real>
__global__ void k_el_force(const ElConst<Real> q, const Real* __restrict__ E, const Real* __restrict__ eps,
                           Real* __restrict__ W) {
  using Cp = Comp<DIM>;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= q.cells) return;
  Real d[Cp::N];
#pragma unroll
  for (int c = 0; c < Cp::N; ++c) d[c] = eps[c * q.cells + idx] - E[c * q.cells + idx];
  Real sig[Cp::N];
#pragma unroll
  for (int i = 0; i < DIM; ++i)
#pragma unroll
    for (int j = i; j < DIM; ++j) {
      Real s = Real(0);
#pragma unroll
      for (int k = 0; k < DIM; ++k)
#pragma unroll
        for (int l = 0; l < DIM; ++l) s += q.C[i][j][k][l] * d[Cp::index(k, l)];
      sig[Cp::index(i, j)] = s;
    }
#pragma unroll
  for (int b = 0; b < NP; ++b) {
    Real w = Real(0);
#pragma unroll
    for (int i = 0; i < DIM; ++i)
#pragma unroll
      for (int j = 0; j < DIM; ++j) w += sig[Cp::index(i, j)] * q.eig[b][Cp::index(i, j)];
    W[b * q.cells + idx] = -w;
  }
}

template <class Real>
ElConst<Real> make_const(const HostModel& m) {
  ElConst<Real> q{};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) q.C[i][j][k][l] = (Real)m.elC[i][j][k][l];
  for (int a = 0; a < m.N; ++a)
    for (int i = 0; i < m.dim; ++i)
      for (int j = 0; j < m.dim; ++j)
        q.eig[a][m.dim == 3 ? Comp<3>::index(i, j) : Comp<2>::index(i, j)] = (Real)m.eig[a][i][j];
  const double two_pi = 6.28318530717958647692;
  q.kstep[0] = (Real)(two_pi / (m.nx * m.dx));
  q.kstep[1] = (Real)(two_pi / (m.ny * m.dx));
  q.kstep[2] = (Real)(two_pi / ((m.dim == 3 ? m.nz : 1) * m.dx));
  q.nx = m.nx;
  q.ny = m.ny;
  q.nz = m.dim == 3 ? m.nz : 1;
  q.nxh = m.nx / 2 + 1;
  q.pitch = m.pitch;
  q.nyp = m.nyp;
  q.xoff = m.xoff;
  q.zoff = m.zoff;
  q.fstride = m.fstride;
  q.cells = (long long)m.nx * m.ny * q.nz;
  q.ncplx = (long long)q.nxh * m.ny * q.nz;
  return q;
}

template <int DIM, int NP, class Real>
cudaError_t launch_el_cells(const ElConst<Real>& q, const void* st, ElasticState& s, int stage, cudaStream_t str) {
  const int blocks = (int)((q.cells + 255) / 256);
  if (stage == 0)
    k_el_eig<DIM, NP, Real><<<blocks, 256, 0, str>>>(q, static_cast<const Real*>(st), static_cast<Real*>(s.E));
  else
    k_el_force<DIM, NP, Real><<<blocks, 256, 0, str>>>(q, static_cast<const Real*>(s.E),
                                                        static_cast<const Real*>(s.eps), static_cast<Real*>(s.W));
  return cudaGetLastError();
}

template <int DIM, class Real>
cudaError_t launch_el_np(int np, const ElConst<Real>& q, const void* st, ElasticState& s, int stage,
                         cudaStream_t str) {
  switch (np) {
    case 2: return launch_el_cells<DIM, 2, Real>(q, st, s, stage, str);
    case 3: return launch_el_cells<DIM, 3, Real>(q, st, s, stage, str);
    case 8: return launch_el_cells<DIM, 8, Real>(q, st, s, stage, str);
    default: return cudaErrorInvalidValue;
  }
}

template <class Real>
cudaError_t solve(const HostModel& m, const void* st, ElasticState& s, cudaStream_t str) {
  const FftApi& f = fft_api();
  const ElConst<Real> q = make_const<Real>(m);
  cudaError_t e = m.dim == 3 ? launch_el_np<3, Real>(m.N, q, st, s, 0, str) : launch_el_np<2, Real>(m.N, q, st, s, 0, str);
  if (e != cudaSuccess) return e;
  const bool dbl = sizeof(Real) == 8;
  cufftResult r = dbl ? f.d2z(s.plan_r2c, static_cast<cufftDoubleReal*>(s.E), static_cast<cufftDoubleComplex*>(s.spec))
                      : f.r2c(s.plan_r2c, static_cast<cufftReal*>(s.E), static_cast<cufftComplex*>(s.spec));
  if (r != CUFFT_SUCCESS) return cudaErrorUnknown;
  const int blocks = (int)((q.ncplx + 255) / 256);
  if (m.dim == 3)
    k_el_spec<3, Real><<<blocks, 256, 0, str>>>(q, static_cast<Cplx<Real>*>(s.spec));
  else
    k_el_spec<2, Real><<<blocks, 256, 0, str>>>(q, static_cast<Cplx<Real>*>(s.spec));
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  r = dbl ? f.z2d(s.plan_c2r, static_cast<cufftDoubleComplex*>(s.spec), static_cast<cufftDoubleReal*>(s.eps))
          : f.c2r(s.plan_c2r, static_cast<cufftComplex*>(s.spec), static_cast<cufftReal*>(s.eps));
  if (r != CUFFT_SUCCESS) return cudaErrorUnknown;
  return m.dim == 3 ? launch_el_np<3, Real>(m.N, q, st, s, 1, str) : launch_el_np<2, Real>(m.N, q, st, s, 1, str);
}

}  // namespace

bool elastic_available() { return fft_api().ok; }

namespace {
void release_state(ms_ctx* c, ElasticState& s) {
  const FftApi& f = fft_api();
  if (f.ok) {
    if (s.has_r2c) f.destroy(s.plan_r2c);
    if (s.has_c2r) f.destroy(s.plan_c2r);
  }
  dev_free(c->hook, s.E);
  dev_free(c->hook, s.eps);
  dev_free(c->hook, s.spec);
  dev_free(c->hook, s.W);
  s = ElasticState{};
}
}  // namespace

bool elastic_grid_fits(const HostModel& m) {
  // the batched plans take the per-transform distance (cells) as an int
  const long long cells = (long long)m.nx * m.ny * (m.dim == 3 ? m.nz : 1);
  return cells <= 0x7FFFFFFFll;
}

ms_status elastic_setup(ms_ctx* c) {
  const HostModel& m = c->m;
  // the step kernels read the elastic potentials only while elasticity is on
  // (ms_update_params may turn it on or off)
  c->lg.elw = m.el && c->el.ready ? c->el.W : nullptr;
  if (!m.el || c->el.ready) return MS_OK;
  const FftApi& f = fft_api();
  if (!f.ok) return fail(c, MS_ERR_UNSUPPORTED, "elasticity needs cuFFT (libcufft.so.12), which could not be opened");
  if (m.N != 2 && m.N != 3 && m.N != 8) return fail(c, MS_ERR_UNSUPPORTED, "elasticity: phases must be 2, 3 or 8");
  if (!elastic_grid_fits(m)) return fail(c, MS_ERR_UNSUPPORTED, "grid too large for the FFT plans of the elasticity");
  // everything is built in a local state and handed to the context only when
  // every buffer and both plans exist; a failure part-way frees what was made
  ElasticState s;
  const int nz = m.dim == 3 ? m.nz : 1;
  const long long cells = (long long)m.nx * m.ny * nz;
  const long long ncplx = (long long)(m.nx / 2 + 1) * m.ny * nz;
  s.ncomp = m.dim == 3 ? 6 : 3;
  const size_t real = m.dtype == MS_F64 ? 8 : 4;
  s.E = dev_alloc(c->hook, s.ncomp * cells * real);
  s.eps = dev_alloc(c->hook, s.ncomp * cells * real);
  s.spec = dev_alloc(c->hook, s.ncomp * ncplx * 2 * real);
  s.W = dev_alloc(c->hook, (size_t)m.N * cells * real);
  if (!s.E || !s.eps || !s.spec || !s.W) {
    release_state(c, s);
    return fail(c, MS_ERR_OOM, "elasticity buffers");
  }
  int n3[3] = {nz, m.ny, m.nx};
  int* n = m.dim == 3 ? n3 : n3 + 1;
  const int rank = m.dim;
  const int idist = (int)cells, odist = (int)ncplx;
  int inr[3] = {nz, m.ny, m.nx}, onr[3] = {nz, m.ny, m.nx / 2 + 1};
  int* inb = m.dim == 3 ? inr : inr + 1;
  int* onb = m.dim == 3 ? onr : onr + 1;
  const bool dbl = m.dtype == MS_F64;
  cufftHandle p1 = 0, p2 = 0;
  const bool ok1 = f.plan_many(&p1, rank, n, inb, 1, idist, onb, 1, odist, dbl ? CUFFT_D2Z : CUFFT_R2C, s.ncomp) ==
                   CUFFT_SUCCESS;
  if (ok1) {
    s.plan_r2c = p1;
    s.has_r2c = true;
  }
  const bool ok2 = ok1 && f.plan_many(&p2, rank, n, onb, 1, odist, inb, 1, idist, dbl ? CUFFT_Z2D : CUFFT_C2R,
                                      s.ncomp) == CUFFT_SUCCESS;
  if (ok2) {
    s.plan_c2r = p2;
    s.has_c2r = true;
  }
  if (!ok1 || !ok2) {
    release_state(c, s);
    return fail(c, MS_ERR_CUDA, "cuFFT plan creation failed");
  }
  if (f.set_stream(p1, c->stream) != CUFFT_SUCCESS || f.set_stream(p2, c->stream) != CUFFT_SUCCESS) {
    release_state(c, s);
    return fail(c, MS_ERR_CUDA, "cuFFT stream");
  }
  s.ready = true;
  c->el = s;
  c->lg.elw = s.W;
  return MS_OK;
}

ms_status elastic_solve(ms_ctx* c, const void* state) {
  cudaError_t e = c->m.dtype == MS_F64 ? solve<double>(c->m, state, c->el, c->stream)
                                       : solve<float>(c->m, state, c->el, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "elastic equilibrium");
  return MS_OK;
}

void elastic_free(ms_ctx* c) { release_state(c, c->el); }

}  // namespace msgb
