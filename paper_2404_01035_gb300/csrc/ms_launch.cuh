// Host launchers of the forward step and diagnostics kernels for one
// (dim, phases, solutes, dtype) instantiation; included by the ms_inst_*.cu
// units, each of which registers its instantiations.
#pragma once

#include <cmath>
#include <cstring>

#include "ms_at.cuh"
#include "ms_diag.cuh"
#include "ms_internal.h"
#include "ms_split.cuh"
#include "ms_step.cuh"

namespace msgb {

template <int DIM, int NP, int NM, class Real>
void fill_args(void* blob, const HostModel& m, int zchunk, int* status) {
  using A = StepArgs<Real, NP, NM>;
  A& g = *reinterpret_cast<A*>(blob);
  std::memset(&g, 0, sizeof(A));
  g.nx = m.nx;
  g.ny = m.ny;
  g.nz = m.nz;
  g.pitch = m.pitch;
  g.nyp = m.nyp;
  g.nzp = m.nzp;
  g.fstride = m.fstride;
  g.xoff = m.xoff;
  g.zoff = m.zoff;
  g.zchunk = zchunk;
  g.zorg = m.zorg;
  g.noise_amp = (Real)m.noise_amp;
  g.noise_seed = m.noise_seed;
  for (int d = 0; d < 3; ++d) g.bc[d] = m.bc[d];
  g.status = status;
  g.dt = (Real)m.dt;
  g.eps = (Real)m.eps;
  g.inv_eps = (Real)(1.0 / m.eps);
  g.mob = (Real)(1.0 / m.tau);
  g.inv_dx = (Real)(1.0 / m.dx);
  g.half_inv_dx = (Real)(0.5 / m.dx);
  g.quarter_inv_dx = (Real)(0.25 / m.dx);
  g.inv_dx2 = (Real)(1.0 / (m.dx * m.dx));
  g.potential = m.potential;
  g.gg = m.gg;
  g.has_g3 = m.has_g3 ? 1 : 0;
  const double PI = 3.14159265358979323846;
  int p = 0;
  for (int a = 0; a < NP; ++a)
    for (int b = a + 1; b < NP; ++b, ++p) {
      g.gam2[p] = (Real)(2.0 * m.gamma[a][b]);
      g.delta[p] = (Real)m.delta[a][b];
      g.aniso[p] = m.delta[a][b] != 0.0;
      g.rotated[p] = m.rotated[a][b];
      for (int k = 0; k < 9; ++k) g.rot[p][k] = (Real)m.rot[a][b][k];
    }
  for (int a = 0; a < NP; ++a)
    for (int b = 0; b < NP; ++b)
      g.cw[a][b] = (Real)(m.potential == 1 ? 16.0 * m.gamma[a][b] / (PI * PI) : 18.0 * m.gamma[a][b]);
  for (int a = 0; a < NP; ++a)
    for (int b = 0; b < NP; ++b)
      for (int e = 0; e < NP; ++e) g.g3[a][b][e] = (Real)m.g3[a][b][e];
  for (int a = 0; a < NP; ++a) {
    for (int k = 0; k < NM * NM; ++k) {
      g.chi[a][k] = (Real)m.chi[a][k];
      g.DX[a][k] = (Real)m.DX[a][k];
    }
    for (int i = 0; i < NM; ++i) {
      g.B0[a][i] = (Real)m.B0[a][i];
      g.B1[a][i] = (Real)m.B1[a][i];
      double cb = 0;
      for (int j = 0; j < NM; ++j) cb += m.chi[a][i * NM + j] * m.B1[a][j];
      g.dcT[a][i] = (Real)(cb * m.G * m.V * m.dt);
    }
    {
      // (chi^a)^-1 = Hessian of f^a; Kb = dt/dx^2 H D chi, eb = H dcT
      double Hm[9] = {0};
      const double* c = m.chi[a];
      if (NM == 1) {
        Hm[0] = 1.0 / c[0];
      } else if (NM == 2) {
        double det = c[0] * c[3] - c[1] * c[2];
        Hm[0] = c[3] / det; Hm[1] = -c[1] / det; Hm[2] = -c[2] / det; Hm[3] = c[0] / det;
      } else {
        double c00 = c[4] * c[8] - c[5] * c[7], c01 = c[5] * c[6] - c[3] * c[8];
        double c02 = c[3] * c[7] - c[4] * c[6];
        double det = c[0] * c00 + c[1] * c01 + c[2] * c02;
        Hm[0] = c00 / det; Hm[3] = c01 / det; Hm[6] = c02 / det;
        Hm[1] = (c[2] * c[7] - c[1] * c[8]) / det; Hm[4] = (c[0] * c[8] - c[2] * c[6]) / det;
        Hm[7] = (c[1] * c[6] - c[0] * c[7]) / det; Hm[2] = (c[1] * c[5] - c[2] * c[4]) / det;
        Hm[5] = (c[2] * c[3] - c[0] * c[5]) / det; Hm[8] = (c[0] * c[4] - c[1] * c[3]) / det;
      }
      const double scale = m.dt / (m.dx * m.dx);
      for (int i = 0; i < NM; ++i) {
        double e = 0;
        for (int k = 0; k < NM; ++k) {
          double cb = 0;
          for (int j = 0; j < NM; ++j) cb += m.chi[a][k * NM + j] * m.B1[a][j];
          e += Hm[i * NM + k] * cb * m.G * m.V * m.dt;
        }
        g.eb[a][i] = m.gg ? Real(0) : (Real)e;   // grain growth holds mu
        for (int j = 0; j < NM; ++j) {
          double kk = 0;
          for (int k = 0; k < NM; ++k) kk += Hm[i * NM + k] * m.DX[a][k * NM + j];
          g.Kb[a][i * NM + j] = m.gg ? Real(0) : (Real)(scale * kk);
        }
      }
    }
    g.C0[a] = (Real)m.C0[a];
    g.C1[a] = (Real)m.C1[a];
    g.C2[a] = (Real)m.C2[a];
  }
  g.tzg = (Real)(m.G * m.dx);
  g.segs = segments(m);
  g.seg_bits = bits_for(g.segs);
  g.y_bits = bits_for(m.ny);
}

// T^n - T_ref at the first cell centre along the last axis, minus G dx / 2.
inline double temp_offset(const HostModel& m, double t) {
  return m.T0 - m.T_ref - m.G * (m.z0 + m.V * t);
}

template <class Real, int NP, int NM>
void set_launch_args(StepArgs<Real, NP, NM>& g, const HostModel& m, double t, void* out, const uint8_t* codes_in,
                     uint8_t* codes_out, const LaunchGeom& lg) {
  g.out = reinterpret_cast<Real*>(out);
  g.codes_in = codes_in;
  g.codes_out = codes_out;
  g.tz0 = (Real)temp_offset(m, t);
  g.zchunk = lg.zchunk;
  g.iface = lg.iface;
  g.iface2 = lg.iface2;
  g.iface_cap = lg.iface_cap;
  g.reuse_prev = lg.reuse_prev;
  g.step = (unsigned long long)lg.step;
  g.at_list = lg.at_list;
  g.at_cap = lg.at_cap;
  g.elw = reinterpret_cast<const Real*>(lg.elw);
}

// A model that uses none of the optional paths of the cell update (rotated
// pairs, gamma_abc, phi noise, elasticity, grain growth) and in which only
// the liquid diffuses (the one-sided model: D = 0 in every other phase).
inline bool plain_model(const HostModel& m) {
  for (int a = 0; a < m.N; ++a)
    for (int b = 0; b < m.N; ++b)
      if (a != b && m.rotated[a][b]) return false;
  for (int a = 0; a + 1 < m.N; ++a)
    for (int k = 0; k < m.NM * m.NM; ++k)
      if (m.DX[a][k] != 0.0) return false;
  return !m.has_g3 && m.noise_amp == 0.0 && !m.el && !m.gg;
}

// Fused step: one kernel updates every cell.
template <int DIM, int NP, int NM, class Real, int TX, int TY>
cudaError_t launch_step(const CUtensorMap* tm, const CUtensorMap*, void* blob, const HostModel& m, double t,
                        void* out, const uint8_t* codes_in, uint8_t* codes_out, const LaunchGeom& lg,
                        cudaStream_t st) {
  using Sh = StepShape<DIM, NP, NM, Real, TX, TY>;
  auto& g = *reinterpret_cast<StepArgs<Real, NP, NM>*>(blob);
  set_launch_args(g, m, t, out, codes_in, codes_out, lg);
  auto kern = k_gp_step<DIM, NP, NM, Real, TX, TY>;
  static bool configured = false;   // attribute is per function, set once
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  kern<<<dim3(lg.tiles, lg.zchunks), Sh::NTHREADS, Sh::SMEM_BYTES, st>>>(*tm, g);
  return cudaGetLastError();
}

// Split 3-D FP32 step: the bulk streaming kernel (tm = mu-only tile map),
// then the interface kernel over the rows it listed (tmi = interface boxes).
template <int NP, int NM, int TY>
cudaError_t launch_split(const CUtensorMap* tm, const CUtensorMap* tmi, void* blob, const HostModel& m, double t,
                         void* out, const uint8_t* codes_in, uint8_t* codes_out, const LaunchGeom& lg,
                         cudaStream_t st) {
  using Ss = StreamShape<NP, NM, TY>;
  using Si = IfaceShape<NP, NM, float>;
  constexpr bool two = NP > kSparseK;   // a second launch for rows with many phases
  if (!lg.iface || !lg.iface2 || !tmi || lg.iface_blocks < 1) return cudaErrorInvalidValue;
  auto& g = *reinterpret_cast<StepArgs<float, NP, NM>*>(blob);
  set_launch_args(g, m, t, out, codes_in, codes_out, lg);
  // the interface kernel fills the anti-trapping list only when the
  // correction runs after this step (launch_at with LISTED)
  if (!m.at) g.at_list = nullptr;
  // the interface kernels in two builds: every optional path of the cell
  // update, and none of them (when the model uses none: the common case)
  const bool plain = plain_model(m);
  auto ks = k_gp_stream<NP, NM, TY>;
  auto ki = plain ? k_gp_iface<3, NP, NM, float, 0, 0> : k_gp_iface<3, NP, NM, float, 0, kFeatAll>;
  auto kf = plain ? k_gp_iface<3, NP, NM, float, two ? 1 : 0, 0>   // only launched when two
                  : k_gp_iface<3, NP, NM, float, two ? 1 : 0, kFeatAll>;
  static bool configured = false;   // attributes are per function, set once
  static int iface_per_sm[2] = {0, 0}, full_per_sm[2] = {0, 0};   // resident CTAs per SM (all, plain)
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(ks, cudaFuncAttributeMaxDynamicSharedMemorySize, Ss::SMEM_BYTES);
    for (int v = 0; v < 2 && e == cudaSuccess; ++v) {
      auto vi = v ? k_gp_iface<3, NP, NM, float, 0, 0> : k_gp_iface<3, NP, NM, float, 0, kFeatAll>;
      auto vf = v ? k_gp_iface<3, NP, NM, float, two ? 1 : 0, 0> : k_gp_iface<3, NP, NM, float, two ? 1 : 0, kFeatAll>;
      e = cudaFuncSetAttribute(vi, cudaFuncAttributeMaxDynamicSharedMemorySize, Si::SMEM_BYTES);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(vi, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&iface_per_sm[v], vi, Si::THREADS, Si::SMEM_BYTES);
      if (two && e == cudaSuccess)
        e = cudaFuncSetAttribute(vf, cudaFuncAttributeMaxDynamicSharedMemorySize, Si::SMEM_BYTES);
      if (two && e == cudaSuccess)
        e = cudaFuncSetAttribute(vf, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
      if (two && e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&full_per_sm[v], vf, Si::THREADS, Si::SMEM_BYTES);
      iface_per_sm[v] = iface_per_sm[v] < 1 ? 1 : iface_per_sm[v];
      full_per_sm[v] = full_per_sm[v] < 1 ? 1 : full_per_sm[v];
    }
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int v = plain ? 1 : 0;
  ks<<<dim3(lg.tiles, lg.zchunks), Ss::NTHREADS, Ss::SMEM_BYTES, st>>>(*tm, g);
  ki<<<lg.iface_blocks * iface_per_sm[v], Si::THREADS, Si::SMEM_BYTES, st>>>(*tmi, g);
  if constexpr (two) kf<<<lg.iface_blocks * full_per_sm[v], Si::THREADS, Si::SMEM_BYTES, st>>>(*tmi, g);
  return cudaGetLastError();
}

// The anti-trapping correction after a step.  LISTED: the step's interface
// kernel has already listed the segments (split step), so the listing pass
// is skipped.
template <int DIM, int NP, int NM, class Real, bool LISTED = false>
cudaError_t launch_at(const void* in, void* blob, const HostModel& m, double t, void* out, const uint8_t* codes_in,
                      uint8_t* codes_out, const LaunchGeom& lg, cudaStream_t st) {
  using Sh = AtShape<DIM, NP, NM, Real>;
  if (!lg.at_list || lg.sms < 1) return cudaErrorInvalidValue;
  auto& g = *reinterpret_cast<StepArgs<Real, NP, NM>*>(blob);
  set_launch_args(g, m, t, out, codes_in, codes_out, lg);
  auto kw = k_at_work<DIM, NP, NM, Real>;
  static bool configured = false;   // attributes are per function, set once
  static int per_sm = 1;            // resident CTAs per SM
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kw, cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM_BYTES);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kw, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kw, Sh::THREADS, Sh::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    per_sm = per_sm < 1 ? 1 : per_sm;
    configured = true;
  }
  if constexpr (!LISTED) {
    const long long nseg = (long long)segments(m) * m.ny * (DIM == 3 ? m.nz : 1);
    k_at_list<DIM, NP, NM, Real><<<(int)((nseg + 255) / 256), 256, 0, st>>>(g);
  }
  kw<<<lg.sms * per_sm, Sh::THREADS, Sh::SMEM_BYTES, st>>>(g, reinterpret_cast<const Real*>(in));
  return cudaGetLastError();
}

template <int DIM, int NP, class Real>
cudaError_t launch_codes(const void* state, const HostModel& m, uint8_t* codes, cudaStream_t st) {
  const long long warps = (long long)segments(m) * m.ny * m.nz;   // interior planes
  const int blocks = (int)((warps * 32 + 255) / 256);
  k_codes<DIM, NP, Real><<<blocks, 256, 0, st>>>(reinterpret_cast<const Real*>(state), m.nx, m.ny, m.nz,
                                                 m.pitch, m.nyp, m.fstride, m.xoff, m.zoff, segments(m),
                                                 codes);
  return cudaGetLastError();
}

template <int DIM, int NP, int NM, class Real, int TX, int TY>
StepKernel make_step_kernel() {
  StepKernel k;
  k.dim = DIM;
  k.np = NP;
  k.nm = NM;
  k.dtype = sizeof(Real) == 8 ? 1 : 0;
  k.tx = TX;
  k.ty = TY;
  k.split = 0;
  k.smem_bytes = StepShape<DIM, NP, NM, Real, TX, TY>::SMEM_BYTES;
  k.args_bytes = sizeof(StepArgs<Real, NP, NM>);
  k.fill = &fill_args<DIM, NP, NM, Real>;
  k.launch = &launch_step<DIM, NP, NM, Real, TX, TY>;
  k.codes = &launch_codes<DIM, NP, Real>;
  k.at = &launch_at<DIM, NP, NM, Real>;
  return k;
}

// Split 3-D FP32 variant; tiles are StreamShape::TX x TY cells.
template <int NP, int NM, int TY>
StepKernel make_split_kernel() {
  StepKernel k;
  k.dim = 3;
  k.np = NP;
  k.nm = NM;
  k.dtype = 0;
  k.tx = StreamShape<NP, NM, TY>::TX;
  k.ty = TY;
  k.split = 1;
  k.smem_bytes = StreamShape<NP, NM, TY>::SMEM_BYTES;
  k.args_bytes = sizeof(StepArgs<float, NP, NM>);
  k.fill = &fill_args<3, NP, NM, float>;
  k.launch = &launch_split<NP, NM, TY>;
  k.codes = &launch_codes<3, NP, float>;
  k.at = &launch_at<3, NP, NM, float, true>;
  return k;
}

template <int DIM, int NP, int NM, class Real>
DiagKernel make_diag_kernel() {
  DiagKernel k;
  k.dim = DIM;
  k.np = NP;
  k.nm = NM;
  k.dtype = sizeof(Real) == 8 ? 1 : 0;
  k.launch = &launch_diag<DIM, NP, NM, Real>;
  return k;
}

}  // namespace msgb
