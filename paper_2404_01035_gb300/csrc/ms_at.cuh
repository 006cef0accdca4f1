// Anti-trapping current in the mu update (MICROSIM paper, arXiv 2404.01035,
// Sec. 2.1, Eq. jatr and the obstacle / well forms of j^{at,alpha} below it):
// j_at = sum_{alpha < liquid} A_alpha (c^alpha - c^liq) d phi_alpha/dt
// n_alpha (-n_alpha . n_liq), subtracted from M grad mu inside the divergence
// of Eq. (Mu_explicit_temperature).
//
// It needs d phi/dt at both cells of every face, so it runs after the step
// that wrote phi^{n+1} and mu* (the mu update without the current) into the
// output buffer: mu^{n+1} = mu* - chi(h(phi^{n+1}))^-1 dt div j_at (the update
// is linear in its right-hand side).  One warp per 32-cell row segment, one
// lane per cell; a segment whose 3 x 3 (x 3) block of segments holds one
// unchanged pure phase in both states has d phi/dt = 0 at every face of its
// cells and is left as it is.
#pragma once

#include "ms_step.cuh"

namespace msgb {

// Coefficient A of j^{at,alpha} at the face value p of phi_alpha (read as the
// 1-D equilibrium profile value there): obstacle pi eps p (1 - h(p)) /
// (4 sqrt(p (1 - p))) with the two-phase h(p) = p^2 (3 - 2p), 0 outside
// 0 < p < 1; well eps / (2 sqrt 2).
template <class Real>
__device__ __forceinline__ Real at_coefficient(int potential, Real eps, Real p) {
  if (potential != 1) return eps * Real(0.35355339059327376220);   // 1 / (2 sqrt 2)
  if (!(p > Real(0) && p < Real(1))) return Real(0);
  const Real h = p * p * (Real(3) - Real(2) * p);
  return Real(0.78539816339744830962) * eps * p * (Real(1) - h) / sqrt(p * (Real(1) - p));   // pi / 4
}

// Padded-state reads around one cell: (x, y, z) interior or ghost coordinates.
template <int DIM, class Real>
struct AtState {
  const Real* p;
  long long fstride, plane, pitch;
  int xoff, zoff;
  __device__ __forceinline__ Real at(int f, int x, int y, int z) const {
    return p[f * fstride + (long long)(DIM == 3 ? z + zoff : 0) * plane + (long long)(y + 1) * pitch + x + xoff];
  }
};

// Normal component along axis d of j_at_i at the face between (x, y, z) and
// its +d neighbour: faces values as for the gradient-energy fluxes (means of
// the two cells; normal difference and 4-point averaged tangential
// differences of phi^n), T the mean of the two cells' temperatures.
template <int DIM, int NP, int NM, class Real>
__device__ __forceinline__ void at_face(const StepArgs<Real, NP, NM>& g, const AtState<DIM, Real>& sn,
                                        const AtState<DIM, Real>& s1, int x, int y, int z, int d, Real* J) {
  constexpr int L = NP - 1;   // the liquid
  const int rx = x + (d == 0), ry = y + (d == 1), rz = z + (d == 2);
  Real pf[NP], rate[NP], nrm[NP][DIM];
  bool has_n[NP];
  const Real inv_dt = Real(1) / g.dt;
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    const Real vl = sn.at(a, x, y, z), vr = sn.at(a, rx, ry, rz);
    pf[a] = Real(0.5) * (vl + vr);
    rate[a] = Real(0.5) * ((s1.at(a, x, y, z) - vl) + (s1.at(a, rx, ry, rz) - vr)) * inv_dt;
    Real gr[DIM], g2 = Real(0);
#pragma unroll
    for (int t = 0; t < DIM; ++t) {
      if (t == d) {
        gr[t] = (vr - vl) * g.inv_dx;
      } else {
        const int ox = t == 0, oy = t == 1, oz = t == 2;
        gr[t] = ((sn.at(a, x + ox, y + oy, z + oz) + sn.at(a, rx + ox, ry + oy, rz + oz)) -
                 (sn.at(a, x - ox, y - oy, z - oz) + sn.at(a, rx - ox, ry - oy, rz - oz))) *
                g.quarter_inv_dx;
      }
      g2 += gr[t] * gr[t];
    }
    has_n[a] = g2 >= Real(1e-12);
    const Real inv = has_n[a] ? Real(1) / sqrt(g2) : Real(0);
#pragma unroll
    for (int t = 0; t < DIM; ++t) nrm[a][t] = gr[t] * inv;
  }
#pragma unroll
  for (int i = 0; i < NM; ++i) J[i] = Real(0);
  if (!has_n[L]) return;
  Real mf[NM];
#pragma unroll
  for (int i = 0; i < NM; ++i) mf[i] = Real(0.5) * (sn.at(NP + i, x, y, z) + sn.at(NP + i, rx, ry, rz));
  // T - T_ref at the two cells (lab index along the last axis, after the
  // boundary mapping) and their mean
  const int kl = DIM == 3 ? z : y, kr = DIM == 3 ? rz : ry;
  const int n = DIM == 3 ? g.nz : g.ny, bc = g.bc[DIM - 1];
  const int kml = bc_map(kl, n, bc), kmr = bc_map(kr, n, bc);
  const Real sf = g.tz0 + g.tzg * (Real(0.5) * Real(kml + kmr) + Real(g.zorg) + Real(0.5));
  Real cl[NM];
#pragma unroll
  for (int i = 0; i < NM; ++i) {
    Real c = Real(0);
#pragma unroll
    for (int j = 0; j < NM; ++j) c += g.chi[L][i * NM + j] * (mf[j] - (g.B0[L][j] + g.B1[L][j] * sf));
    cl[i] = c;
  }
#pragma unroll
  for (int al = 0; al < L; ++al) {
    if (!has_n[al]) continue;
    Real proj = Real(0);   // -n_alpha . n_liq
#pragma unroll
    for (int t = 0; t < DIM; ++t) proj -= nrm[al][t] * nrm[L][t];
    const Real k = at_coefficient<Real>(g.potential, g.eps, pf[al]) * rate[al] * nrm[al][d] * proj;
#pragma unroll
    for (int i = 0; i < NM; ++i) {
      Real c = Real(0);
#pragma unroll
      for (int j = 0; j < NM; ++j) c += g.chi[al][i * NM + j] * (mf[j] - (g.B0[al][j] + g.B1[al][j] * sf));
      J[i] += k * (c - cl[i]);
    }
  }
}

template <int DIM, int NP, int NM, class Real>
__global__ void __launch_bounds__(256) k_at(const __grid_constant__ StepArgs<Real, NP, NM> g,
                                            const Real* __restrict__ in) {
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int nzi = DIM == 3 ? g.nz : 1;
  if (w >= (long long)g.segs * g.ny * nzi) return;   // whole warps
  const int s = (int)(w % g.segs);
  const int y = (int)((w / g.segs) % g.ny);
  const int z = (int)(w / ((long long)g.segs * g.ny));
  // the segment block: unchanged and pure in one phase in both states?
  {
    constexpr int NB = DIM == 3 ? 27 : 9;
    const int c0 = load_code_from(g.codes_in, g, s, y, z) & kCodePhase;
    bool same = true;
    if (lane < NB) {
      const int ds = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = DIM == 3 ? lane / 9 - 1 : 0;
      const int ci = load_code_from(g.codes_in, g, s + ds, y + dy, z + dz) & kCodePhase;
      const int co = load_code_from(g.codes_out, g, s + ds, y + dy, z + dz) & kCodePhase;
      same = c0 != 0 && ci == c0 && co == c0;
    }
    if (__all_sync(0xffffffffu, same)) return;
  }
  const int x = 32 * s + lane;
  if (x >= g.nx) return;
  AtState<DIM, Real> sn{in, g.fstride, (long long)g.nyp * g.pitch, g.pitch, g.xoff, g.zoff};
  AtState<DIM, Real> s1{g.out, g.fstride, (long long)g.nyp * g.pitch, g.pitch, g.xoff, g.zoff};
  Real div[NM];
#pragma unroll
  for (int i = 0; i < NM; ++i) div[i] = Real(0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    Real Jp[NM], Jm[NM];
    at_face<DIM, NP, NM, Real>(g, sn, s1, x, y, z, d, Jp);
    at_face<DIM, NP, NM, Real>(g, sn, s1, x - (d == 0), y - (d == 1), z - (d == 2), d, Jm);
#pragma unroll
    for (int i = 0; i < NM; ++i) div[i] += (Jp[i] - Jm[i]) * g.inv_dx;
  }
  // mu^{n+1} = mu* + chi(h(phi^{n+1}))^-1 (-dt div j_at)
  Real pn[NP], h[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) pn[a] = s1.at(a, x, y, z);
  interp_h<NP>(pn, h);
  Real chi[NM * NM], rhs[NM], dmu[NM], mn[NM];
#pragma unroll
  for (int k = 0; k < NM * NM; ++k) {
    chi[k] = h[0] * g.chi[0][k];
#pragma unroll
    for (int a = 1; a < NP; ++a) chi[k] += h[a] * g.chi[a][k];
  }
#pragma unroll
  for (int i = 0; i < NM; ++i) rhs[i] = -g.dt * div[i];
  solve_small<NM>(chi, rhs, dmu);
#pragma unroll
  for (int i = 0; i < NM; ++i) mn[i] = s1.at(NP + i, x, y, z) + dmu[i];
  store_cell<DIM>(g, x, y, z, pn, mn, false);
}

}  // namespace msgb
