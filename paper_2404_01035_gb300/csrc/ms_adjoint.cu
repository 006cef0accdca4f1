// Discrete adjoint of the explicit grand-potential step (reverse mode over
// time, checkpointed), plus the snapshot bookkeeping it needs.
//
// One reverse step maps lambda^{n+1} = dL/d(phi^{n+1}, mu^{n+1}) to
// lambda^n = J_n^T lambda^{n+1}, J_n the Jacobian of the step at state n, and
// adds lambda^{n+1} . d(step)/d(theta) to the parameter gradients, theta =
// (delta_ab per pair, phase mobility 1/tau, D^a entries).
//
// The step of cell i is a stencil part -- the face-flux divergence divJ_i,
// the centre term Gc_i, the mu flux divergence div_i -- followed by a tail
// that is local to the cell (potential, driving force, rate, projection, mu
// update).  The reverse step runs in three passes, none with atomics (the
// result is deterministic):
//   1. k_adj_cell, per cell i: the tail once in forward mode with one
//      derivative slot per tail input (phi_i, mu_i, divJ_i, Gc_i, div_i,
//      1/tau), contracted with lambda_i: the adjoints of those inputs.  The
//      centre term's Jacobian in phi_i and in the central differences it
//      reads turns the Gc_i adjoint into adjoints of those differences.  The
//      stencil parts carry slots on delta (divJ, Gc) and on D (div), so the
//      cell's parameter gradient follows at once.
//   2. k_adj_faces, per face: the flux adjoint (adj divJ(L) - adj divJ(R)) / dx
//      of the two cells it separates, through the face flux differentiated in
//      its face values and face gradients, gives one adjoint per place in the
//      face's stencil (L, R, and the tangential neighbours).
//   3. k_adj_gather, per input cell j: lambda_j^n is the direct part plus, for
//      j and each ghost image of it, the face records and the central
//      differences that read the position, and the transposed mu flux
//      (written out by hand: div is linear in mu and in the cell mobilities,
//      chained through M(phi_j) once).
// Parameter partials are reduced per block in FP64, summed over the reverse
// steps in place and over the blocks in a fixed order at the end.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/microsim_gb.h"
#include "ms_launch.cuh"
#include "ms_rt.h"
#include "ms_trace.h"

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

// Tail inputs of one cell, in the order of the derivative slots of pass 1.
template <int NP, int NM>
struct TailSlots {
  static constexpr int PH = 0, MC = NP, DJ = NP + NM, GC = 2 * NP + NM, DIV = 3 * NP + NM;
  static constexpr int MOB = 3 * NP + 2 * NM;   // the mobility slot
  static constexpr int T = MOB + 1;
};

// Per-cell adjoints stored by pass 1 for the later passes: the cell's own phi
// (tail and centre term) and mu, divJ (for the face fluxes), the unscaled
// central differences gcr[a][d] of the centre term, and div.
template <int DIM, int NP, int NM>
struct CellStore {
  static constexpr int PH = 0, MC = NP, DJ = NP + NM, GCR = 2 * NP + NM, DIV = GCR + NP * DIM;
  static constexpr int TB = DIV + NM;
};

// Per-face adjoints of pass 2: the face's phases at its lower cell L and
// upper cell R, and the tangential gradient of each phase along each axis t
// != D (applied with +- 1/(4 dx) to L +- e_t and R +- e_t).
template <int DIM, int NP>
struct FaceStore {
  static constexpr int AL = 0, AR = NP, TG = 2 * NP;   // TG + a (DIM - 1) + tt
  static constexpr int N = NP * (DIM + 1);
};

// Faces along axis D, indexed by their lower cell L, whose coordinate along D
// runs over -1 .. n_D - 1 (shifted by one).
template <int DIM, int D, class Real, int NP, int NM>
__device__ __forceinline__ long long face_id(const StepArgs<Real, NP, NM>& g, int lx, int ly, int lz) {
  const long long ex = g.nx + (D == 0), ey = g.ny + (D == 1);
  return ((long long)(lz + (D == 2)) * ey + (ly + (D == 1))) * ex + (lx + (D == 0));
}

inline long long faces_along(const HostModel& m, int D) {
  return (long long)(m.nx + (D == 0)) * (m.ny + (D == 1)) * (m.nz + (D == 2));
}

// Stencil accessor yielding plain values as the scalar S (no derivative).
template <int NP, int NM, class Real, class S>
struct ValAcc {
  const Real* st;
  long long fstride, plane, base;
  int pitch;
  __device__ __forceinline__ S ld(int f, int dx, int dy, int dz) const {
    return S(st[f * fstride + base + dz * plane + (long long)dy * pitch + dx]);
  }
  __device__ __forceinline__ S phi(int a, int dx, int dy, int dz) const { return ld(a, dx, dy, dz); }
  __device__ __forceinline__ S mu(int i, int dx, int dy, int dz) const { return ld(NP + i, dx, dy, dz); }
  __device__ __forceinline__ uint32_t mask() const { return (1u << NP) - 1u; }
};

// Stencil accessor yielding phases as Dual<Real, NP> with slot a = 1 for
// phase a at the padded index `seed`.
template <int NP, int NM, class Real>
struct SeedAcc {
  using D = Dual<Real, NP>;
  const Real* st;
  long long fstride, plane, base, seed;
  int pitch;
  __device__ __forceinline__ D phi(int a, int dx, int dy, int dz) const {
    const long long idx = base + dz * plane + (long long)dy * pitch + dx;
    D v(st[a * fstride + idx]);
    if (idx == seed) v.d[a] = Real(1);
    return v;
  }
  __device__ __forceinline__ uint32_t mask() const { return (1u << NP) - 1u; }
};

template <int DIM, class Real, int NP, int NM>
__device__ __forceinline__ bool in_grid(const StepArgs<Real, NP, NM>& g, int x, int y, int z) {
  return x >= 0 && x < g.nx && y >= 0 && y < g.ny && z >= 0 && z < (DIM == 3 ? g.nz : 1);
}

template <int DIM, class Real, int NP, int NM>
__device__ __forceinline__ long long padded_index(const StepArgs<Real, NP, NM>& g, int x, int y, int z) {
  return (long long)(z + g.zoff) * ((long long)g.nyp * g.pitch) + (long long)(y + 1) * g.pitch + x + g.xoff;
}

template <int DIM>
__device__ __forceinline__ bool any_aniso(const unsigned char* aniso, int P) {
  bool r = false;
  for (int p = 0; p < P; ++p) r = r || aniso[p] != 0;
  return r;
}

// Pass 1 (see the file comment).  tbar: [TB][cells], dense cell order.
template <int DIM, int NP, int NM, class Real>
__global__ void __launch_bounds__(128) k_adj_cell(const Real* __restrict__ st, const Real* __restrict__ lam_in,
                                                  Real* __restrict__ tbar,
                                                  const __grid_constant__ StepArgs<Real, NP, NM> g,
                                                  const __grid_constant__ AdjExtra<Real, NP, NM> ex,
                                                  double* __restrict__ partials) {
  constexpr int P = NP * (NP - 1) / 2;
  constexpr int ND = NP * NM * NM;
  constexpr int NPRM = ParamCount<NP, NM>::value;
  using TS = TailSlots<NP, NM>;
  using DP = Dual<Real, P>;
  using DD = Dual<Real, ND>;
  using DT = Dual<Real, TS::T>;
  const long long cells = (long long)g.nx * g.ny * g.nz;
  const long long plane = (long long)g.nyp * g.pitch;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double gpar[NPRM];
#pragma unroll
  for (int k = 0; k < NPRM; ++k) gpar[k] = 0.0;
  if (i < cells) {
    const int x = (int)(i % g.nx), y = (int)((i / g.nx) % g.ny), z = (int)(i / ((long long)g.nx * g.ny));
    const long long base = padded_index<DIM>(g, x, y, z);
    // stencil part: divJ, Gc with delta slots
    DP divJ[NP], Gc[NP];
    {
      ValAcc<NP, NM, Real, DP> A{st, g.fstride, plane, base, g.pitch};
      DiffPrm<DP, P> dp;
      dp.mob = DP(g.mob);
#pragma unroll
      for (int p = 0; p < P; ++p) {
        dp.delta[p] = DP(g.delta[p]);
        dp.delta[p].d[p] = Real(1);
      }
      DP ph[NP];
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        ph[a] = A.phi(a, 0, 0, 0);
        divJ[a] = DP(Real(0));
        Gc[a] = DP(Real(0));
      }
      gradient_terms<DIM, NP, NM, Real, DP, ValAcc<NP, NM, Real, DP>, kFeatAll, false>(
          A, g, dp, ph, A.mask(), any_aniso<DIM>(g.aniso, P), divJ, Gc);
    }
    // stencil part: div with D slots (M = sum_a h_a D^a chi^a)
    DD div[NM];
    {
      ValAcc<NP, NM, Real, DD> B{st, g.fstride, plane, base, g.pitch};
      DD DXd[NP][NM * NM];
#pragma unroll
      for (int a = 0; a < NP; ++a)
#pragma unroll
        for (int r = 0; r < NM; ++r)
#pragma unroll
          for (int c = 0; c < NM; ++c) {
            DD sum(Real(0));
#pragma unroll
            for (int m = 0; m < NM; ++m) {
              DD Dm(ex.D[a][r * NM + m]);
              Dm.d[(a * NM + r) * NM + m] = Real(1);
              sum += Dm * DD(g.chi[a][m * NM + c]);
            }
            DXd[a][r * NM + c] = sum;
          }
      DD ph[NP], mc[NM], Mc[NM * NM];
#pragma unroll
      for (int a = 0; a < NP; ++a) ph[a] = B.phi(a, 0, 0, 0);
#pragma unroll
      for (int k = 0; k < NM; ++k) {
        mc[k] = B.mu(k, 0, 0, 0);
        div[k] = DD(Real(0));
      }
      cell_mobility<NP, NM>(ph, DXd, Mc);
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
#pragma unroll
        for (int sd = -1; sd <= 1; sd += 2) {
          const Off<DIM> o = unit<DIM>(d, sd);
          DD pn[NP], Mn[NM * NM];
#pragma unroll
          for (int a = 0; a < NP; ++a) pn[a] = B.phi(a, o.x, o.y, o.z);
          cell_mobility<NP, NM>(pn, DXd, Mn);
#pragma unroll
          for (int r = 0; r < NM; ++r)
#pragma unroll
            for (int c = 0; c < NM; ++c) {
              DD Mf = Real(0.5) * (Mc[r * NM + c] + Mn[r * NM + c]);
              div[r] += Mf * ((B.mu(c, o.x, o.y, o.z) - mc[c]) * g.inv_dx2);
            }
        }
      }
    }
    // the tail, one slot per input
    Real tb[TS::T];
    {
      DT in[TS::T];
#pragma unroll
      for (int k = 0; k < TS::T; ++k) in[k] = DT(Real(0));
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        in[TS::PH + a] = DT(st[a * g.fstride + base]);
        in[TS::DJ + a] = DT(divJ[a].v);
        in[TS::GC + a] = DT(Gc[a].v);
      }
#pragma unroll
      for (int k = 0; k < NM; ++k) {
        in[TS::MC + k] = DT(st[(NP + k) * g.fstride + base]);
        in[TS::DIV + k] = DT(div[k].v);
      }
      in[TS::MOB] = DT(g.mob);
#pragma unroll
      for (int k = 0; k < TS::T; ++k) in[k].d[k] = Real(1);
      DiffPrm<DT, P> dp;
      dp.mob = in[TS::MOB];
#pragma unroll
      for (int p = 0; p < P; ++p) dp.delta[p] = DT(g.delta[p]);
      const int kz = (DIM == 3 ? z : y) + g.zorg;
      const Real s = g.tz0 + g.tzg * (Real(kz) + Real(0.5));
      DT pn[NP], mn[NM];
      phase_update<DIM, NP, NM, Real, DT, kFeatAll>(g, dp, in + TS::PH, in + TS::MC, in + TS::DJ, in + TS::GC, s,
                                                    lab_cell<DIM>(g, x, y, z), pn);
      mu_update<NP, NM, Real, DT>(g, in + TS::PH, pn, in + TS::MC, in + TS::DIV, s, false, mn);
#pragma unroll
      for (int k = 0; k < TS::T; ++k) tb[k] = Real(0);
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        const Real l = lam_in[a * cells + i];
#pragma unroll
        for (int k = 0; k < TS::T; ++k) tb[k] += l * pn[a].d[k];
      }
#pragma unroll
      for (int m = 0; m < NM; ++m) {
        const Real l = lam_in[(NP + m) * cells + i];
#pragma unroll
        for (int k = 0; k < TS::T; ++k) tb[k] += l * mn[m].d[k];
      }
    }
    // centre term transposed: slots on the cell's phi and the unscaled
    // central differences gcr[a][d] it reads
    {
      using CS = CellStore<DIM, NP, NM>;
      constexpr int WC = NP * (1 + DIM);
      using DC = Dual<Real, WC>;
      ValAcc<NP, NM, Real, Real> V{st, g.fstride, plane, base, g.pitch};
      DiffPrm<DC, P> dp;
      dp.mob = DC(g.mob);
#pragma unroll
      for (int p = 0; p < P; ++p) dp.delta[p] = DC(g.delta[p]);
      DC ph[NP], gcr[NP][DIM], Gcd[NP];
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        ph[a] = DC(V.phi(a, 0, 0, 0));
        ph[a].d[a] = Real(1);
        gcr[a][0] = DC(V.phi(a, 1, 0, 0) - V.phi(a, -1, 0, 0));
        gcr[a][1] = DC(V.phi(a, 0, 1, 0) - V.phi(a, 0, -1, 0));
        if constexpr (DIM == 3) gcr[a][2] = DC(V.phi(a, 0, 0, 1) - V.phi(a, 0, 0, -1));
#pragma unroll
        for (int d = 0; d < DIM; ++d) gcr[a][d].d[NP + a * DIM + d] = Real(1);
        Gcd[a] = DC(Real(0));
      }
      centre_term<DIM, NP, NM, Real, DC, kFeatAll, false>(g, dp, ph, gcr, V.mask(), Gcd);
      Real sb[WC];
#pragma unroll
      for (int k = 0; k < WC; ++k) sb[k] = Real(0);
#pragma unroll
      for (int a = 0; a < NP; ++a)
#pragma unroll
        for (int k = 0; k < WC; ++k) sb[k] += tb[TS::GC + a] * Gcd[a].d[k];
#pragma unroll
      for (int a = 0; a < NP; ++a) tbar[(CS::PH + a) * cells + i] = tb[TS::PH + a] + sb[a];
#pragma unroll
      for (int k = 0; k < NM; ++k) {
        tbar[(CS::MC + k) * cells + i] = tb[TS::MC + k];
        tbar[(CS::DIV + k) * cells + i] = tb[TS::DIV + k];
      }
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        tbar[(CS::DJ + a) * cells + i] = tb[TS::DJ + a];
#pragma unroll
        for (int d = 0; d < DIM; ++d) tbar[(CS::GCR + a * DIM + d) * cells + i] = sb[NP + a * DIM + d];
      }
    }
    // parameter gradient of cell i's update
#pragma unroll
    for (int p = 0; p < P; ++p) {
      Real sp = Real(0);
#pragma unroll
      for (int a = 0; a < NP; ++a) sp += tb[TS::DJ + a] * divJ[a].d[p] + tb[TS::GC + a] * Gc[a].d[p];
      gpar[p] += (double)sp;
    }
    gpar[P] += (double)tb[TS::MOB];
#pragma unroll
    for (int k = 0; k < ND; ++k) {
      Real sd = Real(0);
#pragma unroll
      for (int m = 0; m < NM; ++m) sd += tb[TS::DIV + m] * div[m].d[k];
      gpar[P + 1 + k] += (double)sd;
    }
  }
  if (partials) {
    // per warp by a fixed shuffle tree, then the 4 warps in order
    __shared__ double red[4][NPRM];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NPRM; ++k) {
      double v = gpar[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) red[w][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < NPRM) {
      const int k = threadIdx.x;
      partials[blockIdx.x * NPRM + k] += ((red[0][k] + red[1][k]) + red[2][k]) + red[3][k];   // summed over the reverse steps
    }
  }
}

// Face fluxes along axis D whose stencil contains position (px, py, pz):
// acc[a'] += sum_a Jbar_f[a] dJ_f[a]/dphi_a'(p).  A face is named by its
// lower cell L (upper R = L + e_D); its stencil is L, R and, with
// anisotropy, L +- e_t, R +- e_t for t != D.
template <int DIM, int D, int NP, int NM, class Real>
__device__ __forceinline__ void gather_faces(const Real* __restrict__ st, const Real* __restrict__ tbar,
                                             const StepArgs<Real, NP, NM>& g, bool need_tan, int px, int py, int pz,
                                             long long seed, Real* acc) {
  constexpr int P = NP * (NP - 1) / 2;
  using TS = TailSlots<NP, NM>;
  using DN = Dual<Real, NP>;
  const long long cells = (long long)g.nx * g.ny * g.nz;
  const long long plane = (long long)g.nyp * g.pitch;
  DiffPrm<DN, P> dp;
  dp.mob = DN(g.mob);
#pragma unroll
  for (int p = 0; p < P; ++p) dp.delta[p] = DN(g.delta[p]);
  const int ncand = 2 + (need_tan ? 4 * (DIM - 1) : 0);
#pragma unroll 1
  for (int c = 0; c < ncand; ++c) {
    // offset of L from p
    int o[3] = {0, 0, 0};
    if (c == 0) {
      o[D] = -1;   // p is R
    } else if (c > 1) {
      const int k = c - 2;
      const int t = DIM == 2 ? 1 - D : (D + 1 + (k >> 2)) % 3;   // a tangential axis of D
      const int sgn = (k & 1) ? 1 : -1;
      o[t] = -sgn;                  // p = L + sgn e_t, or
      if ((k >> 1) & 1) o[D] = -1;  // p = R + sgn e_t
    }
    const int lx = px + o[0], ly = py + o[1], lz = pz + o[2];
    const int rx = lx + (D == 0), ry = ly + (D == 1), rz = lz + (D == 2);
    const bool inL = in_grid<DIM>(g, lx, ly, lz), inR = in_grid<DIM>(g, rx, ry, rz);
    if (!inL && !inR) continue;
    Real Jbar[NP];
    const long long li = ((long long)lz * g.ny + ly) * g.nx + lx, ri = ((long long)rz * g.ny + ry) * g.nx + rx;
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      const Real bl = inL ? tbar[(TS::DJ + a) * cells + li] : Real(0);
      const Real br = inR ? tbar[(TS::DJ + a) * cells + ri] : Real(0);
      Jbar[a] = (bl - br) * g.inv_dx;
    }
    SeedAcc<NP, NM, Real> A{st, g.fstride, plane, padded_index<DIM>(g, lx, ly, lz), seed, g.pitch};
    DN J[NP];
    face_flux<DIM, D, NP, NM, Real, DN, SeedAcc<NP, NM, Real>, kFeatAll>(A, g, dp, A.mask(), 1, need_tan, J);
#pragma unroll
    for (int a = 0; a < NP; ++a)
#pragma unroll
      for (int b = 0; b < NP; ++b) acc[b] += Jbar[a] * J[a].d[b];
  }
}

// Pass 2 for the faces along axis D of one cell i: the face with lower cell
// L = i and, at the lower domain end, the face with L = i - e_D.  The flux
// adjoint is Jbar = (tbar_divJ(L) - tbar_divJ(R)) / dx over the cells of the
// grid among L, R; the face flux is differentiated in forward mode with one
// slot per face value pf_a and face gradient component gr_a,d, and the result
// is written per stencil position class (FaceStore).
template <int DIM, int D, int NP, int NM, class Real>
__device__ __forceinline__ void face_adjoint(const Real* __restrict__ st, const Real* __restrict__ tbar,
                                             Real* __restrict__ frec, const StepArgs<Real, NP, NM>& g,
                                             bool need_tan, int lx, int ly, int lz) {
  constexpr int P = NP * (NP - 1) / 2;
  constexpr int W = NP * (1 + DIM);
  using CS = CellStore<DIM, NP, NM>;
  using FS = FaceStore<DIM, NP>;
  using DW = Dual<Real, W>;
  const long long cells = (long long)g.nx * g.ny * g.nz;
  const long long plane = (long long)g.nyp * g.pitch;
  const int rx = lx + (D == 0), ry = ly + (D == 1), rz = lz + (D == 2);
  const bool inL = in_grid<DIM>(g, lx, ly, lz), inR = in_grid<DIM>(g, rx, ry, rz);
  const long long li = ((long long)lz * g.ny + ly) * g.nx + lx, ri = ((long long)rz * g.ny + ry) * g.nx + rx;
  Real Jbar[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    const Real bl = inL ? tbar[(CS::DJ + a) * cells + li] : Real(0);
    const Real br = inR ? tbar[(CS::DJ + a) * cells + ri] : Real(0);
    Jbar[a] = (bl - br) * g.inv_dx;
  }
  ValAcc<NP, NM, Real, Real> V{st, g.fstride, plane, padded_index<DIM>(g, lx, ly, lz), g.pitch};
  DW pf[NP], gr[NP][DIM];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    const Real vl = V.phi(a, 0, 0, 0);
    const Real vr = V.phi(a, D == 0, D == 1, D == 2);
    pf[a] = DW(Real(0.5) * (vl + vr));
    pf[a].d[a] = Real(1);
    gr[a][D] = DW((vr - vl) * g.inv_dx);
#pragma unroll
    for (int t = 0; t < DIM; ++t) {
      if (t == D) continue;
      Real v = Real(0);
      if (need_tan) {
        const int ux = t == 0, uy = t == 1, uz = t == 2;
        const int rdx = D == 0, rdy = D == 1, rdz = D == 2;
        v = ((V.phi(a, ux, uy, uz) + V.phi(a, rdx + ux, rdy + uy, rdz + uz)) -
             (V.phi(a, -ux, -uy, -uz) + V.phi(a, rdx - ux, rdy - uy, rdz - uz))) *
            g.quarter_inv_dx;
      }
      gr[a][t] = DW(v);
    }
#pragma unroll
    for (int d = 0; d < DIM; ++d) gr[a][d].d[NP + a * DIM + d] = Real(1);
  }
  DiffPrm<DW, P> dp;
  dp.mob = DW(g.mob);
#pragma unroll
  for (int p = 0; p < P; ++p) dp.delta[p] = DW(g.delta[p]);
  DW J[NP];
  face_flux_from<DIM, D, NP, NM, Real, DW, kFeatAll>(g, dp, (1u << NP) - 1u, pf, gr, J);
  Real sb[W];
#pragma unroll
  for (int k = 0; k < W; ++k) sb[k] = Real(0);
#pragma unroll
  for (int a = 0; a < NP; ++a)
#pragma unroll
    for (int k = 0; k < W; ++k) sb[k] += Jbar[a] * J[a].d[k];
  const long long fid = face_id<DIM, D>(g, lx, ly, lz);
  const long long nfaces = (long long)(g.nx + (D == 0)) * (g.ny + (D == 1)) * ((DIM == 3 ? g.nz : 1) + (D == 2));
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    const Real gn = sb[NP + a * DIM + D] * g.inv_dx;
    frec[(FS::AL + a) * nfaces + fid] = Real(0.5) * sb[a] - gn;
    frec[(FS::AR + a) * nfaces + fid] = Real(0.5) * sb[a] + gn;
    int tt = 0;
#pragma unroll
    for (int t = 0; t < DIM; ++t) {
      if (t == D) continue;
      frec[(FS::TG + a * (DIM - 1) + tt) * nfaces + fid] = sb[NP + a * DIM + t] * g.quarter_inv_dx;
      ++tt;
    }
  }
}

template <int DIM, int NP, int NM, class Real>
__global__ void __launch_bounds__(128) k_adj_faces(const Real* __restrict__ st, const Real* __restrict__ tbar,
                                                   Real* __restrict__ frec0, Real* __restrict__ frec1,
                                                   Real* __restrict__ frec2,
                                                   const __grid_constant__ StepArgs<Real, NP, NM> g) {
  constexpr int P = NP * (NP - 1) / 2;
  const long long cells = (long long)g.nx * g.ny * g.nz;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= cells) return;
  const int x = (int)(i % g.nx), y = (int)((i / g.nx) % g.ny), z = (int)(i / ((long long)g.nx * g.ny));
  const bool need_tan = any_aniso<DIM>(g.aniso, P);
  face_adjoint<DIM, 0, NP, NM, Real>(st, tbar, frec0, g, need_tan, x, y, z);
  if (x == 0) face_adjoint<DIM, 0, NP, NM, Real>(st, tbar, frec0, g, need_tan, -1, y, z);
  face_adjoint<DIM, 1, NP, NM, Real>(st, tbar, frec1, g, need_tan, x, y, z);
  if (y == 0) face_adjoint<DIM, 1, NP, NM, Real>(st, tbar, frec1, g, need_tan, x, -1, z);
  if constexpr (DIM == 3) {
    face_adjoint<DIM, 2, NP, NM, Real>(st, tbar, frec2, g, need_tan, x, y, z);
    if (z == 0) face_adjoint<DIM, 2, NP, NM, Real>(st, tbar, frec2, g, need_tan, x, y, -1);
  }
}

// Face records along axis D read by position (px, py, pz): acc[a] += the
// record's entry for the position's place in the face's stencil.
template <int DIM, int D, int NP, int NM, class Real>
__device__ __forceinline__ void gather_faces(const Real* __restrict__ frec, const StepArgs<Real, NP, NM>& g,
                                             bool need_tan, int px, int py, int pz, Real* acc) {
  using FS = FaceStore<DIM, NP>;
  const long long nfaces = (long long)(g.nx + (D == 0)) * (g.ny + (D == 1)) * ((DIM == 3 ? g.nz : 1) + (D == 2));
  // (unrolled: every candidate's loads can be in flight at once)
#pragma unroll
  for (int c = 0; c < 2 + 4 * (DIM - 1); ++c) {
    if (c >= 2 && !need_tan) continue;
    int o[3] = {0, 0, 0};
    int slot, sgn = 1;
    if (c == 0) {
      o[D] = -1;   // p is R
      slot = FS::AR;
    } else if (c == 1) {
      slot = FS::AL;   // p is L
    } else {
      const int k = c - 2;
      const int t = DIM == 2 ? 1 - D : (D + 1 + (k >> 2)) % 3;   // a tangential axis of D
      const int tt = t > D ? t - 1 : t;                          // its rank among the axes != D
      sgn = (k & 1) ? 1 : -1;
      o[t] = -sgn;                  // p = L + sgn e_t, or
      if ((k >> 1) & 1) o[D] = -1;  // p = R + sgn e_t
      slot = FS::TG + tt;           // + a (DIM - 1) below
    }
    const int lx = px + o[0], ly = py + o[1], lz = pz + o[2];
    if (!in_grid<DIM>(g, lx, ly, lz) && !in_grid<DIM>(g, lx + (D == 0), ly + (D == 1), lz + (D == 2))) continue;
    const long long fid = face_id<DIM, D>(g, lx, ly, lz);
    const int astride = c < 2 ? 1 : DIM - 1;
#pragma unroll
    for (int a = 0; a < NP; ++a) acc[a] += Real(sgn) * frec[(slot + a * astride) * nfaces + fid];
  }
}

// Pass 3, per input cell j: the direct part, the face records and
// centre-term differences that read j's positions, and the mu flux.  A block
// covers 32 cells with DIM + 1 warps (the loads are latency-bound: more of
// them in flight): warp w < DIM reads the face records along axis w, warp DIM
// the rest; the parts are summed in warp order (deterministic).
template <int DIM>
struct GatherShape {
  static constexpr int PARTS = DIM + 1;
  static constexpr int THREADS = 32 * PARTS;
};

template <int DIM, int NP, int NM, class Real>
__global__ void __launch_bounds__(GatherShape<DIM>::THREADS)
    k_adj_gather(const Real* __restrict__ st, const Real* __restrict__ tbar, const Real* __restrict__ frec0,
                 const Real* __restrict__ frec1, const Real* __restrict__ frec2, Real* __restrict__ lam_out,
                 const __grid_constant__ StepArgs<Real, NP, NM> g) {
  constexpr int NF = NP + NM;
  constexpr int P = NP * (NP - 1) / 2;
  using CS = CellStore<DIM, NP, NM>;
  using DN = Dual<Real, NP>;
  __shared__ Real s_acc[DIM][NF][32];
  const int part = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long cells = (long long)g.nx * g.ny * g.nz;
  const long long plane = (long long)g.nyp * g.pitch;
  const long long j = blockIdx.x * 32ll + lane;
  const bool live = j < cells;
  Real acc[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) acc[f] = Real(0);
  if (live) {
    const int x = (int)(j % g.nx), y = (int)((j / g.nx) % g.ny), z = (int)(j / ((long long)g.nx * g.ny));
    const long long jb = padded_index<DIM>(g, x, y, z);
    auto dense = [&](int px, int py, int pz) { return ((long long)pz * g.ny + py) * g.nx + px; };
    const bool need_tan = any_aniso<DIM>(g.aniso, P);
    Real phj[NP], muj[NM], Mj[NM * NM], Mbar[NM * NM];
    if (part == DIM) {
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        acc[a] = tbar[(CS::PH + a) * cells + j];
        phj[a] = st[a * g.fstride + jb];
      }
#pragma unroll
      for (int k = 0; k < NM; ++k) {
        acc[NP + k] = tbar[(CS::MC + k) * cells + j];
        muj[k] = st[(NP + k) * g.fstride + jb];
      }
      cell_mobility<NP, NM>(phj, g.DX, Mj);
#pragma unroll
      for (int k = 0; k < NM * NM; ++k) Mbar[k] = Real(0);
    }

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
#pragma unroll 1
    for (int iz = 0; iz < nzs; ++iz)
#pragma unroll 1
      for (int iy = 0; iy < nys; ++iy)
#pragma unroll 1
        for (int ix = 0; ix < nxs; ++ix) {
          const int px = xs[ix], py = ys[iy], pz = zs[iz];
          if (part == 0) gather_faces<DIM, 0, NP, NM, Real>(frec0, g, need_tan, px, py, pz, acc);
          if (part == 1) gather_faces<DIM, 1, NP, NM, Real>(frec1, g, need_tan, px, py, pz, acc);
          if constexpr (DIM == 3)
            if (part == 2) gather_faces<DIM, 2, NP, NM, Real>(frec2, g, need_tan, px, py, pz, acc);
          if (part != DIM) continue;
          // centre terms: p = i + sgn e_d enters gcr_i[a][d] with sign sgn
#pragma unroll
          for (int c = 0; c < 2 * DIM; ++c) {
            const int d = c >> 1, sgn = (c & 1) ? 1 : -1;
            const int cx = px - (d == 0 ? sgn : 0), cy = py - (d == 1 ? sgn : 0), cz = pz - (d == 2 ? sgn : 0);
            if (!in_grid<DIM>(g, cx, cy, cz)) continue;
            const long long ci = dense(cx, cy, cz);
#pragma unroll
            for (int a = 0; a < NP; ++a) acc[a] += Real(sgn) * tbar[(CS::GCR + a * DIM + d) * cells + ci];
          }
          // mu flux of the in-grid neighbours i = p - o: p is their neighbour at o
#pragma unroll
          for (int c = 0; c < 2 * DIM; ++c) {
            const int d = c >> 1, sgn = (c & 1) ? 1 : -1;
            const int ix2 = px - (d == 0 ? sgn : 0), iy2 = py - (d == 1 ? sgn : 0), iz2 = pz - (d == 2 ? sgn : 0);
            if (!in_grid<DIM>(g, ix2, iy2, iz2)) continue;
            const long long ii = dense(ix2, iy2, iz2), ib = padded_index<DIM>(g, ix2, iy2, iz2);
            Real phi_i[NP], Mi[NM * NM];
#pragma unroll
            for (int a = 0; a < NP; ++a) phi_i[a] = st[a * g.fstride + ib];
            cell_mobility<NP, NM>(phi_i, g.DX, Mi);
#pragma unroll
            for (int r = 0; r < NM; ++r) {
              const Real db = tbar[(CS::DIV + r) * cells + ii];
#pragma unroll
              for (int q = 0; q < NM; ++q) {
                const Real mci = st[(NP + q) * g.fstride + ib];
                acc[NP + q] += db * (Real(0.5) * (Mi[r * NM + q] + Mj[r * NM + q])) * g.inv_dx2;
                Mbar[r * NM + q] += db * (Real(0.5) * (muj[q] - mci)) * g.inv_dx2;
              }
            }
          }
        }
    if (part == DIM) {
      // mu flux of cell j itself (its own mu and mobility at the centre)
      Real db[NM];
#pragma unroll
      for (int r = 0; r < NM; ++r) db[r] = tbar[(CS::DIV + r) * cells + j];
#pragma unroll
      for (int c = 0; c < 2 * DIM; ++c) {
        const int d = c >> 1, sgn = (c & 1) ? 1 : -1;
        const long long nb = jb + (d == 0 ? sgn : 0) + (d == 1 ? (long long)sgn * g.pitch : 0) +
                             (d == 2 ? (long long)sgn * plane : 0);
        Real phn[NP], Mn[NM * NM];
#pragma unroll
        for (int a = 0; a < NP; ++a) phn[a] = st[a * g.fstride + nb];
        cell_mobility<NP, NM>(phn, g.DX, Mn);
#pragma unroll
        for (int r = 0; r < NM; ++r)
#pragma unroll
          for (int q = 0; q < NM; ++q) {
            const Real mun = st[(NP + q) * g.fstride + nb];
            acc[NP + q] -= db[r] * (Real(0.5) * (Mj[r * NM + q] + Mn[r * NM + q])) * g.inv_dx2;
            Mbar[r * NM + q] += db[r] * (Real(0.5) * (mun - muj[q])) * g.inv_dx2;
          }
      }
      // M(phi_j): chain the mobility adjoint to the phases
      DN ph[NP], M[NM * NM];
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        ph[a] = DN(phj[a]);
        ph[a].d[a] = Real(1);
      }
      cell_mobility<NP, NM>(ph, g.DX, M);
#pragma unroll
      for (int k = 0; k < NM * NM; ++k)
#pragma unroll
        for (int b = 0; b < NP; ++b) acc[b] += Mbar[k] * M[k].d[b];
    }
  }
  if (part > 0) {
#pragma unroll
    for (int f = 0; f < NF; ++f) s_acc[part - 1][f][lane] = acc[f];
  }
  __syncthreads();
  if (part == 0 && live) {
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      Real v = acc[f];
#pragma unroll
      for (int q = 0; q < DIM; ++q) v += s_acc[q][f][lane];
      lam_out[f * cells + j] = v;
    }
  }
}

// gsum[k] += sum over blocks of partials[b][k]: one warp per parameter, lane
// l summing blocks l, l + 32, ... in order, then a fixed shuffle tree
// (deterministic).
__global__ void k_accumulate_params(const double* __restrict__ partials, int nblocks, int nprm,
                                    double* __restrict__ gsum) {
  const int k = blockIdx.x, lane = threadIdx.x;
  if (k >= nprm) return;
  double s = 0.0;
  for (int b = lane; b < nblocks; b += 32) s += partials[(long long)b * nprm + k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) gsum[k] += s;
}

// Size of the gradient sum buffer: an upper bound on the parameter count of
// every compiled adjoint (checked at compile time for each one).
constexpr int kMaxGradParams = 64;

struct AdjKernel {
  int dim, np, nm, dtype, nprm;
  cudaError_t (*launch)(const void* state, const void* lam_in, void* lam_out, void* tbar, const void* blob,
                        const HostModel& m, double t, double* partials, cudaStream_t st);
};

// Work buffer of the reverse step, in elements: the per-cell store of pass 1
// and the face records of pass 2 along every axis.
inline long long adjoint_work_elems(const HostModel& m) {
  const long long cells = (long long)m.nx * m.ny * m.nz;
  long long n = (long long)(2 * m.N + 2 * m.NM + m.N * m.dim) * cells;
  for (int D = 0; D < m.dim; ++D) n += (long long)m.N * (m.dim + 1) * faces_along(m, D);
  return n;
}

template <int DIM, int NP, int NM, class Real>
cudaError_t launch_adjoint(const void* state, const void* lam_in, void* lam_out, void* tbar, const void* blob,
                           const HostModel& m, double t, double* partials, cudaStream_t st) {
  StepArgs<Real, NP, NM> g = *reinterpret_cast<const StepArgs<Real, NP, NM>*>(blob);
  g.tz0 = (Real)temp_offset(m, t);
  AdjExtra<Real, NP, NM> ex;
  for (int a = 0; a < NP; ++a)
    for (int k = 0; k < NM * NM; ++k) ex.D[a][k] = (Real)m.D[a][k];
  const long long cells = (long long)m.nx * m.ny * m.nz;
  const int blocks = (int)((cells + 127) / 128);
  const Real* s = reinterpret_cast<const Real*>(state);
  k_adj_cell<DIM, NP, NM, Real><<<blocks, 128, 0, st>>>(s, reinterpret_cast<const Real*>(lam_in),
                                                        reinterpret_cast<Real*>(tbar), g, ex, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  Real* tb = reinterpret_cast<Real*>(tbar);
  Real* fr[3] = {nullptr, nullptr, nullptr};
  {
    Real* q = tb + (long long)CellStore<DIM, NP, NM>::TB * cells;
    for (int D = 0; D < DIM; ++D) {
      fr[D] = q;
      q += (long long)FaceStore<DIM, NP>::N * faces_along(m, D);
    }
  }
  k_adj_faces<DIM, NP, NM, Real><<<blocks, 128, 0, st>>>(s, tb, fr[0], fr[1], fr[2], g);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_adj_gather<DIM, NP, NM, Real><<<(unsigned)((cells + 31) / 32), GatherShape<DIM>::THREADS, 0, st>>>(
      s, tb, fr[0], fr[1], fr[2], reinterpret_cast<Real*>(lam_out), g);
  return cudaGetLastError();
}

template <int DIM, int NP, int NM, class Real>
AdjKernel make_adjoint() {
  static_assert(ParamCount<NP, NM>::value <= kMaxGradParams, "gradient scratch too small");
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
  dev_free(c->hook, a.tbar);
  a.tbar = nullptr;
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
  // the reverse step maps ghost positions back to their source cells by the
  // boundary rule; a halo face's ghosts belong to another slab
  if (every > 0 && c->m.dim == 3 && c->m.bc[2] == kBcHalo)
    return fail(c, MS_ERR_UNSUPPORTED, "the adjoint needs the whole domain (no halo faces)");
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
  TraceRange trace("ms_grad");
  if (!c || !dphi_T) return fail(c, MS_ERR_ARG, "ctx and dphi_T are required");
  AdjointStore& A = c->adj;
  if (A.every <= 0) return fail(c, MS_ERR_STATE, "checkpoints are not enabled (ms_enable_checkpoints)");
  if (c->m.noise_amp != 0.0) return fail(c, MS_ERR_UNSUPPORTED, "the adjoint does not support phi noise (noise_amp != 0)");
  if (c->m.at || c->m.gg || c->m.el)
    return fail(c, MS_ERR_UNSUPPORTED,
                "the adjoint does not support the anti-trapping current, grain growth or elasticity");
  if (c->m.dim == 3 && c->m.bc[2] == kBcHalo)
    return fail(c, MS_ERR_UNSUPPORTED, "the adjoint needs the whole domain (no halo faces)");
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
  const int blocks = (int)((cells + 127) / 128);   // blocks of the cell pass (parameter partials)
  if (nprm > kMaxGradParams) return fail(c, MS_ERR_UNSUPPORTED, "too many parameters for the gradient scratch");
  // lazily sized work buffers, each allocated while it is missing: a failed
  // allocation leaves its pointer null and the next call retries it
  for (int b = 0; b < 2; ++b)
    if (!A.adj[b]) {
      A.adj[b] = dev_alloc(c->hook, lam_bytes);
      if (!A.adj[b]) return fail(c, MS_ERR_OOM, "adjoint state allocation failed");
    }
  if (!A.tbar) {
    A.tbar = dev_alloc(c->hook, (size_t)adjoint_work_elems(m) * s);
    if (!A.tbar) return fail(c, MS_ERR_OOM, "adjoint tail buffer allocation failed");
  }
  if (!A.gpart) {
    A.gpart = static_cast<double*>(dev_alloc(c->hook, sizeof(double) * (size_t)blocks * nprm));
    if (!A.gpart) return fail(c, MS_ERR_OOM, "gradient scratch allocation failed");
  }
  if (!A.gsum) {
    A.gsum = static_cast<double*>(dev_alloc(c->hook, sizeof(double) * kMaxGradParams));
    if (!A.gsum) return fail(c, MS_ERR_OOM, "gradient scratch allocation failed");
  }
  const size_t seg_need = (size_t)A.every * c->state_bytes;
  if (!A.seg || A.seg_bytes < seg_need) {
    dev_free(c->hook, A.seg);
    A.seg_bytes = 0;
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
  if (e == cudaSuccess) e = cudaMemsetAsync(A.gsum, 0, sizeof(double) * kMaxGradParams, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(A.gpart, 0, sizeof(double) * (size_t)blocks * nprm, st);
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
      e = ak->launch(slots + (size_t)k * c->state_bytes, A.adj[cur], A.adj[1 - cur], A.tbar, c->args.data(), m,
                     t, A.gpart, st);
      if (e != cudaSuccess) return cuda_fail(c, e, "adjoint step");
      cur = 1 - cur;
    }
  }
  k_accumulate_params<<<nprm, 32, 0, st>>>(A.gpart, blocks, nprm, A.gsum);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "gradient reduction");
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
