// Anti-trapping current in the mu update (MICROSIM paper, arXiv 2404.01035,
// Sec. 2.1, Eq. jatr and the obstacle / well forms of j^{at,alpha} below it):
// j_at = sum_{alpha < liquid} A_alpha (c^alpha - c^liq) d phi_alpha/dt
// n_alpha (-n_alpha . n_liq), subtracted from M grad mu inside the divergence
// of Eq. (Mu_explicit_temperature).
//
// It needs d phi/dt at both cells of every face, so it runs after the step
// that wrote phi^{n+1} and mu* (the mu update without the current) into the
// output buffer: mu^{n+1} = mu* - chi(h(phi^{n+1}))^-1 dt div j_at (the update
// is linear in its right-hand side).  Two kernels: k_at_list lists the 32-cell
// row segments whose 3 x 3 (x 3) block of segments is not one pure phase in
// phi^n (elsewhere every phase gradient at every face of the segment's cells
// is zero, so no face has a normal and the current vanishes); k_at_work stages
// the block around each listed segment in shared memory (phi^n and mu^n from
// the input, phi^{n+1} from the output) and corrects mu, one lane per cell.
#pragma once

#include "ms_step.cuh"

namespace msgb {

// 1 / sqrt(x): the hardware reciprocal square root in FP32 (rsqrtf, a few
// ulp: the current is a correction far inside the FP32 tolerance), exact in
// FP64.
__device__ __forceinline__ float inv_sqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double inv_sqrt(double x) { return 1.0 / sqrt(x); }

// Coefficient A of j^{at,alpha} at the face value p of phi_alpha (read as the
// 1-D equilibrium profile value there): obstacle pi eps p (1 - h(p)) /
// (4 sqrt(p (1 - p))) with the two-phase h(p) = p^2 (3 - 2p), 0 outside
// 0 < p < 1; well eps / (2 sqrt 2).
template <class Real>
__device__ __forceinline__ Real at_coefficient(int potential, Real eps, Real p) {
  if (potential != 1) return eps * Real(0.35355339059327376220);   // 1 / (2 sqrt 2)
  if (!(p > Real(0) && p < Real(1))) return Real(0);
  const Real h = p * p * (Real(3) - Real(2) * p);
  return Real(0.78539816339744830962) * eps * p * (Real(1) - h) * inv_sqrt(p * (Real(1) - p));   // pi / 4
}

// Shape of the staged block of one row segment: fields [phi^n (NP), mu^n
// (NM), phi^{n+1} (NP)] x planes (3 in 3-D, 1 in 2-D) x 3 rows x 34 cells
// (x0 - 1 .. x0 + 32).
template <int DIM, int NP, int NM, class Real>
struct AtShape {
  static constexpr int NF = 2 * NP + NM;
  static constexpr int BX = 34;
  static constexpr int NPL = DIM == 3 ? 3 : 1;
  static constexpr int ROWS = NF * NPL * 3;
  static constexpr int WARP_ELEMS = ROWS * BX;
  static constexpr int WARP_BYTES = WARP_ELEMS * (int)sizeof(Real);
  static constexpr int WARPS_RAW = (160 * 1024) / WARP_BYTES;
  static constexpr int WARPS = WARPS_RAW < 1 ? 1 : (WARPS_RAW > 8 ? 8 : WARPS_RAW);
  static constexpr int THREADS = 32 * WARPS;
  static constexpr int SMEM_BYTES = WARPS * WARP_BYTES;
};

// Asynchronous copy of one element from global to shared memory (cp.async
// through L1, bypassing registers), and the wait for this thread's copies.
template <class Real>
__device__ __forceinline__ void cp_async_elem(Real* dst, const Real* src) {
  if constexpr (sizeof(Real) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Reads of the staged block relative to the lane's cell: field f, offsets
// dx, dy, dz in [-1, 1] (dz = 0 in 2-D).
template <int DIM, int NP, int NM, class Real>
struct AtBox {
  using Sh = AtShape<DIM, NP, NM, Real>;
  const Real* s;   // the warp's block
  int lane;
  __device__ __forceinline__ Real at(int f, int dx, int dy, int dz) const {
    return s[((f * Sh::NPL + (DIM == 3 ? dz + 1 : 0)) * 3 + dy + 1) * Sh::BX + lane + 1 + dx];
  }
  __device__ __forceinline__ Real phi(int a, int dx, int dy, int dz) const { return at(a, dx, dy, dz); }
  __device__ __forceinline__ Real mu(int i, int dx, int dy, int dz) const { return at(NP + i, dx, dy, dz); }
  __device__ __forceinline__ Real phin(int a, int dx, int dy, int dz) const { return at(NP + NM + a, dx, dy, dz); }
};

// dt times the normal component along axis d of j_at_i (the rates are taken
// as phi^{n+1} - phi^n) at the face between the cell at
// offset (ox, oy, oz) from the lane's cell and its +d neighbour: face values
// as for the gradient-energy fluxes (means of the two cells; normal
// difference and 4-point averaged tangential differences of phi^n), T the
// mean of the two cells' temperatures; kl = index of the left cell along the
// last axis.
template <int DIM, int NP, int NM, class Real>
__device__ __forceinline__ void at_face(const StepArgs<Real, NP, NM>& g, const AtBox<DIM, NP, NM, Real>& A, int ox,
                                        int oy, int oz, int d, int kl, Real* J) {
  constexpr int L = NP - 1;   // the liquid
  const int rx = ox + (d == 0), ry = oy + (d == 1), rz = oz + (d == 2);
  Real pf[NP], rate[NP], nrm[NP][DIM];
  bool has_n[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    const Real vl = A.phi(a, ox, oy, oz), vr = A.phi(a, rx, ry, rz);
    pf[a] = Real(0.5) * (vl + vr);
    rate[a] = Real(0.5) * ((A.phin(a, ox, oy, oz) - vl) + (A.phin(a, rx, ry, rz) - vr));   // dt d phi/dt
    Real gr[DIM], g2 = Real(0);
#pragma unroll
    for (int t = 0; t < DIM; ++t) {
      if (t == d) {
        gr[t] = (vr - vl) * g.inv_dx;
      } else {
        const int tx = t == 0, ty = t == 1, tz = t == 2;
        gr[t] = ((A.phi(a, ox + tx, oy + ty, oz + tz) + A.phi(a, rx + tx, ry + ty, rz + tz)) -
                 (A.phi(a, ox - tx, oy - ty, oz - tz) + A.phi(a, rx - tx, ry - ty, rz - tz))) *
                g.quarter_inv_dx;
      }
      g2 += gr[t] * gr[t];
    }
    has_n[a] = g2 >= Real(1e-12);
    const Real inv = has_n[a] ? inv_sqrt(g2) : Real(0);
#pragma unroll
    for (int t = 0; t < DIM; ++t) nrm[a][t] = gr[t] * inv;
  }
#pragma unroll
  for (int i = 0; i < NM; ++i) J[i] = Real(0);
  if (!has_n[L]) return;
  Real mf[NM];
#pragma unroll
  for (int i = 0; i < NM; ++i) mf[i] = Real(0.5) * (A.mu(i, ox, oy, oz) + A.mu(i, rx, ry, rz));
  // T - T_ref at the two cells (after the boundary mapping) and their mean
  const int n = DIM == 3 ? g.nz : g.ny, bc = g.bc[DIM - 1];
  const int kr = kl + (d == DIM - 1);
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

// One thread per row segment: append the segments whose block of segments is
// not one pure phase in phi^n to the work list ([0] count, [1] ticket).
template <int DIM, int NP, int NM, class Real>
__global__ void __launch_bounds__(256) k_at_list(const __grid_constant__ StepArgs<Real, NP, NM> g) {
  const long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int nzi = DIM == 3 ? g.nz : 1;
  const long long nseg = (long long)g.segs * g.ny * nzi;
  bool need = false;
  if (w < nseg) {
    const int s = (int)(w % g.segs);
    const int y = (int)((w / g.segs) % g.ny);
    const int z = (int)(w / ((long long)g.segs * g.ny));
    const int c0 = load_code_from(g.codes_in, g, s, y, z) & kCodePhase;
    bool pure = c0 != 0;
#pragma unroll
    for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz)
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int ds = -1; ds <= 1; ++ds)
          pure = pure && (load_code_from(g.codes_in, g, s + ds, y + dy, z + dz) & kCodePhase) == c0;
    need = !pure;
  }
  const unsigned int m = __ballot_sync(0xffffffffu, need);
  if (m == 0u) return;
  const int first = __ffs(m) - 1;
  unsigned int base = 0;
  if (lane == first) base = atomicAdd(&g.at_list[0], (unsigned int)__popc(m));
  base = __shfl_sync(0xffffffffu, base, first);
  if (need) {
    const unsigned int i = base + __popc(m & ((1u << lane) - 1u));
    if (i < g.at_cap) g.at_list[2 + i] = (unsigned int)w;
  }
}

// Warps over the listed segments: stage the block, correct mu.  The last CTA
// to finish clears the list (ticket), so the launches replay from a graph.
template <int DIM, int NP, int NM, class Real>
__global__ void __launch_bounds__(AtShape<DIM, NP, NM, Real>::THREADS)
    k_at_work(const __grid_constant__ StepArgs<Real, NP, NM> g, const Real* __restrict__ in) {
  using Sh = AtShape<DIM, NP, NM, Real>;
  extern __shared__ unsigned char smem_raw[];
  __shared__ unsigned int s_count;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  Real* const box = reinterpret_cast<Real*>(smem_raw) + wid * Sh::WARP_ELEMS;
  if (threadIdx.x == 0) s_count = min(*(volatile unsigned int*)&g.at_list[0], g.at_cap);
  __syncthreads();
  const unsigned int count = s_count;
  const long long plane = (long long)g.nyp * g.pitch;
  const AtBox<DIM, NP, NM, Real> A{box, lane};
  for (unsigned int i = blockIdx.x * Sh::WARPS + wid; i < count; i += gridDim.x * Sh::WARPS) {
    const unsigned int r = g.at_list[2 + i];
    const int s = (int)(r % (unsigned int)g.segs);
    const unsigned int zy = r / (unsigned int)g.segs;
    const int y = (int)(zy % (unsigned int)g.ny), z = (int)(zy / (unsigned int)g.ny);
    const int x0 = 32 * s;
    // stage: rows (field, plane, row) of 34 cells x0 - 1 .. x0 + 32, all
    // copies in flight at once; cells past the +x ghost (x > nx) are never
    // read by an active lane and stay unset.  mu^n and phi^{n+1} are read
    // only at the two cells of a face, never on the four corner rows (a
    // y and a z offset together), which are left unset for them.
    const int xa = x0 - 1 + lane, xb = x0 + 31 + lane;
    for (int row = 0; row < Sh::ROWS; ++row) {
      const int f = row / (3 * Sh::NPL), pl = (row / 3) % Sh::NPL, ry = row % 3;
      if (DIM == 3 && f >= NP && pl != 1 && ry != 1) continue;
      const int zz = DIM == 3 ? z + pl - 1 : 0, yy = y + ry - 1;
      const Real* src = f < NP + NM ? in + (long long)f * g.fstride : g.out + (long long)(f - NP - NM) * g.fstride;
      src += (long long)(DIM == 3 ? zz + g.zoff : 0) * plane + (long long)(yy + 1) * g.pitch + g.xoff;
      if (xa <= g.nx) cp_async_elem(box + row * Sh::BX + lane, src + xa);
      if (lane < 2 && xb <= g.nx) cp_async_elem(box + row * Sh::BX + 32 + lane, src + xb);
    }
    cp_async_wait_all();
    __syncwarp();
    const int x = x0 + lane;
    if (x < g.nx) {
      const int k = DIM == 3 ? z : y;   // index along the last axis
      Real div[NM];
#pragma unroll
      for (int q = 0; q < NM; ++q) div[q] = Real(0);
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        Real Jp[NM], Jm[NM];
        at_face<DIM, NP, NM, Real>(g, A, 0, 0, 0, d, k, Jp);
        at_face<DIM, NP, NM, Real>(g, A, -(d == 0), -(d == 1), -(d == 2), d, k - (d == DIM - 1), Jm);
#pragma unroll
        for (int q = 0; q < NM; ++q) div[q] += (Jp[q] - Jm[q]) * g.inv_dx;
      }
      // mu^{n+1} = mu* + chi(h(phi^{n+1}))^-1 (-dt div j_at)
      Real pn[NP], h[NP];
#pragma unroll
      for (int a = 0; a < NP; ++a) pn[a] = A.phin(a, 0, 0, 0);
      interp_h<NP>(pn, h);
      Real chi[NM * NM], rhs[NM], dmu[NM], mn[NM];
#pragma unroll
      for (int q = 0; q < NM * NM; ++q) {
        chi[q] = h[0] * g.chi[0][q];
#pragma unroll
        for (int a = 1; a < NP; ++a) chi[q] += h[a] * g.chi[a][q];
      }
#pragma unroll
      for (int q = 0; q < NM; ++q) rhs[q] = -div[q];   // the rates above carry no 1/dt: dt div j_at
      solve_small<NM>(chi, rhs, dmu);
      const long long o = (long long)(DIM == 3 ? z + g.zoff : 0) * plane + (long long)(y + 1) * g.pitch + x + g.xoff;
#pragma unroll
      for (int q = 0; q < NM; ++q) mn[q] = g.out[(long long)(NP + q) * g.fstride + o] + dmu[q];
      store_cell<DIM>(g, x, y, z, pn, mn, false);
    }
    __syncwarp();   // the block is refilled for the next segment
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&g.at_list[1], 1u) == gridDim.x - 1) {
      g.at_list[0] = 0u;
      g.at_list[1] = 0u;
    }
  }
}

}  // namespace msgb
