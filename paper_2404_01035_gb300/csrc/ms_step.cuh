// Forward step kernel: one fused launch reads phi^n, mu^n once from HBM and
// writes phi^{n+1}, mu^{n+1} once.
//
// Layout (per state buffer): NF = N + K-1 fields, each [nzp][nyp][pitch] with
// one ghost layer per side (ghost = periodic image or mirrored neighbour);
// interior x = 0 sits at element `xoff` = 16 bytes into the row so that every
// TMA box starts on a 16-byte boundary.
//
// CTA = TX x TY cells of one xy tile, marching over `zchunk` planes in z.
// One elected thread loads each halo'ed plane of all NF fields with a single
// 4-D TMA box {TX + 2H, TY + 2, 1, NF} into a ring of NST shared-memory stages
// (completion on an mbarrier, bounded waits).  When a plane lands, the CTA
// computes per cell of the plane (with halo) the phase-presence bits and the
// cell mobility M = sum h D chi once; the stencil of a cell then ORs 19 (3-D)
// or 9 (2-D) presence bytes, which lets the bulk shortcut and the pair skip
// work without touching every phase value.  Outputs are written with plain
// coalesced stores, boundary cells also writing their ghost images, so no
// separate halo kernel runs between steps.
#pragma once

#include "ms_cell.cuh"

namespace msgb {

template <class Real>
struct Halo {
  static constexpr int H = 16 / sizeof(Real);   // elements per 16 bytes
};

template <int DIM, int NP, int NM, class Real, int TX, int TY>
struct StepShape {
  static constexpr int NF = NP + NM;
  static constexpr int H = Halo<Real>::H;
  static constexpr int SX = TX + 2 * H;
  static constexpr int SY = TY + 2;
  static constexpr int NT = TX * TY;
  static constexpr int NST = DIM == 3 ? 6 : 1;          // ring stages
  static constexpr int NAUX = DIM == 3 ? 3 : 1;         // preprocessed planes
  static constexpr int AX = TX + 2, AY = TY + 2;       // aux plane extents
  static constexpr int STAGE_ELEMS = NF * SY * SX;
  static constexpr int STAGE_BYTES = STAGE_ELEMS * (int)sizeof(Real);
  static constexpr int STAGE_STRIDE = (STAGE_BYTES + 127) / 128 * 128;
  static constexpr int MOB_BYTES = NAUX * NM * NM * AX * AY * (int)sizeof(Real);
  static constexpr int BITS_BYTES = (NAUX * AX * AY + 15) / 16 * 16;
  static constexpr int OFF_MOB = NST * STAGE_STRIDE;
  static constexpr int OFF_BITS = OFF_MOB + (MOB_BYTES + 15) / 16 * 16;
  static constexpr int OFF_BAR = OFF_BITS + BITS_BYTES;
  static constexpr int SMEM_BYTES = OFF_BAR + NST * 8 + 128;  // + alignment slack
};

// Stencil accessor over the shared-memory ring (planes k-1, k, k+1).
template <int DIM, int NP, int NM, class Real, int TX, int TY>
struct SmemAcc {
  using Sh = StepShape<DIM, NP, NM, Real, TX, TY>;
  const Real* st[3];
  const Real* mob[3];
  const uint8_t* bits[3];
  int sidx, aidx;

  __device__ __forceinline__ Real phi(int a, int dx, int dy, int dz) const {
    return st[1 + dz][a * Sh::SY * Sh::SX + sidx + dy * Sh::SX + dx];
  }
  __device__ __forceinline__ Real mu(int i, int dx, int dy, int dz) const {
    return st[1 + dz][(NP + i) * Sh::SY * Sh::SX + sidx + dy * Sh::SX + dx];
  }
  __device__ __forceinline__ uint32_t mask() const {
    const uint8_t* b = bits[1] + aidx;
    uint32_t m = b[-Sh::AX - 1] | b[-Sh::AX] | b[-Sh::AX + 1] | b[-1] | b[0] | b[1] |
                 b[Sh::AX - 1] | b[Sh::AX] | b[Sh::AX + 1];
    if constexpr (DIM == 3) {
      const uint8_t* u = bits[2] + aidx;
      const uint8_t* d = bits[0] + aidx;
      m |= u[0] | u[-1] | u[1] | u[-Sh::AX] | u[Sh::AX];
      m |= d[0] | d[-1] | d[1] | d[-Sh::AX] | d[Sh::AX];
    }
    return m;
  }
  __device__ __forceinline__ void mobility(int dx, int dy, int dz, Real* M) const {
    const int i = aidx + dy * Sh::AX + dx;
#pragma unroll
    for (int k = 0; k < NM * NM; ++k) M[k] = mob[1 + dz][k * Sh::AX * Sh::AY + i];
  }
};

// Write one output value of cell (x, y, z) and its ghost images.
template <int DIM, class Real, int NP, int NM>
__device__ __forceinline__ void store_with_ghosts(const StepArgs<Real, NP, NM>& g, Real* base,
                                                  int x, int y, int z, Real v) {
  int xs[3], ys[3], zs[3];
  int nxs = 1, nys = 1, nzs = 1;
  xs[0] = x;
  ys[0] = y;
  zs[0] = z;
  if (x == 0) xs[nxs++] = g.bc[0] == 3 ? g.nx : -1;
  if (x == g.nx - 1) xs[nxs++] = g.bc[0] == 3 ? -1 : g.nx;
  if (y == 0) ys[nys++] = g.bc[1] == 3 ? g.ny : -1;
  if (y == g.ny - 1) ys[nys++] = g.bc[1] == 3 ? -1 : g.ny;
  if constexpr (DIM == 3) {
    if (z == 0) zs[nzs++] = g.bc[2] == 3 ? g.nz : -1;
    if (z == g.nz - 1) zs[nzs++] = g.bc[2] == 3 ? -1 : g.nz;
  }
  const long long plane = (long long)g.nyp * g.pitch;
  base[(long long)(z + g.zoff) * plane + (long long)(y + 1) * g.pitch + x + g.xoff] = v;
  if (nxs == 1 && nys == 1 && nzs == 1) return;
  for (int iz = 0; iz < nzs; ++iz)
    for (int iy = 0; iy < nys; ++iy)
      for (int ix = 0; ix < nxs; ++ix) {
        if (ix == 0 && iy == 0 && iz == 0) continue;
        base[(long long)(zs[iz] + g.zoff) * plane + (long long)(ys[iy] + 1) * g.pitch + xs[ix] +
             g.xoff] = v;
      }
}

template <int DIM, int NP, int NM, class Real, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) k_gp_step(const __grid_constant__ CUtensorMap tm,
                                                    const __grid_constant__ StepArgs<Real, NP, NM> g) {
  using Sh = StepShape<DIM, NP, NM, Real, TX, TY>;
  constexpr int NST = Sh::NST;
  constexpr int NAUX = Sh::NAUX;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  Real* mobs = reinterpret_cast<Real*>(smem + Sh::OFF_MOB);
  uint8_t* bits = smem + Sh::OFF_BITS;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Sh::OFF_BAR);
  auto stage = [&](int s) { return reinterpret_cast<Real*>(smem + s * Sh::STAGE_STRIDE); };

  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int tiles_x = (g.nx + TX - 1) / TX;
  const int x0 = (blockIdx.x % tiles_x) * TX;
  const int y0 = (blockIdx.x / tiles_x) * TY;
  const int zb = DIM == 3 ? blockIdx.y * g.zchunk : 0;
  const int ze = DIM == 3 ? min(g.nz, zb + g.zchunk) : 1;
  const int nplanes = DIM == 3 ? (ze - zb + 2) : 1;
  const int bx = x0 + g.xoff - Sh::H;   // TMA box origin (16-byte aligned)

  if (tid == 0) {
    for (int s = 0; s < NST; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  __syncthreads();

  int issued = 0;   // planes issued (meaningful in thread 0)
  auto issue = [&](int j) {
    const int s = j % NST;
    mbar_expect_tx(&bars[s], Sh::STAGE_BYTES);
    const int zc = DIM == 3 ? (zb - 1 + j + g.zoff) : 0;
    tma_load_4d(stage(s), &tm, &bars[s], bx, y0, zc, 0);
  };
  if (tid == 0) {
    prefetch_tensormap(&tm);
    const int n0 = nplanes < NST ? nplanes : NST;
    for (int j = 0; j < n0; ++j) issue(j);
    issued = n0;
  }

  // presence bits and cell mobility of every (halo'ed) cell of plane j
  auto preprocess = [&](int j) {
    const Real* st = stage(j % NST);
    const int slot = j % NAUX;
    for (int i = tid; i < Sh::AX * Sh::AY; i += Sh::NT) {
      const int ay = i / Sh::AX, ax = i % Sh::AX;
      const int si = ay * Sh::SX + ax + Sh::H - 1;
      Real ph[NP];
      uint32_t b = 0;
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        ph[a] = st[a * Sh::SY * Sh::SX + si];
        b |= (ph[a] != Real(0) ? 1u : 0u) << a;
      }
      bits[slot * Sh::AX * Sh::AY + i] = (uint8_t)b;
      Real M[NM * NM];
      cell_mobility<NP, NM>(ph, g.DX, M);
#pragma unroll
      for (int k = 0; k < NM * NM; ++k)
        mobs[(slot * NM * NM + k) * Sh::AX * Sh::AY + i] = M[k];
    }
  };

  // Abort path after a timed-out wait: wait (bounded) for the copies still in
  // flight so that no TMA writes into freed shared memory, then leave.
  auto abort_cta = [&]() {
    if (tid == 0) {
      atomicOr(g.status, kStatusTimeout);
      for (int s = 0; s < NST; ++s) {
        if (issued <= s) continue;
        const int j = s + ((issued - 1 - s) / NST) * NST;   // last plane issued into stage s
        mbar_wait_bounded(&bars[s], (j / NST) & 1);
      }
    }
  };

  bool ok = true;
  const int first = DIM == 3 ? 2 : 1;   // planes needed before the first compute
  for (int j = 0; j < first; ++j) {
    ok = ok && mbar_wait_bounded(&bars[j % NST], (j / NST) & 1);
    if (ok) preprocess(j);
  }
  const int nk = DIM == 3 ? (ze - zb) : 1;
  for (int k = 0; k < nk; ++k) {
    if constexpr (DIM == 3) {
      const int j = k + 2;
      ok = ok && mbar_wait_bounded(&bars[j % NST], (j / NST) & 1);
      if (ok) preprocess(j);
    }
    if (__syncthreads_or(!ok)) {
      abort_cta();
      return;
    }
    const int z = zb + k;
    const int x = x0 + tx, y = y0 + ty;
    SmemAcc<DIM, NP, NM, Real, TX, TY> acc;
    if constexpr (DIM == 3) {
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        acc.st[r] = stage((k + r) % NST);
        acc.mob[r] = mobs + ((k + r) % NAUX) * NM * NM * Sh::AX * Sh::AY;
        acc.bits[r] = bits + ((k + r) % NAUX) * Sh::AX * Sh::AY;
      }
    } else {
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        acc.st[r] = stage(0);
        acc.mob[r] = mobs;
        acc.bits[r] = bits;
      }
    }
    acc.sidx = (ty + 1) * Sh::SX + tx + Sh::H;
    acc.aidx = (ty + 1) * Sh::AX + tx + 1;
    if (x < g.nx && y < g.ny) {
      DiffPrm<Real, StepArgs<Real, NP, NM>::P> dp;
      dp.mob = g.mob;
#pragma unroll
      for (int p = 0; p < StepArgs<Real, NP, NM>::P; ++p) dp.delta[p] = g.delta[p];
      Real pn[NP], mn[NM];
      gp_cell<DIM, NP, NM, Real, Real>(acc, g, dp, DIM == 3 ? z : y, pn, mn);
#pragma unroll
      for (int a = 0; a < NP; ++a) store_with_ghosts<DIM>(g, g.out + a * g.fstride, x, y, z, pn[a]);
#pragma unroll
      for (int i = 0; i < NM; ++i)
        store_with_ghosts<DIM>(g, g.out + (NP + i) * g.fstride, x, y, z, mn[i]);
    }
    if constexpr (DIM == 3) {
      __syncthreads();   // everyone is done with plane k's stage
      if (tid == 0 && k + NST < nplanes) {
        issue(k + NST);
        issued = k + NST + 1;
      }
    }
  }
}

}  // namespace msgb
