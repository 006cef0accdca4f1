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
// (completion on an mbarrier, bounded waits).  When a plane lands, each warp
// classifies whole rows of it: per cell a presence code (which phases are
// non-zero, and whether the cell is exactly a pure phase), per row a flag
// saying "every cell of this halo'ed row is the same pure phase".  A warp whose
// 3 x 3 neighbouring rows (3 rows x 3 planes in 3-D) all carry the same flag
// is in bulk: phi is unchanged there bit for bit and mu follows a constant-
// mobility diffusion update, so it skips the interface arithmetic entirely.
// Other warps run the full cell update with the per-cell phase mask (absent
// pairs are skipped exactly).  Outputs are written with coalesced stores;
// boundary cells also write their ghost images, so no halo kernel runs
// between steps.
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
  static constexpr int NT = TX * TY;                    // consumer threads (one per cell)
  static constexpr int NCW = NT / 32;                   // consumer warps
  static constexpr int NTHREADS = NT + 32;              // + one producer warp
  static constexpr int WC = TX / 32;                    // warps per row
  static constexpr int STAGE_ELEMS = NF * SY * SX;
  static constexpr int STAGE_BYTES = STAGE_ELEMS * (int)sizeof(Real);
  static constexpr int STAGE_STRIDE = (STAGE_BYTES + 127) / 128 * 128;
  // Ring depth: as many planes in flight as a shared-memory budget allows
  // (two CTAs per SM for up to 5 fields, one for more), 4..12 stages.
  static constexpr int RING_BUDGET = NF <= 5 ? 100 * 1024 : 190 * 1024;
  static constexpr int NST_RAW = RING_BUDGET / STAGE_STRIDE;
  static constexpr int NST = DIM == 3 ? (NST_RAW < 4 ? 4 : (NST_RAW > 12 ? 12 : NST_RAW)) : 1;
  static constexpr int NFL = SY * WC;                   // row flags per plane
  static constexpr int NWF = TY * WC;                   // combined flags per plane (one per warp row)
  static constexpr int FLAG_BYTES = (NST * NWF + 15) / 16 * 16;   // one flag set per stage
  static constexpr int CSEG = WC + 2;                   // segments per halo row (one each side)
  static constexpr int MAXPL = DIM == 3 ? kMaxZChunk + 2 : 1;     // ring entries of a CTA at most
  static constexpr int CODE_ENTRIES = MAXPL * SY * CSEG;          // segment codes a CTA reads
  static constexpr int CODE_BYTES = (CODE_ENTRIES + 15) / 16 * 16;
  static constexpr int CODE_ITERS = (CODE_ENTRIES + NTHREADS - 1) / NTHREADS;
  // codes of the previous state at this CTA's own rows (the output buffer
  // still holds that state: bulk rows whose phase did not change skip phi)
  static constexpr int PREV_ENTRIES = (DIM == 3 ? kMaxZChunk : 1) * TY * WC;
  static constexpr int PREV_BYTES = (PREV_ENTRIES + 15) / 16 * 16;
  static constexpr int PREV_ITERS = (PREV_ENTRIES + NTHREADS - 1) / NTHREADS;
  static constexpr int OFF_FLAG = NST * STAGE_STRIDE;
  static constexpr int OFF_CODE = OFF_FLAG + FLAG_BYTES;
  static constexpr int OFF_PREV = OFF_CODE + CODE_BYTES;
  static constexpr int OFF_BAR = OFF_PREV + PREV_BYTES;            // full[NST], empty[NST]
  static constexpr int OFF_ABORT = OFF_BAR + 2 * NST * 8;
  static constexpr int SMEM_BYTES = OFF_ABORT + 16 + 128;         // + alignment slack
  static_assert(TX % 32 == 0, "a warp must cover cells of a single row");
  static_assert(NFL <= 32, "the producer warp holds one row flag per lane");
};

// Phases present anywhere in the 19-point (3-D) / 9-point (2-D) stencil of
// an accessor's centre cell (bit a set when phi_a != 0 somewhere).
template <int DIM, int NP, class Acc>
__device__ __forceinline__ uint32_t stencil_mask(const Acc& A) {
  uint32_t m = 0;
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    bool any = false;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) any = any || A.phi(a, dx, dy, 0) != 0;
    if constexpr (DIM == 3) {
#pragma unroll
      for (int dz = -1; dz <= 1; dz += 2)
        any = any || A.phi(a, 0, 0, dz) != 0 || A.phi(a, -1, 0, dz) != 0 || A.phi(a, 1, 0, dz) != 0 ||
              A.phi(a, 0, -1, dz) != 0 || A.phi(a, 0, 1, dz) != 0;
    }
    m |= (any ? 1u : 0u) << a;
  }
  return m;
}

// Stencil accessor over the shared-memory ring (planes k-1, k, k+1).
template <int DIM, int NP, int NM, class Real, int TX, int TY>
struct SmemAcc {
  using Sh = StepShape<DIM, NP, NM, Real, TX, TY>;
  const Real* st[3];
  const StepArgs<Real, NP, NM>* g;
  int sidx;

  __device__ __forceinline__ Real phi(int a, int dx, int dy, int dz) const {
    return st[1 + dz][a * Sh::SY * Sh::SX + sidx + dy * Sh::SX + dx];
  }
  __device__ __forceinline__ Real mu(int i, int dx, int dy, int dz) const {
    return st[1 + dz][(NP + i) * Sh::SY * Sh::SX + sidx + dy * Sh::SX + dx];
  }
  __device__ __forceinline__ uint32_t mask() const { return stencil_mask<DIM, NP>(*this); }
  // cell mobility M = sum_a h_a D^a chi^a of a neighbour, from its phi
  __device__ __forceinline__ void mobility(int dx, int dy, int dz, Real* M) const {
    Real ph[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) ph[a] = phi(a, dx, dy, dz);
    cell_mobility<NP, NM>(ph, g->DX, M);
  }
};

// Index along an axis with the boundary mapping (ghost = periodic image or
// the adjacent interior cell).
__device__ __forceinline__ int bc_map(int i, int n, int bc) {
  if (i >= 0 && i < n) return i;
  if (bc == 3) return ((i % n) + n) % n;
  return i < 0 ? 0 : n - 1;
}

// Segment code of (segment s, row y, plane z) of a code array (the input
// state's by default), with the boundary mapping of each axis (out-of-range
// indices give the periodic image or the adjacent interior segment, row or
// plane).
template <class Real, int NP, int NM>
__device__ __forceinline__ uint8_t load_code_from(const uint8_t* codes, const StepArgs<Real, NP, NM>& g, int s, int y,
                                                  int z) {
  const int ss = bc_map(s, g.segs, g.bc[0]);
  const int yy = bc_map(y, g.ny, g.bc[1]);
  // plane index in the code array (3-D arrays carry one ghost plane per side,
  // filled by the halo exchange when that face is an internal cut)
  int zz;
  if (z >= 0 && z < g.nz)
    zz = z + g.zoff;
  else if (g.bc[2] == kBcHalo)
    zz = z < 0 ? 0 : g.nz + 1;
  else
    zz = bc_map(z, g.nz, g.bc[2]) + g.zoff;
  return __ldg(codes + ((long long)zz * g.ny + yy) * g.segs + ss);
}
template <class Real, int NP, int NM>
__device__ __forceinline__ uint8_t load_code(const StepArgs<Real, NP, NM>& g, int s, int y, int z) {
  return load_code_from(g.codes_in, g, s, y, z);
}

// Row flag: the pure phase + 1 when three adjacent segments agree on it
// (the reuse bit of each code is ignored).
__device__ __forceinline__ int combine_codes(const uint8_t* c) {
  const int a = c[0] & kCodePhase, b = c[1] & kCodePhase, d = c[2] & kCodePhase;
  return (a == b && b == d) ? b : 0;
}

// Bulk cell (whole stencil is the pure phase l): phi unchanged, and
// mu^{n+1} = mu + Kb_l (sum_nb mu_nb - 2d mu) - eb_l, the constant-mobility
// form of the mu update with M = D^l chi^l, chi = chi^l and dh = 0.
template <int DIM, int NP, int NM, class Real, class Acc>
__device__ __forceinline__ void bulk_cell(const Acc& A, const StepArgs<Real, NP, NM>& g, int l,
                                          Real* pn, Real* mn) {
#pragma unroll
  for (int a = 0; a < NP; ++a) pn[a] = a == l ? Real(1) : Real(0);
  Real L[NM], mc[NM];
#pragma unroll
  for (int i = 0; i < NM; ++i) {
    mc[i] = A.mu(i, 0, 0, 0);
    Real s = (A.mu(i, -1, 0, 0) + A.mu(i, 1, 0, 0)) + (A.mu(i, 0, -1, 0) + A.mu(i, 0, 1, 0));
    if constexpr (DIM == 3) s += A.mu(i, 0, 0, -1) + A.mu(i, 0, 0, 1);
    L[i] = s - Real(2 * DIM) * mc[i];
  }
#pragma unroll
  for (int i = 0; i < NM; ++i) {
    Real d = mc[i] - g.eb[l][i];
#pragma unroll
    for (int j = 0; j < NM; ++j) d += g.Kb[l][i * NM + j] * L[j];
    mn[i] = d;
  }
}

// Store the NF outputs of cell (x, y, z), plus ghost images on the boundary;
// with write_phi false only mu (the output buffer already holds phi^{n+1}).
// Coordinate of variant v of cell c along an axis of n cells with boundary
// code bc: v = 0 the cell itself, v = 1 its ghost image when c is the first
// cell (c + n periodic, -1 mirrored), v = 2 when c is the last (-1 periodic,
// n mirrored); kNoImage when that variant does not exist (or `cut`: the
// axis' ghosts are filled by a halo exchange).
constexpr int kNoImage = -0x40000000;
__device__ __forceinline__ int image_coord(int v, int c, int n, int bc, bool cut) {
  if (v == 0) return c;
  if (cut) return kNoImage;
  if (v == 1) return c == 0 ? (bc == 3 ? n : -1) : kNoImage;
  return c == n - 1 ? (bc == 3 ? -1 : n) : kNoImage;
}

template <int DIM, int NP, int NM, class Real>
__device__ __forceinline__ void store_cell(const StepArgs<Real, NP, NM>& g, int x, int y, int z,
                                           const Real* pn, const Real* mn, bool write_phi = true) {
  const long long plane = (long long)g.nyp * g.pitch;
  Real* base = g.out + (long long)(z + g.zoff) * plane + (long long)(y + 1) * g.pitch + x + g.xoff;
  if (write_phi) {
#pragma unroll
    for (int a = 0; a < NP; ++a) base[a * g.fstride] = pn[a];
  }
#pragma unroll
  for (int i = 0; i < NM; ++i) base[(NP + i) * g.fstride] = mn[i];
  const bool edge = x == 0 || x == g.nx - 1 || y == 0 || y == g.ny - 1 ||
                    (DIM == 3 && (z == 0 || z == g.nz - 1));
  if (!edge) return;
  // every combination of the cell and its ghost images along each axis
  // (variant 0 = the cell, 1 = its image when it is the first cell, 2 = when
  // it is the last; scalars, so that nothing lives in local memory)
  const bool zcut = DIM != 3 || g.bc[2] == kBcHalo;   // halo faces: the exchange fills them
  for (int iz = 0; iz < (DIM == 3 ? 3 : 1); ++iz) {
    const int zi = image_coord(iz, z, g.nz, g.bc[2], zcut);
    if (zi == kNoImage) continue;
    for (int iy = 0; iy < 3; ++iy) {
      const int yi = image_coord(iy, y, g.ny, g.bc[1], false);
      if (yi == kNoImage) continue;
      for (int ix = 0; ix < 3; ++ix) {
        if ((ix | iy | iz) == 0) continue;
        const int xi = image_coord(ix, x, g.nx, g.bc[0], false);
        if (xi == kNoImage) continue;
        Real* p = g.out + (long long)(zi + g.zoff) * plane + (long long)(yi + 1) * g.pitch + xi + g.xoff;
        if (write_phi) {
#pragma unroll
          for (int a = 0; a < NP; ++a) p[a * g.fstride] = pn[a];
        }
#pragma unroll
        for (int i = 0; i < NM; ++i) p[(NP + i) * g.fstride] = mn[i];
      }
    }
  }
}

// Minimum CTAs per SM the register allocation must allow: two for the
// few-phase kernels of up to 256 consumer threads, else one.
template <int NP, int NT>
struct MinBlocks {
  static constexpr int value = (NP <= 4 && NT <= 256) ? 2 : 1;
};

template <int DIM, int NP, int NM, class Real, int TX, int TY>
__global__ void __launch_bounds__(TX* TY + 32, MinBlocks<NP, TX * TY>::value)
    k_gp_step(const __grid_constant__ CUtensorMap tm, const __grid_constant__ StepArgs<Real, NP, NM> g) {
  using Sh = StepShape<DIM, NP, NM, Real, TX, TY>;
  constexpr int NST = Sh::NST;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  uint8_t* rowflag = smem + Sh::OFF_FLAG;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Sh::OFF_BAR);
  uint64_t* empty = full + NST;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + Sh::OFF_ABORT);
  auto stage = [&](int s) { return reinterpret_cast<Real*>(smem + s * Sh::STAGE_STRIDE); };

  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int tiles_x = (g.nx + TX - 1) / TX;
  const int x0 = (blockIdx.x % tiles_x) * TX;
  const int y0 = (blockIdx.x / tiles_x) * TY;
  const int zb = DIM == 3 ? blockIdx.y * g.zchunk : 0;
  const int ze = DIM == 3 ? min(g.nz, zb + g.zchunk) : 1;
  const int nplanes = DIM == 3 ? (ze - zb + 2) : 1;   // ring entries j <-> plane zb - 1 + j
  const int nk = DIM == 3 ? (ze - zb) : 1;             // planes computed
  if (nplanes > Sh::MAXPL) {   // the host clamps z-chunks; never touch smem beyond its size
    if (tid == 0) atomicOr(g.status, kStatusLaunch);
    return;
  }

  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], Sh::NCW);
    }
    *abort_flag = 0;
    mbar_fence_init();
  }
  __syncthreads();

  // The producer starts the first ring entries (their flags are published
  // later by a plain arrive), then every thread loads the segment codes of
  // this CTA into shared memory: all loads in flight together, once.
  const int bx = x0 + g.xoff - Sh::H;   // TMA box origin (16-byte aligned)
  const int npre = nplanes < NST ? nplanes : NST;
  if (tid == Sh::NT) {
    prefetch_tensormap(&tm);
    for (int j = 0; j < npre; ++j) {
      mbar_expect_tx_only(&full[j], Sh::STAGE_BYTES);
      const int zc = DIM == 3 ? (zb - 1 + j + g.zoff) : 0;
      tma_load_4d(stage(j), &tm, &full[j], bx, y0, zc, 0);
    }
  }
  {
    const int seg0 = x0 >> 5;
    const int ncode = nplanes * Sh::SY * Sh::CSEG;
    uint8_t v[Sh::CODE_ITERS];
#pragma unroll
    for (int it = 0; it < Sh::CODE_ITERS; ++it) {
      const int e = tid + it * Sh::NTHREADS;
      v[it] = 0;
      if (e < ncode) {
        const int k = e % Sh::CSEG, r = e / Sh::CSEG;
        const int ay = r % Sh::SY, j = r / Sh::SY;
        v[it] = load_code(g, seg0 - 1 + k, y0 - 1 + ay, DIM == 3 ? zb - 1 + j : 0);
      }
    }
    // previous-state codes of this CTA's own rows (read before any is overwritten)
    const int nprev = nk * TY * Sh::WC;
    uint8_t w[Sh::PREV_ITERS];
#pragma unroll
    for (int it = 0; it < Sh::PREV_ITERS; ++it) {
      const int e = tid + it * Sh::NTHREADS;
      w[it] = 0;
      if (e < nprev && g.reuse_prev) {
        const int wc = e % Sh::WC, r = e / Sh::WC;
        const int ty = r % TY, k = r / TY;
        const int y = y0 + ty, sg = seg0 + wc;
        if (y < g.ny && sg < g.segs)
          w[it] = g.codes_out[((long long)((DIM == 3 ? zb + k : 0) + g.zoff) * g.ny + y) * g.segs + sg];
      }
    }
    uint8_t* scode = smem + Sh::OFF_CODE;
#pragma unroll
    for (int it = 0; it < Sh::CODE_ITERS; ++it) {
      const int e = tid + it * Sh::NTHREADS;
      if (e < ncode) scode[e] = v[it];
    }
    uint8_t* sprev = smem + Sh::OFF_PREV;
#pragma unroll
    for (int it = 0; it < Sh::PREV_ITERS; ++it) {
      const int e = tid + it * Sh::NTHREADS;
      if (e < nprev) sprev[e] = w[it];
    }
  }
  __syncthreads();   // the last CTA-wide barrier: roles split below

  if (tid >= Sh::NT) {
    // ---------------- producer warp: TMA loads + row flags of every entry
    const int f_ay = lane / Sh::WC, f_wc = lane % Sh::WC;
    const bool fl = lane < Sh::NFL && (x0 >> 5) + f_wc < g.segs;   // warp column exists
    const uint8_t* scode = smem + Sh::OFF_CODE;
    int issued = npre, arrived = 0;
    bool ok = true;
    // row flags (lane = halo'ed row ay, warp column wc) of entries j-2, j-1, j
    int rf2 = 0, rf1 = 0, rf0 = 0;
    for (int j = 0; j < nplanes; ++j) {
      const int s = j % NST;
      if (j >= NST) {
        ok = ok && mbar_wait_bounded(&empty[s], ((j / NST) - 1) & 1);
        ok = ok && *abort_flag == 0;
        if (__any_sync(0xffffffffu, !ok)) break;
        if (lane == 0) {
          mbar_expect_tx_only(&full[s], Sh::STAGE_BYTES);
          const int zc = DIM == 3 ? (zb - 1 + j + g.zoff) : 0;
          tma_load_4d(stage(s), &tm, &full[s], bx, y0, zc, 0);
        }
        issued = j + 1;
      }
      rf2 = rf1;
      rf1 = rf0;
      rf0 = fl ? combine_codes(scode + (j * Sh::SY + f_ay) * Sh::CSEG + f_wc) : 0;
      // Combined flag of the centre entry (j-1 in 3-D, j in 2-D) for each warp
      // row: non-zero only if the 3 rows x 3 planes around it are one phase.
      {
        const int pc = DIM == 3 ? ((rf2 == rf1 && rf1 == rf0) ? rf1 : 0) : rf0;
        const int up = __shfl_down_sync(0xffffffffu, pc, Sh::WC);
        const int up2 = __shfl_down_sync(0xffffffffu, pc, 2 * Sh::WC);
        const int wf = (pc == up && up == up2) ? pc : 0;   // rows ay, ay+1, ay+2
        const int centre = DIM == 3 ? j - 1 : j;
        if (lane < Sh::NWF && centre >= 0) rowflag[(centre % NST) * Sh::NWF + lane] = (uint8_t)wf;
      }
      __syncwarp();
      if (lane == 0) {
        __threadfence_block();
        mbar_arrive(&full[s]);   // publishes the flags (release); the data lands by complete_tx
      }
      arrived = j + 1;
    }
    if (!ok && lane == 0) {
      // abort: record it, complete the arrivals of entries already issued,
      // then wait (bounded) for the copies still in flight so that no TMA
      // writes into shared memory after the CTA has exited
      atomicOr(g.status, kStatusTimeout);
      *abort_flag = 1;
      for (int j = arrived; j < issued; ++j) mbar_arrive(&full[j % NST]);
      for (int s = 0; s < NST; ++s) {
        if (issued <= s) continue;
        const int j = s + ((issued - 1 - s) / NST) * NST;
        mbar_wait_bounded(&full[s], (j / NST) & 1);
      }
    }
    return;
  }

  // -------------------- consumer warps: one cell per thread, one plane at a time
  const int tx = tid % TX, ty = tid / TX;
  const int wc = tx >> 5;                     // warp column within the row
  const int seg = (x0 >> 5) + wc;             // this warp's 32-cell segment
  const int x = x0 + tx, y = y0 + ty;
  const bool active = x < g.nx && y < g.ny;
  SmemAcc<DIM, NP, NM, Real, TX, TY> acc;
  acc.g = &g;
  const uint8_t* sprev = smem + Sh::OFF_PREV;

  acc.sidx = (ty + 1) * Sh::SX + tx + Sh::H;
  bool ok = true;
  if constexpr (DIM == 3) ok = mbar_wait_bounded(&full[0], 0) && mbar_wait_bounded(&full[1], 0);
  int s0 = 0, s1 = DIM == 3 ? 1 : 0, s2 = DIM == 3 ? 2 % NST : 0;
  uint32_t par2 = DIM == 3 ? (2 / NST) & 1 : 0;
  for (int k = 0; k < nk; ++k) {
    ok = ok && mbar_wait_bounded(&full[s2], par2) && *abort_flag == 0;
    if (!__all_sync(0xffffffffu, ok)) {   // the warp leaves together (votes below)
      if (lane == 0) {
        atomicOr(g.status, kStatusTimeout);
        *abort_flag = 1;
      }
      return;
    }
    const int z = zb + k;
    // warp-uniform bulk test, combined by the producer over the 3 x 3 (x 3
    // planes) rows around row ty
    const int flag = rowflag[s1 * Sh::NWF + ty * Sh::WC + wc];
    const bool bulk = flag != 0;
    int code = 0;
    if (active) {
      acc.st[0] = stage(s0);
      acc.st[1] = stage(s1);
      acc.st[2] = stage(s2);
      Real pn[NP], mn[NM];
      bool write_phi = true;
      if (bulk) {
        bulk_cell<DIM, NP, NM, Real>(acc, g, flag - 1, pn, mn);
        code = flag;
        write_phi = (sprev[(k * TY + ty) * Sh::WC + wc] & kCodePhase) != flag;
      } else {
        DiffPrm<Real, StepArgs<Real, NP, NM>::P> dp;
        dp.mob = g.mob;
#pragma unroll
        for (int p = 0; p < StepArgs<Real, NP, NM>::P; ++p) dp.delta[p] = g.delta[p];
        gp_cell<DIM, NP, NM, Real, Real>(acc, g, dp, (DIM == 3 ? z : y) + g.zorg, lab_cell<DIM>(g, x, y, z), pn,
                                         mn);
        uint32_t nzm = 0, one = 0;
#pragma unroll
        for (int a = 0; a < NP; ++a) {
          nzm |= (pn[a] != Real(0) ? 1u : 0u) << a;
          one |= (pn[a] == Real(1) ? 1u : 0u) << a;
        }
        code = (__popc(nzm) == 1 && nzm == one) ? __ffs(nzm) : 0;
      }
      store_cell<DIM>(g, x, y, z, pn, mn, write_phi);
    }
    // segment code of the output row: lane 0 is active whenever any lane is
    const int ref = __shfl_sync(0xffffffffu, code, 0);
    const bool same = __all_sync(0xffffffffu, !active || code == ref);
    if (lane == 0) {
      if (active)
        g.codes_out[((long long)(z + g.zoff) * g.ny + y) * g.segs + seg] = same ? (uint8_t)ref : (uint8_t)0;
      if constexpr (DIM == 3) mbar_arrive(&empty[s0]);   // this warp is done with entry k
    }
    if constexpr (DIM == 3) {
      s0 = s1;
      s1 = s2;
      if (++s2 == NST) {
        s2 = 0;
        par2 ^= 1u;
      }
    }
  }
}

// Segment codes of a whole state (used when a state is loaded from outside):
// one warp per 32-cell segment of one row.
template <int DIM, int NP, class Real>
__global__ void __launch_bounds__(256) k_codes(const Real* __restrict__ st, int nx, int ny, int nz,
                                               int pitch, int nyp, long long fstride, int xoff,
                                               int zoff, int segs, uint8_t* __restrict__ codes) {
  // codes[((z + zoff) * ny + y) * segs + s] for the interior planes
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const long long nseg = (long long)segs * ny * nz;
  if (w >= nseg) return;
  const int s = (int)(w % segs);
  const int y = (int)((w / segs) % ny);
  const int z = (int)(w / ((long long)segs * ny));
  const int x = s * 32 + lane;
  const bool active = x < nx;
  int code = 0;
  if (active) {
    const long long i0 = (long long)(z + zoff) * nyp * pitch + (long long)(y + 1) * pitch + x + xoff;
    uint32_t nzm = 0, one = 0;
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      const Real v = st[a * fstride + i0];
      nzm |= (v != Real(0) ? 1u : 0u) << a;
      one |= (v == Real(1) ? 1u : 0u) << a;
    }
    code = (__popc(nzm) == 1 && nzm == one) ? __ffs(nzm) : 0;
  }
  const int ref = __shfl_sync(0xffffffffu, code, 0);
  const bool same = __all_sync(0xffffffffu, !active || code == ref);
  if (lane == 0) codes[((long long)(z + zoff) * ny + y) * segs + s] = same ? (uint8_t)ref : (uint8_t)0;
}

}  // namespace msgb
