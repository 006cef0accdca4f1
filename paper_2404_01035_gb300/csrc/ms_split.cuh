// Split 3-D step (FP32): a streaming kernel that updates every 32-cell row
// segment whose stencil lies in one pure phase, and lists the others for the
// interface kernel, which applies the full cell update (Sec. 2.1) to them.
//
// Bulk rows (MICROSIM paper, arXiv 2404.01035, Sec. 2.1 with a single
// phase present): every q_ab vanishes and the projection keeps the vertex,
// so phi^{n+1} = phi^n, and the mu update of Eq. (Mu_explicit_temperature)
// reduces to the constant-coefficient form mu + Kb_l Lap(mu) - eb_l with
// M = D^l chi^l, chi = chi^l and dh = 0.  The streaming kernel therefore
// reads only mu (phi is the pure phase the segment codes name) and writes phi
// only where the output buffer does not already hold it.
#pragma once

#include "ms_step.cuh"

namespace msgb {

// ---------------------------------------------------------------- streaming
// Each consumer thread updates 4 consecutive cells of one row (16-byte shared
// loads and global stores), a warp one 128-cell row of the tile; one producer
// warp streams the mu planes of the tile through a TMA ring and derives the
// per-segment bulk flags from the segment codes.
template <int NP, int NM, int TY>
struct StreamShape {
  static constexpr int VEC = 4;                   // cells per thread (float4)
  static constexpr int TX = 32 * VEC;             // cells per warp row
  static constexpr int WCS = TX / 32;             // 32-cell segments per warp row
  static constexpr int H = 4;                     // 16-byte halo of the TMA box
  static constexpr int SX = TX + 2 * H;
  static constexpr int SY = TY + 2;
  static constexpr int NCW = TY;                  // consumer warps, one per row
  static constexpr int NT = 32 * NCW;
  static constexpr int NTHREADS = NT + 32;
  static constexpr int FSTRIDE = SY * SX;         // elements per field in a stage
  static constexpr int STAGE_BYTES = NM * FSTRIDE * 4;
  static constexpr int STAGE_STRIDE = (STAGE_BYTES + 127) / 128 * 128;
  static constexpr int NST_RAW = (44 * 1024) / STAGE_STRIDE;   // 4 CTAs per SM
  static constexpr int NST = NST_RAW < 4 ? 4 : (NST_RAW > 12 ? 12 : NST_RAW);
  static constexpr int NFL = SY * WCS;            // row flags per entry (one per producer lane)
  static constexpr int NWF = TY * WCS;            // combined flags per entry
  static constexpr int CSEG = WCS + 2;
  static constexpr int CODE_ENTRIES = (kMaxZChunk + 2) * SY * CSEG;
  static constexpr int OFF_FLAG = NST * STAGE_STRIDE;
  static constexpr int OFF_CODE = OFF_FLAG + (NST * NWF + 15) / 16 * 16;
  static constexpr int NCOEF = NM * NM + NM;     // Kb_l and eb_l of one phase
  static constexpr int OFF_COEF = OFF_CODE + (CODE_ENTRIES + 15) / 16 * 16;
  static constexpr int OFF_BAR = OFF_COEF + (NP * NCOEF * 4 + 15) / 16 * 16;
  static constexpr int OFF_ABORT = OFF_BAR + 2 * NST * 8;
  static constexpr int SMEM_BYTES = OFF_ABORT + 16 + 128;
  static constexpr int MIN_BLOCKS = 4;
  static_assert(NFL <= 32, "the producer warp holds one row flag per lane");
};

// Four cells' worth of one field.
__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void stg4(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}

template <int NP, int NM, int TY>
__global__ void __launch_bounds__(StreamShape<NP, NM, TY>::NTHREADS, StreamShape<NP, NM, TY>::MIN_BLOCKS)
    k_gp_stream(const __grid_constant__ CUtensorMap tm, const __grid_constant__ StepArgs<float, NP, NM> g) {
  using Sh = StreamShape<NP, NM, TY>;
  constexpr int NST = Sh::NST;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  uint8_t* rowflag = smem + Sh::OFF_FLAG;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Sh::OFF_BAR);
  uint64_t* empty = full + NST;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + Sh::OFF_ABORT);
  auto stage = [&](int s) { return reinterpret_cast<float*>(smem + s * Sh::STAGE_STRIDE); };

  const int tid = threadIdx.x, lane = tid & 31;
  const int tiles_x = (g.nx + Sh::TX - 1) / Sh::TX;
  const int x0 = (blockIdx.x % tiles_x) * Sh::TX;
  const int y0 = (blockIdx.x / tiles_x) * TY;
  const int zb = blockIdx.y * g.zchunk;
  const int ze = min(g.nz, zb + g.zchunk);
  const int nplanes = ze - zb + 2;   // ring entries j <-> plane zb - 1 + j
  const int nk = ze - zb;
  if (nplanes > kMaxZChunk + 2) {   // the host clamps z-chunks; never touch smem beyond its size
    if (tid == 0) atomicOr(g.status, kStatusLaunch);
    return;
  }
  const int seg0 = x0 >> 5;

  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], Sh::NCW);
    }
    *abort_flag = 0;
    mbar_fence_init();
  }
  // bulk coefficients of every phase (indexed by the flag below)
  float* scoef = reinterpret_cast<float*>(smem + Sh::OFF_COEF);
  if (tid < NP * Sh::NCOEF) {
    const int a = tid / Sh::NCOEF, r = tid % Sh::NCOEF;
    scoef[tid] = r < NM * NM ? g.Kb[a][r] : g.eb[a][r - NM * NM];
  }
  __syncthreads();

  // The producer starts the first ring entries (their flags are published by
  // a plain arrive later); every thread loads the segment codes the CTA needs
  // (input state, with halo).
  const int npre = nplanes < NST ? nplanes : NST;
  if (tid == Sh::NT) {
    prefetch_tensormap(&tm);
    for (int j = 0; j < npre; ++j) {
      mbar_expect_tx_only(&full[j], Sh::STAGE_BYTES);
      tma_load_4d(stage(j), &tm, &full[j], x0 + g.xoff - Sh::H, y0, zb - 1 + j + g.zoff, 0);
    }
  }
  {
    // thread (pair, group): segment k of row ay (boundary-mapped once), for
    // the entries j = group, group + GROUPS, ... of this CTA's planes
    constexpr int PAIRS = Sh::SY * Sh::CSEG;
    constexpr int GROUPS = Sh::NTHREADS / PAIRS;
    static_assert(GROUPS >= 1, "the code preload needs one thread per (row, segment)");
    uint8_t* scode = smem + Sh::OFF_CODE;
    if (tid < GROUPS * PAIRS) {
      const int pr = tid % PAIRS, j0 = tid / PAIRS;
      const int k = pr % Sh::CSEG, ay = pr / Sh::CSEG;
      const long long rowoff =
          (long long)bc_map(y0 - 1 + ay, g.ny, g.bc[1]) * g.segs + bc_map(seg0 - 1 + k, g.segs, g.bc[0]);
      const long long pstride = (long long)g.ny * g.segs;
#pragma unroll 4
      for (int j = j0; j < nplanes; j += GROUPS) {
        const int z = zb - 1 + j;
        int zz;   // as load_code: ghost code planes at internal cuts
        if (z >= 0 && z < g.nz)
          zz = z + g.zoff;
        else if (g.bc[2] == kBcHalo)
          zz = z < 0 ? 0 : g.nz + 1;
        else
          zz = bc_map(z, g.nz, g.bc[2]) + g.zoff;
        scode[(j * Sh::SY + ay) * Sh::CSEG + k] = __ldg(g.codes_in + zz * pstride + rowoff);
      }
    }
  }
  __syncthreads();   // the last CTA-wide barrier: roles split below

  if (tid >= Sh::NT) {
    // ---------------- producer warp: TMA loads + bulk flags of every entry
    const int f_ay = lane / Sh::WCS, f_wc = lane % Sh::WCS;
    // a segment cut by the end of a ragged row is never bulk: it goes to the
    // interface list, so that bulk groups are always 4 whole cells
    const bool fl = lane < Sh::NFL && (seg0 + f_wc + 1) * 32 <= g.nx;
    const uint8_t* scode = smem + Sh::OFF_CODE;
    int issued = npre, arrived = 0;
    bool ok = true;
    int rf2 = 0, rf1 = 0, rf0 = 0;   // row flags of entries j-2, j-1, j
    for (int j = 0; j < nplanes; ++j) {
      const int s = j % NST;
      if (j >= NST) {
        ok = ok && mbar_wait_bounded(&empty[s], ((j / NST) - 1) & 1);
        ok = ok && *abort_flag == 0;
        if (__any_sync(0xffffffffu, !ok)) break;
        if (lane == 0) {
          mbar_expect_tx_only(&full[s], Sh::STAGE_BYTES);
          tma_load_4d(stage(s), &tm, &full[s], x0 + g.xoff - Sh::H, y0, zb - 1 + j + g.zoff, 0);
        }
        issued = j + 1;
      }
      rf2 = rf1;
      rf1 = rf0;
      rf0 = fl ? combine_codes(scode + (j * Sh::SY + f_ay) * Sh::CSEG + f_wc) : 0;
      // flag of segment wc of row ty at the centre entry j-1: the pure phase
      // + 1 when the 3 x 3 x 3 segments around it all hold that phase
      const int pc = (rf2 == rf1 && rf1 == rf0) ? rf1 : 0;
      const int up = __shfl_down_sync(0xffffffffu, pc, Sh::WCS);
      const int up2 = __shfl_down_sync(0xffffffffu, pc, 2 * Sh::WCS);
      if (lane < Sh::NWF && j >= 1)
        rowflag[((j - 1) % NST) * Sh::NWF + lane] = (uint8_t)((pc == up && up == up2) ? pc : 0);
      __syncwarp();
      if (lane == 0) {
        __threadfence_block();
        mbar_arrive(&full[s]);   // publishes the flags; the data lands by complete_tx
      }
      arrived = j + 1;
    }
    if (!ok && lane == 0) {
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

  // -------------------- consumer warps: 4 cells per thread, one plane at a time
  const int ty = tid >> 5;
  const int wc = lane >> 3;              // segment of this thread within the row
  const int seg = seg0 + wc;
  const int xs = x0 + 4 * lane;          // first of this thread's cells
  const int y = y0 + ty;
  const bool have = y < g.ny && xs < g.nx;
  // a bulk flag implies 4 whole cells (x ghost images of the first / last
  // cell of the row are added as single stores)
  const long long oxl = xs == 0 ? (g.bc[0] == 3 ? g.nx : -1) : 0;                // image of cell q = 0
  const long long oxr = xs + 3 == g.nx - 1 ? (g.bc[0] == 3 ? -g.nx : 1) : 0;     // image of cell q = 3
  const bool leader = (lane & 7) == 0 && y < g.ny && seg < g.segs;
  const long long plane = (long long)g.nyp * g.pitch;
  float* const out0 = g.out + (long long)(zb + g.zoff) * plane + (long long)(y + 1) * g.pitch + xs + g.xoff;
  const long long oy0 = y == 0 ? (long long)(g.bc[1] == 3 ? g.ny : -1) * g.pitch : 0;
  const long long oy1 = y == g.ny - 1 ? (long long)(g.bc[1] == 3 ? -g.ny : 1) * g.pitch : 0;
  const long long cplane = (long long)g.ny * g.segs;
  // z image offsets of the first / last plane of the grid (internal cuts get
  // their ghost planes from the exchange)
  const long long oz_first = g.bc[2] == kBcHalo ? 0 : (g.bc[2] == 3 ? g.nz : -1) * plane;
  const long long oz_last = g.bc[2] == kBcHalo ? 0 : (g.bc[2] == 3 ? -g.nz : 1) * plane;
  uint8_t* const code0 = g.codes_out + ((long long)(zb + g.zoff) * g.ny + y) * g.segs + seg;
  // input code of this thread's segment at plane k: entry k + 1, row ty + 1,
  // segment wc + 1 of the shared copy
  const uint8_t* const scentre = smem + Sh::OFF_CODE + (Sh::SY + ty + 1) * Sh::CSEG + wc + 1;
  const int reuse = g.reuse_prev ? kCodeReuse : 0;
  const int sidx = (ty + 1) * Sh::SX + Sh::H + 4 * lane;
  bool ok = mbar_wait_bounded(&full[0], 0) && mbar_wait_bounded(&full[1], 0);
  int s0 = 0, s1 = 1, s2 = 2 % NST;
  uint32_t par2 = (2 / NST) & 1;
  for (int k = 0; k < nk; ++k) {
    ok = ok && mbar_wait_bounded(&full[s2], par2) && *abort_flag == 0;
    if (!__all_sync(0xffffffffu, ok)) {   // the warp leaves together (shuffles below)
      if (lane == 0) {
        atomicOr(g.status, kStatusTimeout);
        *abort_flag = 1;
      }
      return;
    }
    const int z = zb + k;
    const int flag = rowflag[s1 * Sh::NWF + ty * Sh::WCS + wc];
    // stencil sums of every lane (warp-uniform: the x neighbours come by
    // shuffle; lanes outside the grid read zero-filled box cells)
    float L[NM][4], mc[NM][4];
    {
      const float* c0 = stage(s0) + sidx;
      const float* c1 = stage(s1) + sidx;
      const float* c2 = stage(s2) + sidx;
#pragma unroll
      for (int i = 0; i < NM; ++i) {
        const int fo = i * Sh::FSTRIDE;
        const float4 c = lds4(c1 + fo);
        // x neighbours of the group: from the adjacent lanes, the box halo at the ends
        float xm = __shfl_up_sync(0xffffffffu, c.w, 1), xp = __shfl_down_sync(0xffffffffu, c.x, 1);
        if (lane == 0) xm = c1[fo - 1];
        if (lane == 31) xp = c1[fo + 4];
        const float4 n = lds4(c1 + fo - Sh::SX), sN = lds4(c1 + fo + Sh::SX);
        const float4 d = lds4(c0 + fo), u = lds4(c2 + fo);
        const float cv[4] = {c.x, c.y, c.z, c.w};
        const float lv[4] = {xm, c.x, c.y, c.z}, rv[4] = {c.y, c.z, c.w, xp};
        const float nv[4] = {n.x, n.y, n.z, n.w}, sv[4] = {sN.x, sN.y, sN.z, sN.w};
        const float dv[4] = {d.x, d.y, d.z, d.w}, uv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          mc[i][q] = cv[q];
          float sum = (lv[q] + rv[q]) + (nv[q] + sv[q]);
          sum += dv[q] + uv[q];
          L[i][q] = sum - 6.0f * cv[q];
        }
      }
    }
    if (flag != 0 && have) {
      const int l = flag - 1;
      const float* cf = scoef + l * Sh::NCOEF;
      float mn[NM][4];
#pragma unroll
      for (int i = 0; i < NM; ++i) {
        const float eb = cf[NM * NM + i];
        float kb[NM];
#pragma unroll
        for (int j = 0; j < NM; ++j) kb[j] = cf[i * NM + j];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float dd = mc[i][q] - eb;
#pragma unroll
          for (int j = 0; j < NM; ++j) dd += kb[j] * L[j][q];
          mn[i][q] = dd;
        }
      }
      // a bulk flag implies that the input held phase l here; the output
      // buffer (the state before it) also did when the input's reuse bit is set
      const bool write_phi = (scentre[k * Sh::SY * Sh::CSEG] & reuse) == 0;
      float* p = out0 + k * plane;
      const long long fs = g.fstride;
      // the cell row
      if (write_phi) {
#pragma unroll
        for (int a = 0; a < NP; ++a) {
          const float v = a == l ? 1.0f : 0.0f;
          stg4(p + a * fs, v, v, v, v);
        }
      }
#pragma unroll
      for (int i = 0; i < NM; ++i) stg4(p + (NP + i) * fs, mn[i][0], mn[i][1], mn[i][2], mn[i][3]);
      // x ghost images of the row's first / last cell (lanes 0 and 31 of the
      // tiles at the x ends)
      if (oxl | oxr) {
#pragma unroll
        for (int a = 0; a < NP + NM; ++a) {
          if (a < NP && !write_phi) continue;
          const float v0 = a < NP ? (a == l ? 1.0f : 0.0f) : mn[a < NP ? 0 : a - NP][0];
          const float v3 = a < NP ? (a == l ? 1.0f : 0.0f) : mn[a < NP ? 0 : a - NP][3];
          if (oxl) p[oxl + a * fs] = v0;
          if (oxr) p[3 + oxr + a * fs] = v3;
        }
      }
      // rows at a y or z boundary (rare): their y / z images, with x images
      const long long oz0 = z == 0 ? oz_first : 0, oz1 = z == g.nz - 1 ? oz_last : 0;
      if ((oy0 | oy1 | oz0 | oz1) != 0) {
        // (the loops are unrolled so that every array index is a constant
        // and nothing lives in local memory)
        const long long oy[3] = {0, oy0, oy1}, oz[3] = {0, oz0, oz1};
#pragma unroll
        for (int iz = 0; iz < 3; ++iz)
#pragma unroll
          for (int iy = 0; iy < 3; ++iy) {
            if ((iy | iz) == 0 || (iy && !oy[iy]) || (iz && !oz[iz])) continue;
            float* q = p + oy[iy] + oz[iz];
#pragma unroll
            for (int a = 0; a < NP + NM; ++a) {
              if (a < NP && !write_phi) continue;
              float c4[4];
              if (a < NP) {
                const float v = a == l ? 1.0f : 0.0f;
                c4[0] = c4[1] = c4[2] = c4[3] = v;
              } else {
#pragma unroll
                for (int u = 0; u < 4; ++u) c4[u] = mn[a - NP][u];
              }
              stg4(q + a * fs, c4[0], c4[1], c4[2], c4[3]);
              if (oxl) q[oxl + a * fs] = c4[0];
              if (oxr) q[3 + oxr + a * fs] = c4[3];
            }
          }
      }
    }
    // segment codes of bulk segments (input and output pure phase l: reuse
    // bit set); the others go to the interface list
    if (leader && flag != 0) code0[k * cplane] = (uint8_t)(flag | kCodeReuse);
    const unsigned int need = __ballot_sync(0xffffffffu, leader && flag == 0);
    if (need) {
      const int first = __ffs(need) - 1;
      unsigned int base = 0;
      if (lane == first) base = atomicAdd(&g.iface[0], (unsigned int)__popc(need));
      base = __shfl_sync(0xffffffffu, base, first);
      if ((need >> lane) & 1u) {
        const unsigned int i = base + __popc(need & ((1u << lane) - 1u));
        if (i < g.iface_cap)
          g.iface[2 + i] = ((unsigned int)z << (g.seg_bits + g.y_bits)) | ((unsigned int)y << g.seg_bits) |
                           (unsigned int)seg;
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s0]);   // this warp is done with entry k
    s0 = s1;
    s1 = s2;
    if (++s2 == NST) {
      s2 = 0;
      par2 ^= 1u;
    }
  }
}

// Phases the compact update of the interface kernel handles (more phases
// than this around a row take the full update).
constexpr int kSparseK = 4;

// Interface kernel of the split 3-D step (shape of its shared memory).  Each
// warp owns two buffers of one TMA box: 32 + 2H cells x 3 rows x 3 planes x
// all fields around one listed 32-cell row, so the next row is in flight
// while the current one is updated.
template <int NP, int NM, class Real>
struct IfaceShape {
  static constexpr int NF = NP + NM;
  static constexpr int H = Halo<Real>::H;
  static constexpr int BX = 32 + 2 * H;                 // box extent along x
  static constexpr int BOX_ELEMS = NF * 9 * BX;
  static constexpr int BOX_BYTES = BOX_ELEMS * (int)sizeof(Real);
  static constexpr int BOX_STRIDE = (BOX_BYTES + 127) / 128 * 128;
  static constexpr int WARPS = 4;                       // warps per CTA
  static constexpr int THREADS = 32 * WARPS;
  static constexpr int OFF_BAR = WARPS * 2 * BOX_STRIDE;
  static constexpr int SMEM_BYTES = OFF_BAR + WARPS * 2 * 8 + 128;   // + alignment slack
  static constexpr int MIN_BLOCKS = NP <= 4 ? 3 : 2;
};

// Stencil accessor over one interface box ([field][plane][row][x]).
template <int DIM, int NP, int NM, class Real>
struct BoxAcc {
  using Sh = IfaceShape<NP, NM, Real>;
  const Real* s;
  const StepArgs<Real, NP, NM>* g;
  int sidx;         // centre of this lane's cell: plane 1, row 1, x = H + lane
  uint32_t wmask;   // phases present anywhere in the warp's box (a superset of
                    // each cell's stencil: absent phases then contribute exact
                    // zeros, so the update is the same as with the cell's own)

  __device__ __forceinline__ Real ld(int f, int dx, int dy, int dz) const {
    return s[f * (9 * Sh::BX) + sidx + dz * (3 * Sh::BX) + dy * Sh::BX + dx];
  }
  __device__ __forceinline__ Real phi(int a, int dx, int dy, int dz) const { return ld(a, dx, dy, dz); }
  __device__ __forceinline__ Real mu(int i, int dx, int dy, int dz) const { return ld(NP + i, dx, dy, dz); }
  __device__ __forceinline__ uint32_t mask() const { return wmask; }
  __device__ __forceinline__ void mobility(int dx, int dy, int dz, Real* M) const {
    Real ph[NP];
#pragma unroll
    for (int a = 0; a < NP; ++a) ph[a] = phi(a, dx, dy, dz);
    cell_mobility<NP, NM>(ph, g->DX, M);
  }
};

// Phases present anywhere in an interface box, OR-ed over the warp (every
// lane its own column of the 3 x 3 rows, lanes 0 and 31 also the halo column
// on their side).  Called by all lanes of the warp.
template <int NP, int NM, class Real>
__device__ __forceinline__ uint32_t box_phase_mask(const Real* box, int lane) {
  using Sh = IfaceShape<NP, NM, Real>;
  uint32_t m = 0;
  if constexpr (sizeof(Real) == 4) {
    // phase fractions are never negative: the OR of the bit patterns is
    // non-zero exactly when some value is (a -0.0 could only mark a phase
    // present, which costs work, never correctness)
    const unsigned int* bx = reinterpret_cast<const unsigned int*>(box);
    const int xh = lane == 0 ? Sh::H - 1 : Sh::H + 32;
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      unsigned int any = 0u;
#pragma unroll
      for (int r = 0; r < 9; ++r) any |= bx[a * (9 * Sh::BX) + r * Sh::BX + Sh::H + lane];
      if (lane == 0 || lane == 31) {
#pragma unroll
        for (int r = 0; r < 9; ++r) any |= bx[a * (9 * Sh::BX) + r * Sh::BX + xh];
      }
      m |= (any != 0u ? 1u : 0u) << a;
    }
  } else {
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      bool any = false;
#pragma unroll
      for (int r = 0; r < 9; ++r) any = any || box[a * (9 * Sh::BX) + r * Sh::BX + Sh::H + lane] != Real(0);
      if (lane == 0 || lane == 31) {
        const int xh = lane == 0 ? Sh::H - 1 : Sh::H + 32;
#pragma unroll
        for (int r = 0; r < 9; ++r) any = any || box[a * (9 * Sh::BX) + r * Sh::BX + xh] != Real(0);
      }
      m |= (any ? 1u : 0u) << a;
    }
  }
  return __reduce_or_sync(0xffffffffu, m);
}

// Scan of an interface box by the warp: lane = column H + lane of the 3 x 3
// rows; lanes 0..17 also take one cell of the halo column on either side
// (lanes 0..8 the left one, 9..17 the right one, row lane % 9).  Returns the
// phases present anywhere in the box (OR over the warp: a superset of every
// cell's stencil) and sets `bulk` to l + 1 when every cell of the 3 x 3 x 3
// block around the lane's cell is exactly pure phase l (phi_l = 1, all others
// 0), else 0.  Called by all lanes of the warp.
template <int NP, int NM, class Real>
__device__ __forceinline__ uint32_t box_scan(const Real* box, int lane, int& bulk) {
  using Sh = IfaceShape<NP, NM, Real>;
  uint32_t m = 0;
  // pure code of one box cell (l + 1 or 0); ORs its nonzero phases into nzm
  auto code_of = [&](int r, int x, uint32_t& nzm) {
    uint32_t nz = 0, one = 0;
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      const Real v = box[a * (9 * Sh::BX) + r * Sh::BX + x];
      nz |= (v != Real(0) ? 1u : 0u) << a;
      one |= (v == Real(1) ? 1u : 0u) << a;
    }
    nzm |= nz;
    return (__popc(nz) == 1 && nz == one) ? __ffs(nz) : 0;
  };
  int col = code_of(0, Sh::H + lane, m);   // common code of the lane's 9 cells, or 0
#pragma unroll
  for (int r = 1; r < 9; ++r) {
    const int c = code_of(r, Sh::H + lane, m);
    col = c == col ? col : 0;
  }
  uint32_t hm = 0;
  const int hc = code_of(lane % 9, lane < 9 ? Sh::H - 1 : Sh::H + 32, hm);
  if (lane < 18) m |= hm;
  const uint32_t wmask = __reduce_or_sync(0xffffffffu, m);
  const int lc = __shfl_sync(0xffffffffu, hc, 0), rc = __shfl_sync(0xffffffffu, hc, 9);
  const uint32_t lb = __ballot_sync(0xffffffffu, lane < 9 && hc == lc);
  const uint32_t rb = __ballot_sync(0xffffffffu, lane >= 9 && lane < 18 && hc == rc);
  int left = __shfl_up_sync(0xffffffffu, col, 1), right = __shfl_down_sync(0xffffffffu, col, 1);
  if (lane == 0) left = lb == 0x1FFu ? lc : 0;
  if (lane == 31) right = rb == (0x1FFu << 9) ? rc : 0;
  bulk = (col != 0 && left == col && right == col) ? col : 0;
  return wmask;
}

// Bulk update of one cell of an interface box whose 3 x 3 x 3 block is pure
// phase l (c = the cell in field 0, cf = Kb_l then eb_l): phi unchanged and
// mu + Kb_l Lap(mu) - eb_l, the form of the streaming kernel.
template <int NP, int NM, class Real>
__device__ __forceinline__ void box_bulk_mu(const Real* c, const Real* cf, Real* mn) {
  using Sh = IfaceShape<NP, NM, Real>;
  Real L[NM], mc[NM];
#pragma unroll
  for (int i = 0; i < NM; ++i) {
    const Real* f = c + (NP + i) * (9 * Sh::BX);
    const Real v = f[0];
    Real sum = (f[-1] + f[1]) + (f[-Sh::BX] + f[Sh::BX]);
    sum += f[-3 * Sh::BX] + f[3 * Sh::BX];
    L[i] = sum - Real(6) * v;
    mc[i] = v;
  }
#pragma unroll
  for (int i = 0; i < NM; ++i) {
    Real dd = mc[i] - cf[NM * NM + i];
#pragma unroll
    for (int j = 0; j < NM; ++j) dd += cf[i * NM + j] * L[j];
    mn[i] = dd;
  }
}

// Interface kernel of the split 3-D step: the full cell update of every warp
// row the streaming kernel listed (32 cells of one row of one plane per
// warp), from a TMA box of the input state; writes phi, mu, their ghost
// images and the row's segment code.  With more than kSparseK phases the
// work is shared by two launches: MODE 0 takes the rows whose box holds at
// most kSparseK phases (the compact update) and moves the others to a second
// list, which MODE 1 updates with the full one (each kernel's registers then
// fit its own path).  The last CTA to finish clears its list (ticket in
// list[1]), so the launches can be replayed from a CUDA graph.
template <int DIM, int NP, int NM, class Real, int MODE, int FEAT = kFeatAll>
__global__ void __launch_bounds__(IfaceShape<NP, NM, Real>::THREADS, IfaceShape<NP, NM, Real>::MIN_BLOCKS)
    k_gp_iface(const __grid_constant__ CUtensorMap tmi, const __grid_constant__ StepArgs<Real, NP, NM> g) {
  static_assert(DIM == 3, "the interface list is built by the 3-D streaming kernel");
  constexpr bool kSparse = NP > kSparseK && MODE == 0;   // compact update, defer the rest
  unsigned int* const list = MODE == 0 ? g.iface : g.iface2;
  using Sh = IfaceShape<NP, NM, Real>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  __shared__ unsigned int s_count;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Sh::OFF_BAR) + 2 * wid;
  Real* buf0 = reinterpret_cast<Real*>(smem + (2 * wid) * Sh::BOX_STRIDE);
  if (threadIdx.x == 0) s_count = min(*(volatile unsigned int*)&list[0], g.iface_cap);
  if (MODE == 0 && g.at_list && blockIdx.x == 0 && threadIdx.x == 0)   // see the copy below
    g.at_list[0] = min(*(volatile unsigned int*)&list[0], g.at_cap);
  if (lane == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
    prefetch_tensormap(&tmi);
  }
  __syncthreads();
  const unsigned int count = s_count;
  const unsigned int stride = gridDim.x * Sh::WARPS;
  DiffPrm<Real, StepArgs<Real, NP, NM>::P> dp;
  dp.mob = g.mob;
#pragma unroll
  for (int p = 0; p < StepArgs<Real, NP, NM>::P; ++p) dp.delta[p] = g.delta[p];

  // list entry r -> (segment, y, z) (bit fields)
  const unsigned int seg_mask = (1u << g.seg_bits) - 1u, y_mask = (1u << g.y_bits) - 1u;
  const int zshift = g.seg_bits + g.y_bits;
  // row -> box origin (x, y - 1, z - 1 in padded coordinates)
  auto issue = [&](unsigned int i, int b) {
    const unsigned int r = list[2 + i];
    const int sg = (int)(r & seg_mask);
    const int y = (int)((r >> g.seg_bits) & y_mask), z = (int)(r >> zshift);
    fence_proxy_async_shared();
    mbar_expect_tx(&bar[b], Sh::BOX_BYTES);
    tma_load_4d(reinterpret_cast<unsigned char*>(buf0) + b * Sh::BOX_STRIDE, &tmi, &bar[b],
                32 * sg + g.xoff - Sh::H, y, z + g.zoff - 1, 0);
  };
  // bit b of `pending` / `phase`: buffer b has a copy in flight / the
  // parity its barrier completes next (bits, not arrays: a runtime index
  // would put them in local memory)
  uint32_t pending = 0u, phase = 0u;
  bool aborted = false;
  unsigned int i = blockIdx.x * Sh::WARPS + wid;
  if (i < count && lane == 0) issue(i, 0);
  if (i < count) pending = 1u;
  int b = 0;
  while (i < count) {
    const unsigned int nxt = i + stride;
    if (nxt < count) {
      if (lane == 0) issue(nxt, b ^ 1);
      pending |= 1u << (b ^ 1);
    }
    const bool ok = mbar_wait_bounded(&bar[b], (phase >> b) & 1u);
    if (!__all_sync(0xffffffffu, ok)) {
      aborted = true;
      break;
    }
    pending &= ~(1u << b);
    phase ^= 1u << b;
    const unsigned int r = list[2 + i];
    const int sg = (int)(r & seg_mask);
    const int y = (int)((r >> g.seg_bits) & y_mask), z = (int)(r >> zshift);
    // with the anti-trapping current on, its correction works on the same
    // segments (a block of segments that is not one pure phase in phi^n, plus
    // cut segments, where the current vanishes): the list is copied, by
    // linear segment index, at the same positions
    if (MODE == 0 && g.at_list && lane == 0 && i < g.at_cap)
      g.at_list[2 + i] = (unsigned int)(((long long)z * g.ny + y) * g.segs + sg);
    const int x = 32 * sg + lane;
    const bool active = x < g.nx;
    const Real* box = reinterpret_cast<const Real*>(reinterpret_cast<unsigned char*>(buf0) + b * Sh::BOX_STRIDE);
    uint32_t wmask;
    if constexpr (kSparse) {
      // many phases: rows whose cells all have a pure 3 x 3 x 3 block (listed
      // only because a segment next to them is not pure) take the bulk update
      int bk = 0;
      wmask = box_scan<NP, NM, Real>(box, lane, bk);
      if (__all_sync(0xffffffffu, !active || bk != 0)) {
        if (active) {
          Real pn[NP], mn[NM], cf[NM * NM + NM];
#pragma unroll
          for (int a = 0; a < NP; ++a) pn[a] = a == bk - 1 ? Real(1) : Real(0);
#pragma unroll
          for (int k = 0; k < NM * NM; ++k) cf[k] = g.Kb[bk - 1][k];
#pragma unroll
          for (int k = 0; k < NM; ++k) cf[NM * NM + k] = g.eb[bk - 1][k];
          box_bulk_mu<NP, NM, Real>(box + 4 * Sh::BX + Sh::H + lane, cf, mn);
          store_cell<DIM>(g, x, y, z, pn, mn);
        }
        const int ref = __shfl_sync(0xffffffffu, bk, 0);
        const bool same = __all_sync(0xffffffffu, !active || bk == ref);
        if (lane == 0) {
          const long long ci = ((long long)(z + g.zoff) * g.ny + y) * g.segs + sg;
          int c = same ? ref : 0;
          if (c != 0 && (g.codes_in[ci] & kCodePhase) == c) c |= kCodeReuse;   // pure before and after
          g.codes_out[ci] = (uint8_t)c;
        }
        __syncwarp();
        b ^= 1;
        i = nxt;
        continue;
      }
    } else {
      wmask = box_phase_mask<NP, NM, Real>(box, lane);
    }
    if constexpr (kSparse) {
      if (__popc(wmask) > kSparseK) {   // for the MODE 1 launch
        if (lane == 0) {
          const unsigned int k = atomicAdd(&g.iface2[0], 1u);
          if (k < g.iface_cap) g.iface2[2 + k] = r;
        }
        __syncwarp();
        b ^= 1;
        i = nxt;
        continue;
      }
    }
    int code = 0;
    if (active) {
      BoxAcc<DIM, NP, NM, Real> acc;
      acc.s = box;
      acc.g = &g;
      acc.sidx = 3 * Sh::BX + Sh::BX + Sh::H + lane;
      acc.wmask = wmask;
      Real pn[NP], mn[NM];
      if constexpr (kSparse)   // many phases, at most kSparseK of them around this row
        gp_cell_sparse<DIM, NP, NM, kSparseK, Real, BoxAcc<DIM, NP, NM, Real>, FEAT>(acc, g, z + g.zorg,
                                                                                   lab_cell<DIM>(g, x, y, z), pn, mn);
      else
        gp_cell<DIM, NP, NM, Real, Real, BoxAcc<DIM, NP, NM, Real>, FEAT>(acc, g, dp, z + g.zorg,
                                                                         lab_cell<DIM>(g, x, y, z), pn, mn);
      uint32_t nzm = 0, one = 0;
#pragma unroll
      for (int a = 0; a < NP; ++a) {
        nzm |= (pn[a] != Real(0) ? 1u : 0u) << a;
        one |= (pn[a] == Real(1) ? 1u : 0u) << a;
      }
      code = (__popc(nzm) == 1 && nzm == one) ? __ffs(nzm) : 0;
      store_cell<DIM>(g, x, y, z, pn, mn);
    }
    const int ref = __shfl_sync(0xffffffffu, code, 0);
    const bool same = __all_sync(0xffffffffu, !active || code == ref);
    if (lane == 0) {
      const long long ci = ((long long)(z + g.zoff) * g.ny + y) * g.segs + sg;
      int c = same ? ref : 0;
      if (c != 0 && (g.codes_in[ci] & kCodePhase) == c) c |= kCodeReuse;   // pure before and after
      g.codes_out[ci] = (uint8_t)c;
    }
    __syncwarp();   // every lane is done with buffer b before it is refilled
    b ^= 1;
    i = nxt;
  }
  if (aborted) {
    // a copy did not complete in time: record it and wait (bounded) for the
    // copies still in flight before the CTA exits
    if (lane == 0) {
      atomicOr(g.status, kStatusTimeout);
      for (int k = 0; k < 2; ++k)
        if ((pending >> k) & 1u) mbar_wait_bounded(&bar[k], (phase >> k) & 1u);
    }
  }
  // every CTA read the count before taking its ticket
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&list[1], 1u) == gridDim.x - 1) {
      list[0] = 0u;
      list[1] = 0u;
    }
  }
}

}  // namespace msgb
