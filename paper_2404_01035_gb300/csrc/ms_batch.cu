// Batched form: hundreds of independent 2-D simulations of different sizes
// and parameters advanced by ONE persistent, cooperative kernel launch
// (captured once into a CUDA graph and replayed).
//
// Work list: every (simulation, 32 x TY tile) pair, as precomputed
// descriptors.  Each CTA takes a contiguous range of it every step; a producer
// warp reads the descriptors 32 at a time (one coalesced load, the next chunk
// in flight) and TMA-loads the items' halo'ed tiles (each simulation has its
// own tensor map, kept in global memory) into a shared-memory ring, while the
// consumer warps compute the current one with the same cell update as the
// single-simulation kernel.  A consumer warp takes the bulk update when the
// three halo rows around its row, its 32 columns and the column on each side,
// hold one pure phase in the staged data itself (the exact condition of the
// bulk shortcut; no segment codes are kept).  A grid-wide barrier (atomic
// counter, bounded spin on %globaltimer) separates time steps, because a step
// reads the ghost cells its neighbours wrote in the previous step.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/microsim_gb.h"
#include "ms_launch.cuh"
#include "ms_rt.h"
#include "ms_trace.h"

namespace msgb {

ms_status build_model(ms_ctx* c, const ms_grid* g, int N, int K, const ms_params* p, HostModel& m);

// Per-simulation constants for one buffer parity (out points at the
// destination of a step that reads the other buffer).
template <class Real, int NP, int NM>
struct alignas(64) BatchSim {
  StepArgs<Real, NP, NM> g[2];   // [parity of the source buffer]
};

// One work item: simulation, tile origin, TMA x coordinate of its box.
struct alignas(16) BatchItem {
  int sim, x0, y0, bx;
};

__device__ __forceinline__ bool grid_barrier(unsigned int* counter, unsigned int target) {
  __threadfence();
  fence_proxy_async_global();   // generic stores of this step -> TMA loads of the next
  atomicAdd(counter, 1u);
  const unsigned long long t0 = globaltimer();
  while (atomicAdd(counter, 0u) < target) {
    if (globaltimer() - t0 > kWaitLimitNs) return false;
    __nanosleep(64);
  }
  __threadfence();
  fence_proxy_async_global();
  return true;
}

template <int NP, int NM, class Real, int TX, int TY>
__global__ void __launch_bounds__(TX* TY + 32, TY <= 8 ? 3 : 1)
    k_batch(const BatchSim<Real, NP, NM>* __restrict__ sims, const CUtensorMap* __restrict__ maps,
            const BatchItem* __restrict__ items, int nitems, int nsteps, int parity0,
            unsigned int* barrier, int* status) {
  using Sh = StepShape<2, NP, NM, Real, TX, TY>;
  static_assert(TX == 32, "one warp per tile row");
  constexpr int NST = 8;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  int4* sitem = reinterpret_cast<int4*>(smem + NST * Sh::STAGE_STRIDE);
  uint64_t* full = reinterpret_cast<uint64_t*>(sitem + NST);
  uint64_t* empty = full + NST;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + NST);
  auto stage = [&](int s) { return reinterpret_cast<Real*>(smem + s * Sh::STAGE_STRIDE); };
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], Sh::NCW);
    }
    *abort_flag = 0;
    mbar_fence_init();
  }
  __syncthreads();
  // contiguous item range: consecutive tiles of one simulation share its constants
  const int per = (nitems + (int)gridDim.x - 1) / (int)gridDim.x;
  const int ibeg = min(nitems, (int)blockIdx.x * per);
  const int my_items = min(nitems, ibeg + per) - ibeg;
  long long seq = 0;      // ring position (continues across steps)
  long long issued = 0;   // loads issued (producer lane 0)
  for (int step = 0; step < nsteps; ++step) {
    const int par = (parity0 + step) & 1;
    if (tid >= Sh::NT) {
      // ---------------- producer warp: descriptors 32 at a time, one TMA per item
      auto fetch = [&](int k0) {
        int4 d = make_int4(0, 0, 0, 0);
        if (k0 + lane < my_items) {
          const BatchItem it = items[ibeg + k0 + lane];
          d = make_int4(it.sim, it.x0, it.y0, it.bx);
        }
        return d;
      };
      int4 cur = fetch(0), nxt = fetch(32);
      bool ok = true;
      for (int k = 0; k < my_items; ++k) {
        if ((k & 31) == 0 && k > 0) {
          cur = nxt;
          nxt = fetch(k + 32);
        }
        const long long q = seq + k;
        const int s = (int)(q % NST);
        if (q >= NST) ok = ok && mbar_wait_bounded(&empty[s], (uint32_t)(((q / NST) - 1) & 1));
        ok = ok && *abort_flag == 0;
        if (__any_sync(0xffffffffu, !ok)) {
          if (lane == 0) {
            atomicOr(status, kStatusTimeout);
            *abort_flag = 1;
          }
          break;
        }
        const int j = k & 31;
        const int sim = __shfl_sync(0xffffffffu, cur.x, j);
        const int x0 = __shfl_sync(0xffffffffu, cur.y, j);
        const int y0 = __shfl_sync(0xffffffffu, cur.z, j);
        const int bx = __shfl_sync(0xffffffffu, cur.w, j);
        if (lane == 0) {
          sitem[s] = make_int4(sim, x0, y0, 0);
          __threadfence_block();
          mbar_expect_tx(&full[s], Sh::STAGE_BYTES);   // arrive (release) + expected bytes
          tma_load_4d(stage(s), &maps[2 * sim + par], &full[s], bx, y0, 0, 0);
          issued = q + 1;
        }
      }
    } else {
      // ---------------- consumer warps: one tile row each
      const int tx = tid % TX, ty = tid / TX;
      for (int k = 0; k < my_items; ++k) {
        const long long q = seq + k;
        const int s = (int)(q % NST);
        const bool ok = mbar_wait_bounded(&full[s], (uint32_t)((q / NST) & 1)) && *abort_flag == 0;
        if (!__all_sync(0xffffffffu, ok)) {   // the warp leaves together (votes below)
          if (lane == 0) {
            atomicOr(status, kStatusTimeout);
            *abort_flag = 1;
          }
          break;
        }
        const int4 it = sitem[s];
        const StepArgs<Real, NP, NM>& g = sims[it.x].g[par];
        const int x0 = it.y, y0 = it.z;
        const int x = x0 + tx, y = y0 + ty;
        const bool active = x < g.nx && y < g.ny;
        // bulk test on the staged phi: rows ty..ty+2 (halo'ed) of this lane's
        // column, and of the columns beside the row for lanes 0 and 31
        const Real* st = stage(s);
        auto column_code = [&](int col) {
          int c = -1;
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            uint32_t nz = 0, one = 0;
#pragma unroll
            for (int a = 0; a < NP; ++a) {
              const Real v = st[a * Sh::SY * Sh::SX + (ty + r) * Sh::SX + col];
              nz |= (v != Real(0) ? 1u : 0u) << a;
              one |= (v == Real(1) ? 1u : 0u) << a;
            }
            const int pc = (__popc(nz) == 1 && nz == one) ? __ffs(nz) : 0;
            c = (c == -1 || c == pc) ? pc : 0;
          }
          return c;
        };
        int mine = column_code(Sh::H + tx);
        if (tx == 0 || tx == TX - 1) {
          const int side = column_code(tx == 0 ? Sh::H - 1 : Sh::H + TX);
          mine = mine == side ? mine : 0;
        }
        const int ref = __shfl_sync(0xffffffffu, mine, 0);
        const int flag = __all_sync(0xffffffffu, mine == ref) ? ref : 0;
        if (active) {
          SmemAcc<2, NP, NM, Real, TX, TY> acc;
          acc.st[0] = acc.st[1] = acc.st[2] = st;
          acc.g = &g;
          acc.sidx = (ty + 1) * Sh::SX + tx + Sh::H;
          Real pn[NP], mn[NM];
          if (flag != 0) {
            bulk_cell<2, NP, NM, Real>(acc, g, flag - 1, pn, mn);
          } else {
            DiffPrm<Real, StepArgs<Real, NP, NM>::P> dp;
            dp.mob = g.mob;
#pragma unroll
            for (int p = 0; p < StepArgs<Real, NP, NM>::P; ++p) dp.delta[p] = g.delta[p];
            gp_cell<2, NP, NM, Real, Real>(acc, g, dp, y + g.zorg, lab_cell<2>(g, x, y, 0), pn, mn);
          }
          store_cell<2>(g, x, y, 0, pn, mn);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
      }
    }
    seq += my_items;
    __syncthreads();
    // grid-wide barrier between steps
    if (tid == 0) {
      if (*abort_flag || !grid_barrier(barrier, (unsigned int)(step + 1) * gridDim.x)) {
        atomicOr(status, kStatusTimeout);
        *abort_flag = 1;
      }
    }
    __syncthreads();
    if (*abort_flag) break;
  }
  // drain: every issued load was consumed in a complete run; after an abort,
  // wait (bounded) for the loads still in flight before the CTA exits
  if (*abort_flag && tid == Sh::NT) {
    for (int s = 0; s < NST; ++s) {
      if (issued <= s) continue;
      const long long q = s + ((issued - 1 - s) / NST) * NST;   // last load issued into stage s
      mbar_wait_bounded(&full[s], (uint32_t)((q / NST) & 1));
    }
  }
}

template <int NP, int NM, class Real, int TX, int TY>
struct BatchShape {
  using Sh = StepShape<2, NP, NM, Real, TX, TY>;
  static constexpr int NST = 8;
  static constexpr int SMEM = NST * Sh::STAGE_STRIDE + NST * 16 + 2 * NST * 8 + 16 + 128;
};

}  // namespace msgb

using namespace msgb;

struct ms_batch {
  int nsims = 0, N = 0, NM = 0, dtype = 0;
  std::vector<HostModel> models;
  std::vector<size_t> off;              // byte offset of each simulation's two state buffers
  std::vector<size_t> sbytes;           // state bytes per simulation (one buffer)
  void* state = nullptr;                // all state buffers
  void* sims = nullptr;                 // BatchSim array (device)
  CUtensorMap* maps = nullptr;          // [nsims][2] (device)
  BatchItem* items = nullptr;
  int nitems = 0;
  unsigned int* barrier = nullptr;
  int* status = nullptr;
  int parity = 0;                       // buffer holding the current state
  int64_t steps_done = 0;
  cudaStream_t stream = nullptr;
  AllocHook hook;
  int grid = 0, smem = 0;
  int ty = 0;                           // tile height of the work list (kBTYs)
  cudaGraphExec_t graph = nullptr;
  int64_t graph_n = -1;
  std::string err;
};

namespace {

// Tiles are 32 cells (one warp row) wide; their height is chosen at run time
// among the compiled ones (ms_batch_set_tile / ms_batch_tune).
constexpr int kBTX = 32, kBTY = 8;
constexpr int kBTYs[] = {4, 8, 16};
constexpr int kNBTY = 3;

template <int TY>
void* batch_kernel() {
  return reinterpret_cast<void*>(k_batch<2, 1, float, kBTX, TY>);
}
void* batch_kernel_for(int ty) {
  return ty == 4 ? batch_kernel<4>() : ty == 16 ? batch_kernel<16>() : batch_kernel<8>();
}
int batch_smem_for(int ty) {
  return ty == 4 ? BatchShape<2, 1, float, kBTX, 4>::SMEM
                 : ty == 16 ? BatchShape<2, 1, float, kBTX, 16>::SMEM : BatchShape<2, 1, float, kBTX, 8>::SMEM;
}

ms_status bfail(ms_batch* b, ms_status s, const std::string& m) {
  if (b) b->err = m;
  return fail(nullptr, s, m);
}

void batch_free(ms_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  dev_free(b->hook, b->state);
  dev_free(b->hook, b->sims);
  dev_free(b->hook, b->maps);
  dev_free(b->hook, b->items);
  dev_free(b->hook, b->barrier);
  delete b;
}

cudaError_t launch_batch(ms_batch* b, int64_t n) {
  cudaError_t e = cudaMemsetAsync(b->barrier, 0, sizeof(unsigned int), b->stream);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(b->grid);
  cfg.blockDim = dim3(kBTX * b->ty + 32);
  cfg.dynamicSmemBytes = b->smem;
  cfg.stream = b->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const BatchSim<float, 2, 1>* sims = (const BatchSim<float, 2, 1>*)b->sims;
  const CUtensorMap* maps = (const CUtensorMap*)b->maps;
  const BatchItem* items = (const BatchItem*)b->items;
  if (b->ty == 4)
    return cudaLaunchKernelEx(&cfg, k_batch<2, 1, float, kBTX, 4>, sims, maps, items, b->nitems, (int)n, b->parity,
                              b->barrier, b->status);
  if (b->ty == 16)
    return cudaLaunchKernelEx(&cfg, k_batch<2, 1, float, kBTX, 16>, sims, maps, items, b->nitems, (int)n, b->parity,
                              b->barrier, b->status);
  return cudaLaunchKernelEx(&cfg, k_batch<2, 1, float, kBTX, 8>, sims, maps, items, b->nitems, (int)n, b->parity,
                            b->barrier, b->status);
}

// Work list, tensor maps and persistent grid for tile height ty (one of
// kBTYs): items are (simulation, 32 x ty tile) pairs in simulation order,
// the maps' boxes are the tiles with their halo.  Drops the captured graph.
cudaError_t batch_set_tiles(ms_batch* b, int ty) {
  std::vector<CUtensorMap> hm(2 * b->nsims);
  std::vector<BatchItem> items;
  for (int i = 0; i < b->nsims; ++i) {
    const HostModel& m = b->models[i];
    const size_t half = (b->sbytes[i] + 255) / 256 * 256;
    char* base = static_cast<char*>(b->state) + b->off[i];
    for (int par = 0; par < 2; ++par)
      if (!encode_state_map(&hm[2 * i + par], base + par * half, m, 3, kBTX, ty)) return cudaErrorInvalidValue;
    for (int y0 = 0; y0 < m.ny; y0 += ty)
      for (int x0 = 0; x0 < m.nx; x0 += kBTX) items.push_back(BatchItem{i, x0, y0, x0 + m.xoff - 16 / 4});
  }
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return e;
  dev_free(b->hook, b->items);
  b->items = static_cast<BatchItem*>(dev_alloc(b->hook, sizeof(BatchItem) * items.size()));
  if (!b->items) return cudaErrorMemoryAllocation;
  b->nitems = (int)items.size();
  e = cudaMemcpyAsync(b->items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->maps, hm.data(), sizeof(CUtensorMap) * hm.size(), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  void* kern = batch_kernel_for(ty);
  const int smem = batch_smem_for(ty);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  int per_sm = 0, dev = 0, sms = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBTX * ty + 32, smem);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  b->ty = ty;
  b->smem = smem;
  b->grid = std::max(1, per_sm) * sms;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  b->graph_n = -1;
  return cudaSuccess;
}

}  // namespace

extern "C" {

ms_status ms_batch_create(int nsims, const ms_grid* grids, int n_phases, int n_components,
                          const ms_params* params, void* stream, const ms_allocator* alloc, ms_batch** out) {
  if (!out || nsims < 1 || !grids || !params) return bfail(nullptr, MS_ERR_ARG, "bad batch arguments");
  *out = nullptr;
  ensure_registered();
  ms_batch* b = new ms_batch();
  b->nsims = nsims;
  b->stream = static_cast<cudaStream_t>(stream);
  if (alloc) b->hook = AllocHook{alloc->alloc, alloc->release, alloc->user};
  b->models.resize(nsims);
  for (int i = 0; i < nsims; ++i) {
    ms_status s = build_model(nullptr, &grids[i], n_phases, n_components, &params[i], b->models[i]);
    if (s != MS_OK) {
      std::string m = "simulation " + std::to_string(i) + ": " + ms_last_error(nullptr);
      batch_free(b);
      return bfail(nullptr, s, m);
    }
    HostModel& m = b->models[i];
    if (m.dim != 2 || m.N != 2 || m.NM != 1 || m.dtype != MS_F32) {
      batch_free(b);
      return bfail(nullptr, MS_ERR_UNSUPPORTED, "the batched kernel is compiled for 2-D, N=2, K=2, FP32");
    }
    if (m.noise_amp != 0.0) {
      batch_free(b);
      return bfail(nullptr, MS_ERR_UNSUPPORTED, "batched simulations do not support phi noise (noise_amp != 0)");
    }
    if (m.at || m.gg || m.el) {
      batch_free(b);
      return bfail(nullptr, MS_ERR_UNSUPPORTED,
                   "batched simulations do not support the anti-trapping current, grain growth or elasticity");
    }
    if (m.G * m.V != 0.0) {
      batch_free(b);
      return bfail(nullptr, MS_ERR_UNSUPPORTED, "batched simulations must be isothermal in time (G V = 0)");
    }
    set_layout(m);
  }
  b->N = 2;
  b->NM = 1;
  b->dtype = MS_F32;
  // one allocation for all states (2 buffers each)
  size_t tot = 0;
  for (int i = 0; i < nsims; ++i) {
    const HostModel& m = b->models[i];
    const size_t sb = (size_t)m.fstride * (m.N + m.NM) * 4;
    b->sbytes.push_back(sb);
    b->off.push_back(tot);
    tot += 2 * ((sb + 255) / 256 * 256);
  }
  b->state = dev_alloc(b->hook, tot);
  b->sims = dev_alloc(b->hook, sizeof(BatchSim<float, 2, 1>) * nsims);
  b->maps = static_cast<CUtensorMap*>(dev_alloc(b->hook, sizeof(CUtensorMap) * 2 * nsims));
  b->barrier = static_cast<unsigned int*>(dev_alloc(b->hook, 256));
  if (!b->state || !b->sims || !b->maps || !b->barrier) {
    batch_free(b);
    return bfail(nullptr, MS_ERR_OOM, "batch allocation failed");
  }
  b->status = reinterpret_cast<int*>(reinterpret_cast<char*>(b->barrier) + 128);
  cudaError_t e = cudaMemsetAsync(b->state, 0, tot, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->barrier, 0, 256, b->stream);
  // per-simulation constants
  std::vector<BatchSim<float, 2, 1>> hs(nsims);
  const StepKernel* k = nullptr;
  for (auto& sk : step_registry())
    if (sk.dim == 2 && sk.np == 2 && sk.nm == 1 && sk.dtype == 0 && sk.tx == kBTX && sk.ty == kBTY) k = &sk;
  for (int i = 0; i < nsims && e == cudaSuccess; ++i) {
    const HostModel& m = b->models[i];
    const size_t half = (b->sbytes[i] + 255) / 256 * 256;
    char* base = static_cast<char*>(b->state) + b->off[i];
    for (int par = 0; par < 2; ++par) {
      StepArgs<float, 2, 1>& g = hs[i].g[par];
      k->fill(&g, m, 1, b->status);
      g.out = reinterpret_cast<float*>(base + (1 - par) * half);
      g.tz0 = (float)temp_offset(m, m.t0);
    }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->sims, hs.data(), sizeof(hs[0]) * nsims, cudaMemcpyHostToDevice, b->stream);
  // work list, tensor maps and persistent grid (every CTA resident at once)
  if (e == cudaSuccess) e = batch_set_tiles(b, kBTY);
  if (e != cudaSuccess) {
    std::string m = std::string("batch set-up: ") + cudaGetErrorString(e);
    batch_free(b);
    return bfail(nullptr, e == cudaErrorMemoryAllocation ? MS_ERR_OOM : MS_ERR_CUDA, m);
  }
  *out = b;
  return MS_OK;
}

void ms_batch_destroy(ms_batch* b) { batch_free(b); }

const char* ms_batch_last_error(const ms_batch* b) { return b ? b->err.c_str() : ms_last_error(nullptr); }

ms_status ms_batch_set_fields(ms_batch* b, int sim, const void* phi, const void* mu, int on_device) {
  if (!b || sim < 0 || sim >= b->nsims || !phi || !mu) return bfail(b, MS_ERR_ARG, "bad argument");
  const HostModel& m = b->models[sim];
  const size_t half = (b->sbytes[sim] + 255) / 256 * 256;
  char* buf = static_cast<char*>(b->state) + b->off[sim] + b->parity * half;
  cudaError_t e = copy_fields(m, buf, 0, m.N, phi, nullptr, on_device, b->stream);
  if (e == cudaSuccess) e = copy_fields(m, buf, m.N, m.NM, mu, nullptr, on_device, b->stream);
  if (e == cudaSuccess) e = fill_ghosts(m, buf, m.N + m.NM, b->stream);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, MS_ERR_CUDA, std::string("batch set fields: ") + cudaGetErrorString(e));
  return MS_OK;
}

ms_status ms_batch_get_fields(ms_batch* b, int sim, void* phi, void* mu, int on_device) {
  if (!b || sim < 0 || sim >= b->nsims) return bfail(b, MS_ERR_ARG, "bad argument");
  const HostModel& m = b->models[sim];
  const size_t half = (b->sbytes[sim] + 255) / 256 * 256;
  char* buf = static_cast<char*>(b->state) + b->off[sim] + b->parity * half;
  cudaError_t e = cudaSuccess;
  if (phi) e = copy_fields(m, buf, 0, m.N, nullptr, phi, on_device, b->stream);
  if (e == cudaSuccess && mu) e = copy_fields(m, buf, m.N, m.NM, nullptr, mu, on_device, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, MS_ERR_CUDA, std::string("batch get fields: ") + cudaGetErrorString(e));
  return MS_OK;
}

ms_status ms_batch_step(ms_batch* b, int64_t n) {
  TraceRange trace("ms_batch_step");
  if (!b || n < 0) return bfail(b, MS_ERR_ARG, "bad argument");
  if (n == 0) return MS_OK;
  // the grid barrier counts (steps x CTAs) in 32 bits: at most 2^20 steps per launch
  if (n > ((int64_t)1 << 20)) return bfail(b, MS_ERR_BOUNDS, "at most 1048576 steps per ms_batch_step call");
  // the launch (barrier reset + cooperative kernel) is captured once per
  // (n, parity) and replayed
  cudaError_t e = cudaSuccess;
  if (!b->graph || b->graph_n != n * 2 + b->parity) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    cudaStream_t cap;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
      cudaStream_t keep = b->stream;
      b->stream = cap;
      cudaGraph_t graph;
      e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t le = launch_batch(b, n);
        e = cudaStreamEndCapture(cap, &graph);
        if (le != cudaSuccess) e = le;
      }
      b->stream = keep;
      if (e == cudaSuccess) {
        e = cudaGraphInstantiate(&b->graph, graph, 0);
        cudaGraphDestroy(graph);
      }
      cudaStreamDestroy(cap);
    }
    if (e != cudaSuccess) return bfail(b, MS_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    b->graph_n = n * 2 + b->parity;
  }
  e = cudaGraphLaunch(b->graph, b->stream);
  if (e != cudaSuccess) return bfail(b, MS_ERR_CUDA, std::string("batch launch: ") + cudaGetErrorString(e));
  b->parity = (int)((b->parity + n) & 1);
  b->steps_done += n;
  return MS_OK;
}

ms_status ms_batch_sync(ms_batch* b) {
  if (!b) return bfail(nullptr, MS_ERR_ARG, "batch is NULL");
  int st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, b->status, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(b, MS_ERR_CUDA, std::string("batch sync: ") + cudaGetErrorString(e));
  if (st & kStatusTimeout) return bfail(b, MS_ERR_TIMEOUT, "a bounded device wait timed out");
  return MS_OK;
}

ms_status ms_batch_set_tile(ms_batch* b, int ty) {
  if (!b) return bfail(nullptr, MS_ERR_ARG, "batch is NULL");
  bool ok = false;
  for (int k = 0; k < kNBTY; ++k) ok = ok || kBTYs[k] == ty;
  if (!ok) return bfail(b, MS_ERR_ARG, "tile height must be one of 4, 8, 16");
  if (ty == b->ty) return MS_OK;
  cudaError_t e = batch_set_tiles(b, ty);
  if (e != cudaSuccess) return bfail(b, MS_ERR_CUDA, std::string("batch tiles: ") + cudaGetErrorString(e));
  return MS_OK;
}

int ms_batch_tile(const ms_batch* b) { return b ? b->ty : 0; }

ms_status ms_batch_tune(ms_batch* b, int steps_per_trial, double* best_ms_per_step) {
  TraceRange trace("ms_batch_tune");
  if (!b || steps_per_trial < 1) return bfail(b, MS_ERR_ARG, "bad argument");
  size_t tot = 0;
  for (int i = 0; i < b->nsims; ++i) tot = std::max(tot, b->off[i] + 2 * ((b->sbytes[i] + 255) / 256 * 256));
  void* save = dev_alloc(b->hook, tot);
  if (!save) return bfail(b, MS_ERR_OOM, "batch tuner: state copy allocation failed");
  const int parity0 = b->parity;
  const int64_t done0 = b->steps_done;
  cudaError_t e = cudaMemcpyAsync(save, b->state, tot, cudaMemcpyDeviceToDevice, b->stream);
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  int best = b->ty;
  float best_ms = 0.0f;
  for (int k = 0; k < kNBTY && e == cudaSuccess; ++k) {
    e = batch_set_tiles(b, kBTYs[k]);
    if (e != cudaSuccess) break;
    // a warm-up launch captures the graph for this step count
    if (ms_batch_step(b, steps_per_trial) != MS_OK) {
      e = cudaErrorUnknown;
      break;
    }
    e = cudaEventRecord(t0, b->stream);
    if (e == cudaSuccess && ms_batch_step(b, steps_per_trial) != MS_OK) e = cudaErrorUnknown;
    if (e == cudaSuccess) e = cudaEventRecord(t1, b->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (e == cudaSuccess && (k == 0 || ms < best_ms)) {
      best_ms = ms;
      best = kBTYs[k];
    }
    // back to the saved state
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->state, save, tot, cudaMemcpyDeviceToDevice, b->stream);
    b->parity = parity0;
    b->steps_done = done0;
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  dev_free(b->hook, save);
  if (e == cudaSuccess) e = batch_set_tiles(b, best);
  if (e != cudaSuccess) return bfail(b, MS_ERR_CUDA, std::string("batch tuner: ") + cudaGetErrorString(e));
  if (best_ms_per_step) *best_ms_per_step = best_ms / steps_per_trial;
  return ms_batch_sync(b);
}

int64_t ms_batch_cells(const ms_batch* b) {
  if (!b) return 0;
  int64_t c = 0;
  for (auto& m : b->models) c += (int64_t)m.nx * m.ny * m.nz;
  return c;
}

}  // extern "C"
