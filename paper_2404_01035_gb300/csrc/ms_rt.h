// The context object behind the opaque ms_ctx handle, and runtime helpers
// shared by the C-ABI translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/microsim_gb.h"
#include "ms_internal.h"

namespace msgb {

struct AllocHook {
  void* (*alloc)(size_t, void*) = nullptr;
  void (*release)(void*, void*) = nullptr;
  void* user = nullptr;
};

void* dev_alloc(const AllocHook& h, size_t bytes);
void dev_free(const AllocHook& h, void* p);

// Adjoint bookkeeping: snapshots of the state every `every` steps.
struct AdjointStore {
  int every = 0;               // 0 = recording off
  int64_t first_step = 0;      // step of snapshot 0
  std::vector<void*> snaps;    // device copies of the full padded state
  void* seg = nullptr;         // recompute buffer: `every` states
  size_t seg_bytes = 0;
  void* adj[2] = {nullptr, nullptr};   // adjoint state ping-pong (padded)
  void* tbar = nullptr;        // per-cell adjoints of the step's tail inputs (reverse pass 1 -> 2)
  double* gpart = nullptr;     // per-block FP64 gradient partials
  int gblocks = 0;
  double* gsum = nullptr;      // accumulated parameter gradients (device)
};

// Elasticity buffers and FFT plans (allocated while elasticity is on).
struct ElasticState {
  void* E = nullptr;      // eigenstrain components, dense
  void* eps = nullptr;    // periodic strain components, dense
  void* spec = nullptr;   // their half spectra
  void* W = nullptr;      // -sigma : eps*^b per phase, dense [N][cells]
  int plan_r2c = 0, plan_c2r = 0, ncomp = 0;
  bool has_r2c = false, has_c2r = false;   // the plan handles hold created plans
  bool ready = false;   // every buffer and both plans exist (set only when complete)
};

}  // namespace msgb

struct ms_ctx {
  msgb::HostModel m;
  const msgb::StepKernel* kern = nullptr;
  const msgb::DiagKernel* diagk = nullptr;
  msgb::LaunchGeom lg;
  std::vector<unsigned char> args;   // launch-argument blob of `kern`
  CUtensorMap tm[2];
  CUtensorMap tmi[2];   // interface-box maps of buf[0] / buf[1] (split variants)
  void* buf[2] = {nullptr, nullptr};
  uint8_t* codes[2] = {nullptr, nullptr};   // segment codes of buf[0] / buf[1]
  unsigned int* iface = nullptr;            // work list of the split step (lazily allocated)
  unsigned int* at_list = nullptr;          // anti-trapping work list (allocated while it is on)
  size_t state_bytes = 0;
  int cur = 0;
  int64_t step = 0;
  double t = 0;
  int64_t diag_every = 0;
  cudaStream_t stream = nullptr;
  msgb::AllocHook hook;
  char* small = nullptr;        // status word + diag output + diag partials
  int* status = nullptr;
  double* diag_out = nullptr;
  double* diag_partials = nullptr;
  int diag_blocks = 0;
  void* diag_host = nullptr;
  std::string err;
  msgb::AdjointStore adj;
  msgb::ElasticState el;
  // host-side fault injection (MS_FAULT=step:K,code:X read at ms_create):
  // ms_step fails with fault_code when the context reaches step fault_step
  int64_t fault_step = -1;
  int fault_code = 0;
  int host_status = 0;   // sticky host-side status (an injected fault), 0 = none
};

namespace msgb {
ms_status fail(ms_ctx* c, ms_status s, const std::string& msg);
ms_status cuda_fail(ms_ctx* c, cudaError_t e, const char* what);
ms_status launch_one_step(ms_ctx* c);
ms_status apply_launch(ms_ctx* c, const StepKernel* k, int zchunk);
ms_status ensure_at_list(ms_ctx* c);   // the anti-trapping work list, when the current is on
ms_status refresh_codes(ms_ctx* c);   // segment codes of the current state
// Parse a fault-injection spec "step:K,code:X" (K >= 0, X a non-zero
// ms_status); false for a malformed one.  NULL or empty = no fault (step -1).
bool parse_fault_spec(const char* spec, int64_t* step, int* code);
bool elastic_available();                         // cuFFT could be opened
ms_status elastic_setup(ms_ctx* c);               // buffers and plans, when elasticity is on
bool elastic_grid_fits(const HostModel& m);       // the FFT plans take the grid's cell count
ms_status elastic_solve(ms_ctx* c, const void* state);   // w per phase from the state's phi
void elastic_free(ms_ctx* c);
// Tiled map of a padded state: box of (tx + 2H) x (ty + 2) x bz planes x nf fields.
bool encode_state_map(CUtensorMap* tm, void* base, const HostModel& m, int nf, int tx, int ty, int bz = 1);
// Maps a step variant reads from a state buffer: tm = its tile map (mu only
// for the streaming kernel of a split variant), tmi = the interface-box map
// (split variants only).
bool encode_step_maps(const StepKernel& k, CUtensorMap* tm, CUtensorMap* tmi, void* base, const HostModel& m);
void set_layout(HostModel& m);   // padded layout of one state buffer
std::vector<const StepKernel*> step_variants(int dim, int np, int nm, int dtype);
cudaError_t fill_ghosts(const HostModel& m, void* buf, int nf, cudaStream_t st);
cudaError_t copy_fields(const HostModel& m, void* padded, int f0, int nf, const void* dense, void* dense_out,
                        int on_device, cudaStream_t st);
}  // namespace msgb

// Hooks implemented by the adjoint unit.
ms_status ms_before_step(ms_ctx* c);   // records a snapshot when due
void ms_reset_extra(ms_ctx* c);        // forget snapshots (state replaced)
void ms_release_extra(ms_ctx* c);      // free adjoint buffers
