// Host-side internals shared by the runtime and the kernel instantiation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace msgb {

constexpr int kNMax = 8;
constexpr int kKMax = 3;

// Boundary code of an internal cut whose ghost plane is filled by a halo
// exchange (same value as MS_BC_HALO in the public header).
constexpr int kBcHalo = 16;

// Status bits OR-ed into the device status word.
constexpr int kStatusNonFinite = 1;
constexpr int kStatusTimeout = 2;
constexpr int kStatusLaunch = 4;   // launch geometry beyond a compiled limit (no work done)
// Planes marched by one CTA of the 3-D step at most (bounds the shared-memory
// copy of the segment codes a CTA reads).
constexpr int kMaxZChunk = 64;
// Segment-code byte: pure phase + 1 in the low bits (phases <= kNMax), and a
// bit saying that the state one step earlier held the same pure phase there.
constexpr int kCodePhase = 0x7F;
constexpr int kCodeReuse = 0x80;

// Model constants derived in FP64 from the paper's inputs (Sec. 3).
struct HostModel {
  int dim = 2, N = 2, NM = 1, dtype = 0;
  int nx = 1, ny = 1, nz = 1, bc[3] = {3, 3, 3};
  int zorg = 0;   // lab index of the first cell along the last axis (slabs, moving frame)
  // padded layout (elements)
  int pitch = 0, nyp = 0, nzp = 0, xoff = 0, zoff = 0;
  long long fstride = 0;
  double dx = 1, dt = 0, eps = 1, tau = 1;
  int potential = 1;
  double gamma[kNMax][kNMax] = {};
  double delta[kNMax][kNMax] = {};
  double rot[kNMax][kNMax][9] = {};
  bool rotated[kNMax][kNMax] = {};
  double g3[kNMax][kNMax][kNMax] = {};
  bool has_g3 = false;
  double chi[kNMax][kKMax * kKMax] = {};   // (Hessian)^-1
  double D[kNMax][kKMax * kKMax] = {};
  double DX[kNMax][kKMax * kKMax] = {};    // D chi
  double B0[kNMax][kKMax] = {}, B1[kNMax][kKMax] = {};
  double C0[kNMax] = {}, C1[kNMax] = {}, C2[kNMax] = {};
  double T0 = 0, G = 0, z0 = 0, V = 0, T_ref = 0, t0 = 0;
  double noise_amp = 0;                    // phi noise (0 = off)
  unsigned long long noise_seed = 0;
  int at = 0;                              // anti-trapping current in the mu update
  int gg = 0;                              // grain growth: no chemical driving force, mu held
  int el = 0;                              // elasticity (homogeneous stiffness)
  double elC[3][3][3][3] = {};             // stiffness tensor
  double eig[kNMax][3][3] = {};            // eigenstrain of each phase
};

// Launch geometry of one step.
struct LaunchGeom {
  int tiles = 0;       // gridDim.x
  int zchunks = 1;     // gridDim.y
  int zchunk = 1;
  unsigned int* iface = nullptr;   // work lists of split kernels (see StepArgs)
  unsigned int* iface2 = nullptr;
  unsigned int iface_cap = 0;
  int iface_blocks = 0;            // SMs: the interface grid is this x resident CTAs per SM
  int sms = 0;                     // multiprocessors of the device
  unsigned int* at_list = nullptr; // anti-trapping work list (see StepArgs)
  const void* elw = nullptr;       // elastic part of the phase potentials (see StepArgs)
  unsigned int at_cap = 0;
  int reuse_prev = 1;              // output buffer = state one step before the input (see StepArgs)
  long long step = 0;              // step index of the input state (phi-noise counter)
};

// One compiled forward-step instantiation.
struct StepKernel {
  int dim, np, nm, dtype, tx, ty;
  int split;   // 1: streaming kernel for bulk rows + interface kernel for the rest
  int smem_bytes;
  size_t args_bytes;
  // Fill the launch-argument blob from the model (all constants).
  void (*fill)(void* blob, const HostModel& m, int zchunk, int* status);
  // Launch one step: tm = tensor map of the input state (tile box), tmi =
  // its interface-box map (split variants; may be NULL otherwise), t = time
  // of the input state, out = destination buffer, codes_in / codes_out =
  // segment codes of the input / output state.
  cudaError_t (*launch)(const CUtensorMap* tm, const CUtensorMap* tmi, void* blob, const HostModel& m, double t, void* out,
                        const uint8_t* codes_in, uint8_t* codes_out, const LaunchGeom& lg,
                        cudaStream_t st);
  // Recompute the segment codes of a state loaded from outside.
  cudaError_t (*codes)(const void* state, const HostModel& m, uint8_t* codes, cudaStream_t st);
  // Anti-trapping correction of the mu just written by launch (same
  // arguments; in = the input state).
  cudaError_t (*at)(const void* in, void* blob, const HostModel& m, double t, void* out, const uint8_t* codes_in,
                    uint8_t* codes_out, const LaunchGeom& lg, cudaStream_t st);
};

// Number of 32-cell segments per row.
inline int segments(const HostModel& m) { return (m.nx + 31) / 32; }
// Bits that hold the values 0 .. n - 1.
inline int bits_for(int n) {
  int b = 0;
  while ((1ll << b) < n) ++b;
  return b;
}
// An interface-list entry (z, y, segment) packs into 31 bits (every shift
// of its fields stays below 32).
inline bool list_entry_fits(const HostModel& m) {
  return bits_for(segments(m)) + bits_for(m.ny) + bits_for(m.nz) <= 31;
}
// Bytes of one segment-code array (3-D arrays carry a ghost plane per side).
inline size_t code_bytes(const HostModel& m) { return (size_t)segments(m) * m.ny * m.nzp; }

// One compiled FP64 diagnostics instantiation.
struct DiagKernel {
  int dim, np, nm, dtype;
  cudaError_t (*launch)(const void* state, const HostModel& m, double t, double* partials,
                        int nblocks, double* out, int* status, cudaStream_t st);
};

std::vector<StepKernel>& step_registry();
std::vector<DiagKernel>& diag_registry();
void ensure_registered();

}  // namespace msgb
