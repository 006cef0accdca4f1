// C-ABI runtime of the grand-potential step library (see include/microsim_gb.h).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/microsim_gb.h"
#include "ms_internal.h"
#include "ms_rt.h"
#include "ms_trace.h"

namespace msgb {

thread_local std::string g_thread_error;

std::vector<StepKernel>& step_registry() {
  static std::vector<StepKernel> r;
  return r;
}
std::vector<DiagKernel>& diag_registry() {
  static std::vector<DiagKernel> r;
  return r;
}

void register_2d(std::vector<StepKernel>&, std::vector<DiagKernel>&);
void register_3d_n2(std::vector<StepKernel>&, std::vector<DiagKernel>&);
void register_3d_n3(std::vector<StepKernel>&, std::vector<DiagKernel>&);
void register_3d_n8(std::vector<StepKernel>&, std::vector<DiagKernel>&);

void ensure_registered() {
  static std::once_flag once;
  std::call_once(once, [] {
    register_2d(step_registry(), diag_registry());
    register_3d_n2(step_registry(), diag_registry());
    register_3d_n3(step_registry(), diag_registry());
    register_3d_n8(step_registry(), diag_registry());
  });
}

// ------------------------------------------------------------- error helpers
ms_status fail(ms_ctx* c, ms_status s, const std::string& msg) {
  if (c) c->err = msg;
  g_thread_error = msg;
  return s;
}

ms_status cuda_fail(ms_ctx* c, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(c, e == cudaErrorMemoryAllocation ? MS_ERR_OOM : MS_ERR_CUDA, m);
}

#define MS_CUDA(ctx, call)                                  \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

// ----------------------------------------------------------------- allocation
void* dev_alloc(const AllocHook& h, size_t bytes) {
  if (h.alloc) return h.alloc(bytes, h.user);
  void* p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
  return p;
}
void dev_free(const AllocHook& h, void* p) {
  if (!p) return;
  if (h.release)
    h.release(p, h.user);
  else
    cudaFree(p);
}

// --------------------------------------------------------------- the model
static double a_entry(const ms_params* p, int NM, int a, int i, int j) {
  if (i > j) std::swap(i, j);
  return p->A[(a * NM + i) * NM + j];
}

static bool invert(int n, const double* M, double* out) {
  double a[kKMax][2 * kKMax];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) a[i][j] = j < n ? M[i * n + j] : (i == j - n ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[r][c]) > std::fabs(a[piv][c])) piv = r;
    if (std::fabs(a[piv][c]) < 1e-300) return false;
    if (piv != c)
      for (int j = 0; j < 2 * n; ++j) std::swap(a[c][j], a[piv][j]);
    double d = a[c][c];
    for (int j = 0; j < 2 * n; ++j) a[c][j] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      double f = a[r][c];
      for (int j = 0; j < 2 * n; ++j) a[r][j] -= f * a[c][j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) out[i * n + j] = a[i][j + n];
  return true;
}

// Derive the FP64 model constants from the paper's inputs.
// build_model, also reporting the explicit stability bound on dt (when
// bound_out is not NULL and the checks before it passed).
ms_status build_model_bound(ms_ctx* c, const ms_grid* g, int N, int K, const ms_params* p, HostModel& m,
                            double* bound_out);

ms_status build_model(ms_ctx* c, const ms_grid* g, int N, int K, const ms_params* p, HostModel& m) {
  return build_model_bound(c, g, N, K, p, m, nullptr);
}

ms_status build_model_bound(ms_ctx* c, const ms_grid* g, int N, int K, const ms_params* p, HostModel& m,
                            double* bound_out) {
  if (!g || !p) return fail(c, MS_ERR_ARG, "grid and params are required");
  if (g->dim != 2 && g->dim != 3) return fail(c, MS_ERR_ARG, "dim must be 2 or 3");
  if (N < 2 || N > kNMax) return fail(c, MS_ERR_ARG, "n_phases must be in [2, 8]");
  if (K < 2 || K > kKMax + 1) return fail(c, MS_ERR_ARG, "n_components must be in [2, 4]");
  if (g->nx < 1 || g->ny < 1 || (g->dim == 3 && g->nz < 1))
    return fail(c, MS_ERR_ARG, "grid extents must be >= 1");
  if (!(g->dx > 0)) return fail(c, MS_ERR_ARG, "dx must be > 0");
  for (int d = 0; d < 3; ++d) {
    if (d == 2 && g->dim == 3 && g->bc[d] == MS_BC_HALO) continue;   // internal cut in z
    if (g->bc[d] != MS_BC_PERIODIC && g->bc[d] != MS_BC_NOFLUX)
      return fail(c, MS_ERR_ARG, "boundary codes must be 1 (no-flux) or 3 (periodic); 16 (halo) only for z in 3-D");
  }
  if (p->dtype != MS_F32 && p->dtype != MS_F64) return fail(c, MS_ERR_ARG, "dtype must be MS_F32 or MS_F64");
  if (p->potential != MS_POT_OBSTACLE && p->potential != MS_POT_WELL)
    return fail(c, MS_ERR_ARG, "potential must be 1 (obstacle) or 2 (well)");
  if (!(p->eps > 0) || !(p->tau > 0) || !(p->dt > 0)) return fail(c, MS_ERR_ARG, "eps, tau, dt must be > 0");
  if (!p->gamma || !p->delta || !p->D || !p->A || !p->ceq || !p->slopes)
    return fail(c, MS_ERR_ARG, "gamma, delta, D, A, ceq and slopes are required");
  const int NM = K - 1;
  if (static_cast<long long>(g->nx) * g->ny * (g->dim == 3 ? g->nz : 1) > (1ll << 40))
    return fail(c, MS_ERR_BOUNDS, "grid too large");
  m.dim = g->dim;
  m.N = N;
  m.NM = NM;
  m.dtype = p->dtype;
  m.nx = g->nx;
  m.ny = g->ny;
  m.nz = g->dim == 3 ? g->nz : 1;
  for (int d = 0; d < 3; ++d) m.bc[d] = g->bc[d];
  m.zorg = g->z_origin;
  if (m.zorg < 0) return fail(c, MS_ERR_ARG, "z_origin must be >= 0");
  m.dx = g->dx;
  m.dt = p->dt;
  m.eps = p->eps;
  m.tau = p->tau;
  m.potential = p->potential;
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) {
      m.gamma[a][b] = p->gamma[a * N + b];
      m.delta[a][b] = p->delta[a * N + b];
      if (a != b && (m.gamma[a][b] < 0 || m.delta[a][b] < 0))
        return fail(c, MS_ERR_ARG, "gamma and delta must be >= 0");
      bool rotated = false;
      for (int k = 0; k < 9; ++k) {
        double v = p->rot ? p->rot[(a * N + b) * 9 + k] : (k % 4 == 0 ? 1.0 : 0.0);
        m.rot[a][b][k] = v;
        if (v != (k % 4 == 0 ? 1.0 : 0.0)) rotated = true;
      }
      m.rotated[a][b] = rotated;
    }
  m.has_g3 = false;
  if (p->gamma3)
    for (int a = 0; a < N; ++a)
      for (int b = 0; b < N; ++b)
        for (int e = 0; e < N; ++e) {
          m.g3[a][b][e] = p->gamma3[(a * N + b) * N + e];
          if (m.g3[a][b][e] != 0.0) m.has_g3 = true;
        }
  const int L = N - 1;
  double H[kNMax][kKMax * kKMax];
  for (int a = 0; a < N; ++a) {
    for (int i = 0; i < NM; ++i)
      for (int j = 0; j < NM; ++j) H[a][i * NM + j] = (i == j ? 2.0 : 1.0) * a_entry(p, NM, a, i, j);
    if (!invert(NM, H[a], m.chi[a])) return fail(c, MS_ERR_ARG, "singular free-energy Hessian");
    for (int k = 0; k < NM * NM; ++k) m.D[a][k] = p->D[a * NM * NM + k];
    for (int i = 0; i < NM; ++i)
      for (int j = 0; j < NM; ++j) {
        double s = 0;
        for (int k = 0; k < NM; ++k) s += m.D[a][i * NM + k] * m.chi[a][k * NM + j];
        m.DX[a][i * NM + j] = s;
      }
  }
  // B^a(T) = H^l c_eq^l(T) - H^a c_eq^a(T); C^a(T) = 1/2 c^a H^a c^a - 1/2 c^l H^l c^l + f0^a
  for (int a = 0; a < N; ++a) {
    const double* ca = p->ceq + a * NM;
    const double* cl = p->ceq + L * NM;
    const double* sa = p->slopes + a * NM;
    const double* sl = p->slopes + L * NM;
    for (int j = 0; j < NM; ++j) {
      double b0 = 0, b1 = 0;
      for (int i = 0; i < NM; ++i) {
        b0 += H[L][j * NM + i] * cl[i] - H[a][j * NM + i] * ca[i];
        b1 += H[L][j * NM + i] * sl[i] - H[a][j * NM + i] * sa[i];
      }
      m.B0[a][j] = a == L ? 0.0 : b0;
      m.B1[a][j] = a == L ? 0.0 : b1;
    }
    double c0 = 0, c1 = 0, c2 = 0;
    for (int i = 0; i < NM; ++i)
      for (int j = 0; j < NM; ++j) {
        c0 += 0.5 * (ca[i] * H[a][i * NM + j] * ca[j] - cl[i] * H[L][i * NM + j] * cl[j]);
        c1 += (sa[i] * H[a][i * NM + j] * ca[j] - sl[i] * H[L][i * NM + j] * cl[j]);
        c2 += 0.5 * (sa[i] * H[a][i * NM + j] * sa[j] - sl[i] * H[L][i * NM + j] * sl[j]);
      }
    m.C0[a] = (a == L ? 0.0 : c0) + (p->f0 ? p->f0[a] : 0.0);
    m.C1[a] = a == L ? 0.0 : c1;
    m.C2[a] = a == L ? 0.0 : c2;
  }
  m.T0 = p->T0;
  m.G = p->G;
  m.z0 = p->z0;
  m.V = p->V;
  m.T_ref = p->T_ref;
  m.t0 = p->t0;
  if (!(p->noise_amp >= 0.0) || !std::isfinite(p->noise_amp)) return fail(c, MS_ERR_ARG, "noise_amp must be finite and >= 0");
  m.noise_amp = p->noise_amp;
  m.noise_seed = p->noise_seed;
  m.at = p->anti_trapping ? 1 : 0;
  m.gg = p->grain_growth ? 1 : 0;
  if (m.at && m.gg) return fail(c, MS_ERR_ARG, "grain growth holds mu: the anti-trapping current does not apply");
  m.el = p->elastic_C ? 1 : 0;
  if (m.el) {
    if (!p->eigenstrain) return fail(c, MS_ERR_ARG, "elasticity needs eigenstrain with elastic_C");
    if (m.gg) return fail(c, MS_ERR_UNSUPPORTED, "elasticity is not offered with grain growth");
    if (m.dim == 3 && m.bc[2] == kBcHalo)
      return fail(c, MS_ERR_UNSUPPORTED, "elasticity needs the whole periodic domain (no halo faces)");
    for (int d = 0; d < m.dim; ++d)
      if (m.bc[d] != 3) return fail(c, MS_ERR_UNSUPPORTED, "elasticity (FFT equilibrium) needs periodic boundaries");
    if (!elastic_grid_fits(m))
      return fail(c, MS_ERR_UNSUPPORTED, "grid too large for the FFT plans of the elasticity (more than 2^31-1 cells)");
    // Voigt index of a symmetric pair (xx, yy, zz, yz, xz, xy)
    const int v[3][3] = {{0, 5, 4}, {5, 1, 3}, {4, 3, 2}};
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l) m.elC[i][j][k][l] = p->elastic_C[v[i][j] * 6 + v[k][l]];
    for (int a = 0; a < N; ++a)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) m.eig[a][i][j] = p->eigenstrain[(a * 3 + i) * 3 + j];
  }
  if (m.at && m.dim == 3 && m.bc[2] == kBcHalo)
    return fail(c, MS_ERR_UNSUPPORTED, "the anti-trapping current is not available on slabs with halo faces");
  // explicit stability bound (FP64): (dx^2 / 2d) min(tau / (gamma (1 + 15 delta)), 1 / D_eff)
  double gmax = 0, dmax = 0, Dmax = 0;
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b)
      if (a != b) {
        gmax = std::max(gmax, m.gamma[a][b]);
        dmax = std::max(dmax, m.delta[a][b]);
      }
  for (int a = 0; a < N; ++a) {
    // ||chi^-1 D chi||_inf of phase a: the diffusivity of mu in that phase
    double Hc[kKMax * kKMax];
    for (int i = 0; i < NM; ++i)
      for (int j = 0; j < NM; ++j) {
        double s = 0;
        for (int k = 0; k < NM; ++k) s += H[a][i * NM + k] * m.DX[a][k * NM + j];
        Hc[i * NM + j] = s;
      }
    for (int i = 0; i < NM; ++i) {
      double r = 0;
      for (int j = 0; j < NM; ++j) r += std::fabs(Hc[i * NM + j]);
      Dmax = std::max(Dmax, r);
    }
  }
  const double lim_phi = gmax > 0 ? m.tau / (gmax * (1.0 + 15.0 * dmax)) : 1e300;
  const double lim_mu = Dmax > 0 ? 1.0 / Dmax : 1e300;
  const double bound = m.dx * m.dx / (2.0 * m.dim) * std::min(lim_phi, lim_mu);
  if (bound_out) *bound_out = bound;
  if (m.dt > bound * (1.0 + 1e-12)) {
    char buf[160];
    std::snprintf(buf, sizeof buf, "dt = %.6g exceeds the explicit stability bound %.6g", m.dt, bound);
    return fail(c, MS_ERR_DT_UNSTABLE, buf);
  }
  return MS_OK;
}

void set_layout(HostModel& m) {
  const int s = m.dtype == MS_F64 ? 8 : 4;
  const int H = 16 / s;
  const int align = 128 / s;
  m.xoff = H;
  m.pitch = (m.xoff + m.nx + 1 + align - 1) / align * align;
  m.nyp = m.ny + 2;
  m.nzp = m.dim == 3 ? m.nz + 2 : 1;
  m.zoff = m.dim == 3 ? 1 : 0;
  m.fstride = (long long)m.nzp * m.nyp * m.pitch;
}

// ------------------------------------------------------------- TMA descriptors
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

bool encode_state_map(CUtensorMap* tm, void* base, const HostModel& m, int nf, int tx, int ty, int bz) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const int s = m.dtype == MS_F64 ? 8 : 4;
  const int H = 16 / s;
  cuuint64_t dims[4] = {(cuuint64_t)m.pitch, (cuuint64_t)m.nyp, (cuuint64_t)m.nzp, (cuuint64_t)nf};
  cuuint64_t strides[3] = {(cuuint64_t)m.pitch * s, (cuuint64_t)m.pitch * m.nyp * s,
                           (cuuint64_t)m.fstride * s};
  cuuint32_t box[4] = {(cuuint32_t)(tx + 2 * H), (cuuint32_t)(ty + 2), (cuuint32_t)bz, (cuuint32_t)nf};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = fn(tm, m.dtype == MS_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                  4, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool encode_step_maps(const StepKernel& k, CUtensorMap* tm, CUtensorMap* tmi, void* base, const HostModel& m) {
  const int nf = m.N + m.NM;
  if (!k.split) return encode_state_map(tm, base, m, nf, k.tx, k.ty);
  const size_t s = m.dtype == MS_F64 ? 8 : 4;
  char* mu = static_cast<char*>(base) + (size_t)m.N * m.fstride * s;
  return encode_state_map(tm, mu, m, m.NM, k.tx, k.ty) && encode_state_map(tmi, base, m, nf, 32, 1, 3);
}

// ----------------------------------------------------------------- ghost fill
template <class Real>
__global__ void k_fill_ghosts(Real* buf, int nf, int nx, int ny, int nz, int pitch, int nyp,
                              long long fstride, int xoff, int zoff, int axis, int bc) {
  // one thread per (field, line) perpendicular to `axis`, including the ghost
  // layers of the axes filled before it (x, then y, then z)
  const long long plane = (long long)nyp * pitch;
  long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (axis == 0) {
    long long lines = (long long)nf * nz * ny;
    if (tid >= lines) return;
    int f = (int)(tid / ((long long)nz * ny));
    int r = (int)(tid % ((long long)nz * ny));
    int z = r / ny, y = r % ny;
    Real* row = buf + f * fstride + (z + zoff) * plane + (long long)(y + 1) * pitch + xoff;
    Real lo = bc == 3 ? row[nx - 1] : row[0];
    Real hi = bc == 3 ? row[0] : row[nx - 1];
    row[-1] = lo;
    row[nx] = hi;
  } else if (axis == 1) {
    long long lines = (long long)nf * nz * (nx + 2);
    if (tid >= lines) return;
    int f = (int)(tid / ((long long)nz * (nx + 2)));
    int r = (int)(tid % ((long long)nz * (nx + 2)));
    int z = r / (nx + 2), x = r % (nx + 2) - 1;
    Real* col = buf + f * fstride + (z + zoff) * plane + xoff + x;
    Real lo = bc == 3 ? col[(long long)ny * pitch] : col[(long long)1 * pitch];
    Real hi = bc == 3 ? col[(long long)1 * pitch] : col[(long long)ny * pitch];
    col[0] = lo;
    col[(long long)(ny + 1) * pitch] = hi;
  } else {
    long long lines = (long long)nf * (ny + 2) * (nx + 2);
    if (tid >= lines) return;
    int f = (int)(tid / ((long long)(ny + 2) * (nx + 2)));
    int r = (int)(tid % ((long long)(ny + 2) * (nx + 2)));
    int y = r / (nx + 2) - 1, x = r % (nx + 2) - 1;
    Real* col = buf + f * fstride + (long long)(y + 1) * pitch + xoff + x;
    Real lo = bc == 3 ? col[(long long)nz * plane] : col[(long long)1 * plane];
    Real hi = bc == 3 ? col[(long long)1 * plane] : col[(long long)nz * plane];
    col[0] = lo;
    col[(long long)(nz + 1) * plane] = hi;
  }
}

cudaError_t fill_ghosts(const HostModel& m, void* buf, int nf, cudaStream_t st) {
  for (int axis = 0; axis < m.dim; ++axis) {
    if (m.bc[axis] == kBcHalo) continue;   // filled by the halo exchange
    long long lines = axis == 0 ? (long long)nf * m.nz * m.ny
                      : axis == 1 ? (long long)nf * m.nz * (m.nx + 2)
                                  : (long long)nf * (m.ny + 2) * (m.nx + 2);
    int blocks = (int)((lines + 255) / 256);
    if (m.dtype == MS_F64)
      k_fill_ghosts<double><<<blocks, 256, 0, st>>>((double*)buf, nf, m.nx, m.ny, m.nz, m.pitch, m.nyp,
                                                     m.fstride, m.xoff, m.zoff, axis, m.bc[axis]);
    else
      k_fill_ghosts<float><<<blocks, 256, 0, st>>>((float*)buf, nf, m.nx, m.ny, m.nz, m.pitch, m.nyp,
                                                    m.fstride, m.xoff, m.zoff, axis, m.bc[axis]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Copy nf dense fields [f][z][y][x] into / out of the interior of a padded buffer.
cudaError_t copy_fields(const HostModel& m, void* padded, int f0, int nf, const void* dense, void* dense_out,
                        int on_device, cudaStream_t st) {
  const size_t s = m.dtype == MS_F64 ? 8 : 4;
  for (int f = 0; f < nf; ++f) {
    cudaMemcpy3DParms p = {};
    char* pbase = (char*)padded + ((f0 + f) * m.fstride) * s;
    cudaPitchedPtr pp = make_cudaPitchedPtr(pbase, m.pitch * s, m.pitch, m.nyp);
    cudaPos ppos = make_cudaPos(m.xoff * s, 1, m.zoff);
    const size_t fbytes = (size_t)m.nx * m.ny * m.nz * s;
    if (dense) {
      cudaPitchedPtr dp = make_cudaPitchedPtr((void*)((const char*)dense + f * fbytes), m.nx * s, m.nx, m.ny);
      p.srcPtr = dp;
      p.srcPos = make_cudaPos(0, 0, 0);
      p.dstPtr = pp;
      p.dstPos = ppos;
      p.kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    } else {
      cudaPitchedPtr dp = make_cudaPitchedPtr((char*)dense_out + f * fbytes, m.nx * s, m.nx, m.ny);
      p.srcPtr = pp;
      p.srcPos = ppos;
      p.dstPtr = dp;
      p.dstPos = make_cudaPos(0, 0, 0);
      p.kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    }
    p.extent = make_cudaExtent(m.nx * s, m.ny, m.nz);
    cudaError_t e = cudaMemcpy3DAsync(&p, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

const StepKernel* find_step(int dim, int np, int nm, int dtype, int tx, int ty) {
  for (auto& k : step_registry())
    if (k.dim == dim && k.np == np && k.nm == nm && k.dtype == dtype && (tx == 0 || k.tx == tx) &&
        (ty == 0 || k.ty == ty))
      return &k;
  return nullptr;
}

std::vector<const StepKernel*> step_variants(int dim, int np, int nm, int dtype) {
  std::vector<const StepKernel*> v;
  for (auto& k : step_registry())
    if (k.dim == dim && k.np == np && k.nm == nm && k.dtype == dtype) v.push_back(&k);
  return v;
}

const DiagKernel* find_diag(int dim, int np, int nm, int dtype) {
  for (auto& k : diag_registry())
    if (k.dim == dim && k.np == np && k.nm == nm && k.dtype == dtype) return &k;
  return nullptr;
}

int default_zchunk(const HostModel& m, const StepKernel& k) {
  if (m.dim != 3) return 1;
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long tiles = (long long)((m.nx + k.tx - 1) / k.tx) * ((m.ny + k.ty - 1) / k.ty);
  // aim for >= 8 CTAs per SM worth of work units, chunks of 8..64 planes
  int zc = 64;
  while (zc > 8 && tiles * ((m.nz + zc - 1) / zc) < 8ll * sms) zc /= 2;
  return std::min(zc, m.nz);
}

ms_status ensure_at_list(ms_ctx* c) {
  if (!c->m.at || c->at_list) return MS_OK;
  // count, ticket and one entry per row segment
  const size_t cap = (size_t)segments(c->m) * c->m.ny * (c->m.dim == 3 ? c->m.nz : 1);
  if (cap > 0xFFFFFFF0ull) return fail(c, MS_ERR_UNSUPPORTED, "grid too large for the anti-trapping list");
  c->at_list = static_cast<unsigned int*>(dev_alloc(c->hook, (cap + 2) * sizeof(unsigned int)));
  if (!c->at_list) return fail(c, MS_ERR_OOM, "anti-trapping work-list allocation failed");
  c->lg.at_list = c->at_list;
  c->lg.at_cap = (unsigned int)cap;
  cudaError_t e = cudaMemsetAsync(c->at_list, 0, 2 * sizeof(unsigned int), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "work-list reset");
  return MS_OK;
}

ms_status apply_launch(ms_ctx* c, const StepKernel* k, int zchunk) {
  if (c->lg.sms < 1) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    c->lg.sms = sms;
  }
  ms_status as = ensure_at_list(c);
  if (as != MS_OK) return as;
  if (k->split && !c->iface) {
    // work list of the split step: count, ticket and one entry per warp row
    // (two lists: the second takes the rows left for a second launch)
    const size_t cap = (size_t)segments(c->m) * c->m.ny * c->m.nz;
    if (cap > 0xFFFFFFF0ull || !list_entry_fits(c->m))
      return fail(c, MS_ERR_UNSUPPORTED, "grid too large for the split step");
    c->iface = static_cast<unsigned int*>(dev_alloc(c->hook, 2 * (cap + 2) * sizeof(unsigned int)));
    if (!c->iface) return fail(c, MS_ERR_OOM, "interface work-list allocation failed");
    c->lg.iface = c->iface;
    c->lg.iface2 = c->iface + cap + 2;
    c->lg.iface_cap = (unsigned int)cap;
    cudaError_t e = cudaMemsetAsync(c->lg.iface, 0, 2 * sizeof(unsigned int), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->lg.iface2, 0, 2 * sizeof(unsigned int), c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "work-list reset");
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    c->lg.iface_blocks = sms;
  }
  c->kern = k;
  c->lg.zchunk = c->m.dim == 3 ? std::min(zchunk > 0 ? std::min(zchunk, c->m.nz) : default_zchunk(c->m, *k), kMaxZChunk) : 1;
  c->lg.tiles = ((c->m.nx + k->tx - 1) / k->tx) * ((c->m.ny + k->ty - 1) / k->ty);
  c->lg.zchunks = c->m.dim == 3 ? (c->m.nz + c->lg.zchunk - 1) / c->lg.zchunk : 1;
  c->args.assign(k->args_bytes, 0);
  k->fill(c->args.data(), c->m, c->lg.zchunk, c->status);
  for (int b = 0; b < 2; ++b)
    if (!encode_step_maps(*k, &c->tm[b], &c->tmi[b], c->buf[b], c->m))
      return fail(c, MS_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return MS_OK;
}

ms_status launch_one_step(ms_ctx* c) {
  const int src = c->cur, dst = 1 - c->cur;
  c->lg.step = c->step;
  if (c->m.el) {   // elastic potentials of phi^n before the step
    if (!c->el.ready) return fail(c, MS_ERR_STATE, "elasticity is on but its buffers and FFT plans do not exist");
    ms_status es = elastic_solve(c, c->buf[src]);
    if (es != MS_OK) return es;
  }
  cudaError_t e = c->kern->launch(&c->tm[src], &c->tmi[src], c->args.data(), c->m, c->t, c->buf[dst], c->codes[src],
                                  c->codes[dst], c->lg, c->stream);
  if (e == cudaSuccess && c->m.at)
    e = c->kern->at(c->buf[src], c->args.data(), c->m, c->t, c->buf[dst], c->codes[src], c->codes[dst], c->lg,
                    c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "step launch");
  c->cur = dst;
  c->step += 1;
  c->t = c->m.t0 + (double)c->step * c->m.dt;
  return MS_OK;
}

ms_status refresh_codes(ms_ctx* c) {
  cudaError_t e = c->kern->codes(c->buf[c->cur], c->m, c->codes[c->cur], c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "segment codes");
  // the other buffer no longer holds the state before this one: its codes
  // must not let the next step keep phi there
  e = cudaMemsetAsync(c->codes[1 - c->cur], 0, code_bytes(c->m), c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "segment codes");
  return MS_OK;
}

bool parse_fault_spec(const char* spec, int64_t* step, int* code) {
  *step = -1;
  *code = 0;
  if (!spec || !*spec) return true;
  long long k = -1;
  int x = 0, used = 0;
  if (std::sscanf(spec, "step:%lld,code:%d%n", &k, &x, &used) != 2 || spec[used] != '\0') return false;
  if (k < 0 || x < MS_ERR_ARG || x > MS_ERR_UNSUPPORTED) return false;
  *step = (int64_t)k;
  *code = x;
  return true;
}

ms_status launch_diag_now(ms_ctx* c) {
  cudaError_t e = c->diagk->launch(c->buf[c->cur], c->m, c->t, c->diag_partials, c->diag_blocks,
                                   c->diag_out, c->status, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "diag launch");
  return MS_OK;
}

}  // namespace msgb

using namespace msgb;

extern "C" {

const char* ms_last_error(const ms_ctx* ctx) {
  if (ctx) return ctx->err.c_str();
  return g_thread_error.c_str();
}

ms_status ms_check_params(const ms_grid* grid, int n_phases, int n_components, const ms_params* params,
                          double* dt_bound) {
  ensure_registered();
  HostModel m;
  double bound = 0.0;
  ms_status s = build_model_bound(nullptr, grid, n_phases, n_components, params, m, &bound);
  if (dt_bound) *dt_bound = bound;
  if (s != MS_OK) return s;
  if (!find_step(m.dim, m.N, m.NM, m.dtype, 0, 0) || !find_diag(m.dim, m.N, m.NM, m.dtype)) {
    char buf[200];
    std::snprintf(buf, sizeof buf, "no compiled step kernel for dim=%d N=%d K=%d dtype=%s", m.dim, m.N,
                  n_components, m.dtype ? "f64" : "f32");
    return fail(nullptr, MS_ERR_UNSUPPORTED, buf);
  }
  return MS_OK;
}

ms_status ms_create(const ms_grid* grid, int n_phases, int n_components, const ms_params* params,
                    void* stream, const ms_allocator* alloc, ms_ctx** out) {
  if (!out) return fail(nullptr, MS_ERR_ARG, "out is NULL");
  *out = nullptr;
  ensure_registered();
  ms_ctx* c = new ms_ctx();
  ms_status s = build_model(nullptr, grid, n_phases, n_components, params, c->m);
  if (s != MS_OK) {
    delete c;
    return s;
  }
  set_layout(c->m);
  if (!parse_fault_spec(std::getenv("MS_FAULT"), &c->fault_step, &c->fault_code)) {
    delete c;
    return fail(nullptr, MS_ERR_ARG, "MS_FAULT must read step:K,code:X (K >= 0, X a non-zero ms_status)");
  }
  const StepKernel* k = find_step(c->m.dim, c->m.N, c->m.NM, c->m.dtype, 32, 8);
  if (!k) k = find_step(c->m.dim, c->m.N, c->m.NM, c->m.dtype, 0, 0);
  c->diagk = find_diag(c->m.dim, c->m.N, c->m.NM, c->m.dtype);
  if (!k || !c->diagk) {
    char buf[200];
    std::snprintf(buf, sizeof buf, "no compiled step kernel for dim=%d N=%d K=%d dtype=%s", c->m.dim, c->m.N,
                  n_components, c->m.dtype ? "f64" : "f32");
    delete c;
    return fail(nullptr, MS_ERR_UNSUPPORTED, buf);
  }
  if (alloc) c->hook = AllocHook{alloc->alloc, alloc->release, alloc->user};
  c->stream = static_cast<cudaStream_t>(stream);
  const size_t s_el = c->m.dtype == MS_F64 ? 8 : 4;
  const int nf = c->m.N + c->m.NM;
  c->state_bytes = (size_t)c->m.fstride * nf * s_el;
  const size_t cbytes = code_bytes(c->m);
  for (int b = 0; b < 2; ++b) {
    c->buf[b] = dev_alloc(c->hook, c->state_bytes);
    c->codes[b] = static_cast<uint8_t*>(dev_alloc(c->hook, cbytes));
    if (!c->buf[b] || !c->codes[b]) {
      ms_destroy(c);
      return fail(nullptr, MS_ERR_OOM, "state allocation failed");
    }
  }
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  c->diag_blocks = 4 * sms;
  c->small = static_cast<char*>(dev_alloc(c->hook, 4096 + sizeof(double) * c->diag_blocks * 16));
  if (!c->small) {
    ms_destroy(c);
    return fail(nullptr, MS_ERR_OOM, "scratch allocation failed");
  }
  c->status = reinterpret_cast<int*>(c->small);
  c->diag_out = reinterpret_cast<double*>(c->small + 256);
  c->diag_partials = reinterpret_cast<double*>(c->small + 4096);
  if (cudaMallocHost(&c->diag_host, 4096) != cudaSuccess) {
    ms_destroy(c);
    return fail(nullptr, MS_ERR_OOM, "pinned allocation failed");
  }
  cudaError_t e = cudaMemsetAsync(c->small, 0, 4096, c->stream);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    e = cudaMemsetAsync(c->buf[b], 0, c->state_bytes, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->codes[b], 0, cbytes, c->stream);
  }
  if (e != cudaSuccess) {
    ms_status r = cuda_fail(nullptr, e, "initial memset");
    ms_destroy(c);
    return r;
  }
  s = apply_launch(c, k, 0);
  if (s == MS_OK) s = elastic_setup(c);
  if (s != MS_OK) {
    std::string m = c->err;
    ms_destroy(c);
    return fail(nullptr, s, m);
  }
  c->t = c->m.t0;
  *out = c;
  return MS_OK;
}

void ms_destroy(ms_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  ms_release_extra(c);
  elastic_free(c);
  for (int b = 0; b < 2; ++b) {
    dev_free(c->hook, c->buf[b]);
    dev_free(c->hook, c->codes[b]);
  }
  dev_free(c->hook, c->small);
  dev_free(c->hook, c->iface);
  dev_free(c->hook, c->at_list);
  if (c->diag_host) cudaFreeHost(c->diag_host);
  delete c;
}

ms_status ms_update_params(ms_ctx* c, const ms_params* p) {
  if (!c) return fail(nullptr, MS_ERR_ARG, "ctx is NULL");
  ms_grid g;
  g.dim = c->m.dim;
  g.nx = c->m.nx;
  g.ny = c->m.ny;
  g.nz = c->m.nz;
  g.z_origin = c->m.zorg;
  g.dx = c->m.dx;
  for (int d = 0; d < 3; ++d) g.bc[d] = c->m.bc[d];
  if (!p || p->dtype != c->m.dtype) return fail(c, MS_ERR_ARG, "dtype cannot change");
  HostModel m2;
  ms_status s = build_model(c, &g, c->m.N, c->m.NM + 1, p, m2);
  if (s != MS_OK) return s;
  if (c->adj.every > 0 && (m2.noise_amp != 0.0 || m2.at || m2.gg || m2.el))
    return fail(c, MS_ERR_UNSUPPORTED,
                "adjoint checkpoints are recording: phi noise, the anti-trapping current, grain growth and "
                "elasticity cannot be turned on (ms_enable_checkpoints(ctx, 0) first)");
  set_layout(m2);
  // keep the time line of the current state
  m2.t0 = c->m.t0;
  const HostModel before = c->m;
  c->m = m2;
  ms_status es = ensure_at_list(c);
  if (es == MS_OK) es = elastic_setup(c);
  if (es != MS_OK) {
    // the context keeps running with the parameters it had
    const std::string msg = c->err;
    c->m = before;
    ensure_at_list(c);
    elastic_setup(c);
    c->kern->fill(c->args.data(), c->m, c->lg.zchunk, c->status);
    return fail(c, es, msg);
  }
  c->kern->fill(c->args.data(), c->m, c->lg.zchunk, c->status);
  // recorded adjoint snapshots belong to the old parameters: the recording
  // restarts at the current step
  if (c->adj.every > 0 && c->step > c->adj.first_step) ms_reset_extra(c);
  return MS_OK;
}

ms_status ms_set_fields(ms_ctx* c, const void* phi, const void* mu, int on_device) {
  if (!c || !phi || !mu) return fail(c, MS_ERR_ARG, "ctx, phi and mu are required");
  MS_CUDA(c, copy_fields(c->m, c->buf[c->cur], 0, c->m.N, phi, nullptr, on_device, c->stream));
  MS_CUDA(c, copy_fields(c->m, c->buf[c->cur], c->m.N, c->m.NM, mu, nullptr, on_device, c->stream));
  MS_CUDA(c, fill_ghosts(c->m, c->buf[c->cur], c->m.N + c->m.NM, c->stream));
  ms_status rs = refresh_codes(c);
  if (rs != MS_OK) return rs;
  c->step = 0;
  c->t = c->m.t0;
  ms_reset_extra(c);
  return MS_OK;
}

ms_status ms_get_fields(ms_ctx* c, void* phi, void* mu, int on_device) {
  if (!c) return fail(nullptr, MS_ERR_ARG, "ctx is NULL");
  if (phi) MS_CUDA(c, copy_fields(c->m, c->buf[c->cur], 0, c->m.N, nullptr, phi, on_device, c->stream));
  if (mu) MS_CUDA(c, copy_fields(c->m, c->buf[c->cur], c->m.N, c->m.NM, nullptr, mu, on_device, c->stream));
  MS_CUDA(c, cudaStreamSynchronize(c->stream));
  return MS_OK;
}

ms_status ms_fields(ms_ctx* c, void** phi_dev, void** mu_dev, int64_t strides[4]) {
  if (!c) return fail(nullptr, MS_ERR_ARG, "ctx is NULL");
  const size_t s = c->m.dtype == MS_F64 ? 8 : 4;
  char* base = (char*)c->buf[c->cur] +
               ((long long)c->m.zoff * c->m.nyp * c->m.pitch + (long long)c->m.pitch + c->m.xoff) * s;
  if (phi_dev) *phi_dev = base;
  if (mu_dev) *mu_dev = base + (size_t)c->m.N * c->m.fstride * s;
  if (strides) {
    strides[0] = c->m.fstride;
    strides[1] = (int64_t)c->m.nyp * c->m.pitch;
    strides[2] = c->m.pitch;
    strides[3] = 1;
  }
  return MS_OK;
}

ms_status ms_step(ms_ctx* c, int64_t n) {
  TraceRange trace("ms_step");
  if (!c) return fail(nullptr, MS_ERR_ARG, "ctx is NULL");
  if (n < 0) return fail(c, MS_ERR_ARG, "n must be >= 0");
  for (int64_t i = 0; i < n; ++i) {
    if (c->fault_step >= 0 && c->step == c->fault_step) c->host_status = c->fault_code;
    if (c->host_status) return fail(c, (ms_status)c->host_status, "injected fault (MS_FAULT)");
    ms_status s = ms_before_step(c);
    if (s != MS_OK) return s;
    s = launch_one_step(c);
    if (s != MS_OK) return s;
    if (c->diag_every > 0 && c->step % c->diag_every == 0) {
      s = launch_diag_now(c);
      if (s != MS_OK) return s;
    }
  }
  return MS_OK;
}

ms_status ms_set_diag_every(ms_ctx* c, int64_t k) {
  if (!c || k < 0) return fail(c, MS_ERR_ARG, "bad argument");
  c->diag_every = k;
  return MS_OK;
}

static ms_status read_status(ms_ctx* c) {
  if (c->host_status) return fail(c, (ms_status)c->host_status, "injected fault (MS_FAULT)");
  int st = 0;
  MS_CUDA(c, cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  MS_CUDA(c, cudaStreamSynchronize(c->stream));
  if (st & kStatusTimeout) return fail(c, MS_ERR_TIMEOUT, "a bounded device wait timed out");
  if (st & kStatusLaunch) return fail(c, MS_ERR_BOUNDS, "launch geometry beyond a compiled limit");
  if (st & kStatusNonFinite) return fail(c, MS_ERR_NONFINITE, "non-finite values in the state");
  return MS_OK;
}

ms_status ms_sync(ms_ctx* c) {
  if (!c) return fail(nullptr, MS_ERR_ARG, "ctx is NULL");
  return read_status(c);
}

ms_status ms_diag(ms_ctx* c, double* out) {
  TraceRange trace("ms_diag");
  if (!c || !out) return fail(c, MS_ERR_ARG, "ctx and out are required");
  ms_status s = launch_diag_now(c);
  if (s != MS_OK) return s;
  const int nv = c->m.NM + 5;
  MS_CUDA(c, cudaMemcpyAsync(c->diag_host, c->diag_out, sizeof(double) * nv, cudaMemcpyDeviceToHost, c->stream));
  MS_CUDA(c, cudaStreamSynchronize(c->stream));
  const double* h = static_cast<const double*>(c->diag_host);
  for (int i = 0; i < nv; ++i) out[i] = h[i];
  out[nv] = (double)c->step;
  out[nv + 1] = c->t;
  return read_status(c);
}

ms_status ms_time(const ms_ctx* c, int64_t* step, double* t) {
  if (!c) return fail(nullptr, MS_ERR_ARG, "ctx is NULL");
  if (step) *step = c->step;
  if (t) *t = c->t;
  return MS_OK;
}

struct CkptHeader {
  char magic[8];
  int dim, N, NM, dtype, nx, ny, nz, pad;
  int64_t step;
  double t;
  uint64_t bytes;
};

size_t ms_checkpoint_bytes(const ms_ctx* c) {
  if (!c) return 0;
  return sizeof(CkptHeader) + c->state_bytes;
}

ms_status ms_checkpoint(ms_ctx* c, void* host_buf, size_t bytes) {
  if (!c || !host_buf || bytes < ms_checkpoint_bytes(c)) return fail(c, MS_ERR_ARG, "buffer too small");
  CkptHeader h = {};
  std::memcpy(h.magic, "MSGBCKP1", 8);
  h.dim = c->m.dim;
  h.N = c->m.N;
  h.NM = c->m.NM;
  h.dtype = c->m.dtype;
  h.nx = c->m.nx;
  h.ny = c->m.ny;
  h.nz = c->m.nz;
  h.step = c->step;
  h.t = c->t;
  h.bytes = c->state_bytes;
  std::memcpy(host_buf, &h, sizeof h);
  MS_CUDA(c, cudaMemcpyAsync((char*)host_buf + sizeof h, c->buf[c->cur], c->state_bytes, cudaMemcpyDeviceToHost,
                             c->stream));
  MS_CUDA(c, cudaStreamSynchronize(c->stream));
  return MS_OK;
}

ms_status ms_restore(ms_ctx* c, const void* host_buf, size_t bytes) {
  if (!c || !host_buf || bytes < ms_checkpoint_bytes(c)) return fail(c, MS_ERR_ARG, "buffer too small");
  CkptHeader h;
  std::memcpy(&h, host_buf, sizeof h);
  if (std::memcmp(h.magic, "MSGBCKP1", 8) != 0 || h.dim != c->m.dim || h.N != c->m.N || h.NM != c->m.NM ||
      h.dtype != c->m.dtype || h.nx != c->m.nx || h.ny != c->m.ny || h.nz != c->m.nz ||
      h.bytes != c->state_bytes)
    return fail(c, MS_ERR_ARG, "checkpoint does not match this context");
  MS_CUDA(c, cudaMemcpyAsync(c->buf[c->cur], (const char*)host_buf + sizeof h, c->state_bytes,
                             cudaMemcpyHostToDevice, c->stream));
  ms_status rs = refresh_codes(c);
  if (rs != MS_OK) return rs;
  MS_CUDA(c, cudaStreamSynchronize(c->stream));
  c->step = h.step;
  c->t = h.t;
  ms_reset_extra(c);
  return MS_OK;
}

int ms_tile_split(const ms_ctx* c, int tile) {
  if (!c) return -1;
  auto v = step_variants(c->m.dim, c->m.N, c->m.NM, c->m.dtype);
  if (tile < 0 || tile >= (int)v.size()) return -1;
  return v[tile]->split;
}

ms_status ms_get_launch(const ms_ctx* c, int* tile, int* zchunk) {
  if (!c) return fail(nullptr, MS_ERR_ARG, "ctx is NULL");
  auto v = step_variants(c->m.dim, c->m.N, c->m.NM, c->m.dtype);
  int idx = -1;
  for (size_t i = 0; i < v.size(); ++i)
    if (v[i] == c->kern) idx = (int)i;
  if (tile) *tile = idx;
  if (zchunk) *zchunk = c->lg.zchunk;
  return MS_OK;
}

int ms_tile_count(const ms_ctx* c) {
  if (!c) return 0;
  return (int)step_variants(c->m.dim, c->m.N, c->m.NM, c->m.dtype).size();
}

ms_status ms_tile_shape(const ms_ctx* c, int tile, int* tx, int* ty) {
  if (!c) return fail(nullptr, MS_ERR_ARG, "ctx is NULL");
  auto v = step_variants(c->m.dim, c->m.N, c->m.NM, c->m.dtype);
  if (tile < 0 || tile >= (int)v.size()) return MS_ERR_ARG;
  if (tx) *tx = v[tile]->tx;
  if (ty) *ty = v[tile]->ty;
  return MS_OK;
}

ms_status ms_set_launch(ms_ctx* c, int tile, int zchunk) {
  if (!c) return fail(nullptr, MS_ERR_ARG, "ctx is NULL");
  auto v = step_variants(c->m.dim, c->m.N, c->m.NM, c->m.dtype);
  if (tile < 0 || tile >= (int)v.size() || zchunk < 0) return fail(c, MS_ERR_ARG, "bad tile or zchunk");
  return apply_launch(c, v[tile], zchunk);
}

}  // extern "C"
