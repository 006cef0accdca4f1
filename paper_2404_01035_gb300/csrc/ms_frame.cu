// Moving frame (the SHIFT key of the paper's input files, Sec. 4 "moving
// camera"): the already solidified start of the domain is dropped, the rest
// moves down along the last axis and the far end is filled with liquid of the
// original alloy, while the grid's lab origin advances so that the pulled
// temperature field (and the phi-noise counter) stay in lab coordinates.
#include <cuda_runtime.h>

#include <string>

#include "ms_rt.h"

namespace msgb {
namespace {

// dst(x, y, z) = src at `planes` cells further along the last axis, or the
// fill state (pure last phase, mu = fill) past the end.  One thread per
// interior cell; every field.
template <class Real>
__global__ void k_shift(const Real* __restrict__ src, Real* __restrict__ dst, int dim, int nx, int ny, int nz,
                        int pitch, int nyp, long long fstride, int xoff, int zoff, int N, int NM, int planes,
                        Real f0, Real f1, Real f2) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long cells = (long long)nx * ny * nz;
  if (i >= cells) return;
  const int x = (int)(i % nx);
  const int y = (int)((i / nx) % ny);
  const int z = (int)(i / ((long long)nx * ny));
  const int last = dim == 3 ? z : y, n = dim == 3 ? nz : ny;
  const long long plane = (long long)nyp * pitch;
  const long long od = (long long)(z + zoff) * plane + (long long)(y + 1) * pitch + x + xoff;
  const bool inside = last + planes < n;
  const long long os = od + (long long)planes * (dim == 3 ? plane : (long long)pitch);
  const Real fill[3] = {f0, f1, f2};
  for (int f = 0; f < N + NM; ++f) {
    Real v;
    if (inside)
      v = src[f * fstride + os];
    else
      v = f < N ? (f == N - 1 ? Real(1) : Real(0)) : fill[f - N];
    dst[f * fstride + od] = v;
  }
}

// Highest index along the last axis holding a cell that is not pure last
// phase (atomic max; *out preset to -1).
template <class Real>
__global__ void k_front(const Real* __restrict__ st, int dim, int nx, int ny, int nz, int pitch, int nyp,
                        long long fstride, int xoff, int zoff, int N, int* out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long cells = (long long)nx * ny * nz;
  if (i >= cells) return;
  const int x = (int)(i % nx);
  const int y = (int)((i / nx) % ny);
  const int z = (int)(i / ((long long)nx * ny));
  const long long o = (long long)(z + zoff) * nyp * pitch + (long long)(y + 1) * pitch + x + xoff;
  if (st[(N - 1) * fstride + o] != Real(1)) atomicMax(out, dim == 3 ? z : y);
}

}  // namespace
}  // namespace msgb

using namespace msgb;

extern "C" {

ms_status ms_shift(ms_ctx* c, int planes, const double* mu_fill) {
  if (!c) return fail(nullptr, MS_ERR_ARG, "ctx is NULL");
  const HostModel& m = c->m;
  const int n = m.dim == 3 ? m.nz : m.ny;
  if (planes < 0 || planes > n) return fail(c, MS_ERR_ARG, "planes must be in [0, extent of the last axis]");
  if (m.dim == 3 && m.bc[2] == kBcHalo)
    return fail(c, MS_ERR_UNSUPPORTED, "a slab of a decomposed domain cannot shift on its own");
  if (m.NM > 0 && !mu_fill) return fail(c, MS_ERR_ARG, "mu_fill is required");
  if (planes == 0) return MS_OK;
  double f[3] = {0, 0, 0};
  for (int i = 0; i < m.NM && i < 3; ++i) f[i] = mu_fill[i];
  const long long cells = (long long)m.nx * m.ny * m.nz;
  const int blocks = (int)((cells + 255) / 256);
  void* src = c->buf[c->cur];
  void* dst = c->buf[1 - c->cur];
  if (m.dtype == MS_F64)
    k_shift<double><<<blocks, 256, 0, c->stream>>>((const double*)src, (double*)dst, m.dim, m.nx, m.ny, m.nz, m.pitch,
                                                    m.nyp, m.fstride, m.xoff, m.zoff, m.N, m.NM, planes, f[0], f[1],
                                                    f[2]);
  else
    k_shift<float><<<blocks, 256, 0, c->stream>>>((const float*)src, (float*)dst, m.dim, m.nx, m.ny, m.nz, m.pitch,
                                                   m.nyp, m.fstride, m.xoff, m.zoff, m.N, m.NM, planes, (float)f[0],
                                                   (float)f[1], (float)f[2]);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = fill_ghosts(m, dst, m.N + m.NM, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "frame shift");
  c->cur = 1 - c->cur;
  c->m.zorg += planes;
  c->kern->fill(c->args.data(), c->m, c->lg.zchunk, c->status);
  ms_reset_extra(c);   // snapshots of the adjoint belong to the old frame
  return refresh_codes(c);
}

ms_status ms_front(ms_ctx* c, int* last_plane) {
  if (!c || !last_plane) return fail(c, MS_ERR_ARG, "ctx and last_plane are required");
  const HostModel& m = c->m;
  int* dev = reinterpret_cast<int*>(c->small + 64);
  cudaError_t e = cudaMemsetAsync(dev, 0xFF, sizeof(int), c->stream);   // -1
  const long long cells = (long long)m.nx * m.ny * m.nz;
  const int blocks = (int)((cells + 255) / 256);
  if (e == cudaSuccess) {
    if (m.dtype == MS_F64)
      k_front<double><<<blocks, 256, 0, c->stream>>>((const double*)c->buf[c->cur], m.dim, m.nx, m.ny, m.nz, m.pitch,
                                                      m.nyp, m.fstride, m.xoff, m.zoff, m.N, dev);
    else
      k_front<float><<<blocks, 256, 0, c->stream>>>((const float*)c->buf[c->cur], m.dim, m.nx, m.ny, m.nz, m.pitch,
                                                     m.nyp, m.fstride, m.xoff, m.zoff, m.N, dev);
    e = cudaGetLastError();
  }
  int* host = reinterpret_cast<int*>(c->diag_host);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "front");
  *last_plane = *host;
  return MS_OK;
}

}  // extern "C"
