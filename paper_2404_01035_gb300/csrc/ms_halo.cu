// Halo exchange between z-slab contexts (slab decomposition of one domain).
// Every context stores NF padded fields [nzp][nyp][pitch] and a code array
// [nzp][ny][segs]; plane index z + 1 holds interior plane z, indices 0 and
// nz + 1 the ghost planes.  One exchange moves one whole padded plane per
// field (including the x/y ghost rows the step kernel wrote) and one code
// plane in each direction.
#include <cuda_runtime.h>

#include "../../include/microsim_gb.h"
#include "ms_rt.h"

using namespace msgb;

namespace {

cudaError_t copy_plane(ms_ctx* dst, int dst_plane, ms_ctx* src, int src_plane, cudaStream_t st) {
  const HostModel& m = src->m;
  const size_t s = m.dtype == MS_F64 ? 8 : 4;
  const size_t plane = (size_t)m.nyp * m.pitch * s;
  const int nf = m.N + m.NM;
  for (int f = 0; f < nf; ++f) {
    const char* from = static_cast<const char*>(src->buf[src->cur]) + ((size_t)f * m.fstride) * s + src_plane * plane;
    char* to = static_cast<char*>(dst->buf[dst->cur]) + ((size_t)f * dst->m.fstride) * s + dst_plane * plane;
    cudaError_t e = cudaMemcpyAsync(to, from, plane, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
  }
  const size_t cplane = (size_t)segments(m) * m.ny;
  return cudaMemcpyAsync(dst->codes[dst->cur] + dst_plane * cplane, src->codes[src->cur] + src_plane * cplane,
                         cplane, cudaMemcpyDeviceToDevice, st);
}

// One padded plane of every field, then the plane's segment codes, to
// (pack) or from (unpack) a flat device buffer laid out as
// [field][nyp][pitch] elements followed by [ny][segs] code bytes.
cudaError_t move_plane(ms_ctx* c, int plane_idx, char* flat, bool pack) {
  const HostModel& m = c->m;
  const size_t s = m.dtype == MS_F64 ? 8 : 4;
  const size_t plane = (size_t)m.nyp * m.pitch * s;
  const int nf = m.N + m.NM;
  for (int f = 0; f < nf; ++f) {
    char* st = static_cast<char*>(c->buf[c->cur]) + ((size_t)f * m.fstride) * s + plane_idx * plane;
    cudaError_t e = pack ? cudaMemcpyAsync(flat + f * plane, st, plane, cudaMemcpyDeviceToDevice, c->stream)
                         : cudaMemcpyAsync(st, flat + f * plane, plane, cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return e;
  }
  const size_t cplane = (size_t)segments(m) * m.ny;
  uint8_t* code = c->codes[c->cur] + plane_idx * cplane;
  char* fc = flat + nf * plane;
  return pack ? cudaMemcpyAsync(fc, code, cplane, cudaMemcpyDeviceToDevice, c->stream)
              : cudaMemcpyAsync(code, fc, cplane, cudaMemcpyDeviceToDevice, c->stream);
}

bool compatible(const ms_ctx* a, const ms_ctx* b) {
  return a->m.dim == 3 && b->m.dim == 3 && a->m.nx == b->m.nx && a->m.ny == b->m.ny && a->m.N == b->m.N &&
         a->m.NM == b->m.NM && a->m.dtype == b->m.dtype && a->m.pitch == b->m.pitch && a->m.nyp == b->m.nyp &&
         a->stream == b->stream && a->m.bc[2] == kBcHalo && b->m.bc[2] == kBcHalo;
}

}  // namespace

extern "C" {

ms_status ms_halo_exchange(ms_ctx* lower, ms_ctx* upper) {
  if (!lower || !upper) return fail(nullptr, MS_ERR_ARG, "contexts are required");
  if (!compatible(lower, upper))
    return fail(lower, MS_ERR_ARG,
                "halo exchange needs two 3-D contexts with z faces MS_BC_HALO and equal nx, ny, N, K, dtype, stream");
  cudaStream_t st = lower->stream;
  // lower's top interior plane (index nz) -> upper's bottom ghost (index 0)
  cudaError_t e = copy_plane(upper, 0, lower, lower->m.nz, st);
  // upper's bottom interior plane (index 1) -> lower's top ghost (index nz + 1)
  if (e == cudaSuccess) e = copy_plane(lower, lower->m.nz + 1, upper, 1, st);
  if (e != cudaSuccess) return cuda_fail(lower, e, "halo exchange");
  return MS_OK;
}

ms_status ms_halo_mirror(ms_ctx* c, int face) {
  if (!c || (face != 0 && face != 1)) return fail(c, MS_ERR_ARG, "bad argument");
  if (c->m.dim != 3 || c->m.bc[2] != kBcHalo) return fail(c, MS_ERR_ARG, "context has no halo faces");
  cudaError_t e = face == 0 ? copy_plane(c, 0, c, 1, c->stream) : copy_plane(c, c->m.nz + 1, c, c->m.nz, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "halo mirror");
  return MS_OK;
}

size_t ms_halo_plane_bytes(const ms_ctx* c) {
  if (!c || c->m.dim != 3) return 0;
  const HostModel& m = c->m;
  const size_t s = m.dtype == MS_F64 ? 8 : 4;
  return (size_t)(m.N + m.NM) * m.nyp * m.pitch * s + (size_t)segments(m) * m.ny;
}

ms_status ms_halo_pack(ms_ctx* c, int face, void* dst) {
  if (!c || !dst || (face != 0 && face != 1)) return fail(c, MS_ERR_ARG, "bad argument");
  if (c->m.dim != 3 || c->m.bc[2] != kBcHalo) return fail(c, MS_ERR_ARG, "context has no halo faces");
  cudaError_t e = move_plane(c, face == 0 ? 1 : c->m.nz, static_cast<char*>(dst), true);
  if (e != cudaSuccess) return cuda_fail(c, e, "halo pack");
  return MS_OK;
}

ms_status ms_halo_unpack(ms_ctx* c, int face, const void* src) {
  if (!c || !src || (face != 0 && face != 1)) return fail(c, MS_ERR_ARG, "bad argument");
  if (c->m.dim != 3 || c->m.bc[2] != kBcHalo) return fail(c, MS_ERR_ARG, "context has no halo faces");
  cudaError_t e = move_plane(c, face == 0 ? 0 : c->m.nz + 1, const_cast<char*>(static_cast<const char*>(src)), false);
  if (e != cudaSuccess) return cuda_fail(c, e, "halo unpack");
  return MS_OK;
}

}  // extern "C"
