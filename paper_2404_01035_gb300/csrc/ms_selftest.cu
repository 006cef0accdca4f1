// Failure-path self-test of a context's bounded device waits.
//
// The step kernels wait on mbarriers (the TMA ring) and the batched kernel on
// a grid barrier, each giving up after a fixed limit of %globaltimer time and
// recording MS_ERR_TIMEOUT in the context's sticky status word.  Those waits
// cannot be made to run out on purpose without leaving bulk copies in
// flight, so this entry point exercises the same bounded-wait routine and
// the same status path on a wait that nothing can complete: one thread waits
// on a freshly initialised mbarrier (one expected arrival, none coming) with
// a caller-given limit, records the timeout, then makes the arrival itself
// so that the barrier is left complete before the block exits.  No memory
// copy is in flight at any point.
#include <cuda_runtime.h>

#include "ms_device.cuh"
#include "ms_rt.h"

using namespace msgb;

namespace {

__global__ void k_wait_probe(int* status, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!mbar_wait_bounded(&bar, 0, limit_ns)) atomicOr(status, kStatusTimeout);
    mbar_arrive(&bar);
  }
}

}  // namespace

extern "C" ms_status ms_selftest_timeout(ms_ctx* c, int64_t limit_ns) {
  if (!c) return fail(nullptr, MS_ERR_ARG, "ctx is NULL");
  if (limit_ns < 1000 || limit_ns > 1000000000ll)
    return fail(c, MS_ERR_ARG, "limit_ns must lie in [1e3, 1e9] nanoseconds");
  k_wait_probe<<<1, 32, 0, c->stream>>>(c->status, (unsigned long long)limit_ns);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "wait self-test launch");
  return MS_OK;
}
