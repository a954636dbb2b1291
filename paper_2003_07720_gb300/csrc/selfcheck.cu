// Self-check of the bounded waits of the asynchronous-copy kernels.
#include "async_copy.cuh"
#include "rpm_internal.h"

namespace rpm {

// Self-check of the bounded barrier wait the bulk-copy passes rely on: one
// thread arms an mbarrier for 16 bytes that no copy will ever deliver and
// waits; the wait must give up by itself (about one second, global timer)
// and the kernel must return.  out[0] = 1 when it gave up, 0 otherwise.
__global__ void k_wait_selfcheck(int* out) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
    mbar_arrive_expect_tx(&bar, 16);
    out[0] = mbar_wait(&bar, 0) ? 0 : 1;
  }
}

cudaError_t launch_wait_selfcheck(int* out, cudaStream_t st) {
  k_wait_selfcheck<<<1, 32, 0, st>>>(out);
  return cudaGetLastError();
}

}  // namespace rpm
