// Self-check of the failure path: a kernel whose bounded wait is made to
// expire on purpose, so that tests can see, on the GPU, an expired wait turn
// into a status code the host reads while the context stays usable.  The
// kernels' own waits use the same bounded-wait routine with a ~1 s limit.
#include <cuda_runtime.h>

#include "dd_errors.h"
#include "dd_internal.h"
#include "ptx.cuh"

namespace dd {

// One warp waits on phase 0 of an mbarrier that expects one arrival and gets
// none; the wait gives up after `limit` cycles and the kernel records the
// timeout code, exactly as the forward kernels do.
__global__ void wait_timeout_selfcheck(int* status, long long limit) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const bool done = mbar_wait_bounded(&bar, 0, limit);
  if (!done && threadIdx.x == 0) report_error(status, kDevWaitTimeout);
}

}  // namespace dd

using namespace dd;

extern "C" dd_status dd_check_wait_timeout(dd_plan_t plan, int64_t limit_cycles, void* stream) {
  clear_error();
  if (!plan) return set_error(DD_ERR_ARG, "dd_check_wait_timeout: plan is NULL");
  if (limit_cycles < 1 || limit_cycles > kWaitLimitCycles)
    return set_error(DD_ERR_ARG, "dd_check_wait_timeout: limit_cycles must be in [1, %lld]", kWaitLimitCycles);
  wait_timeout_selfcheck<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(plan->d_status, limit_cycles);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_cuda_error("dd_check_wait_timeout: launch", e);
  return DD_OK;
}
