// Self-test of the stage kernels' bounded mbarrier wait (wait_or_flag): one
// warp waits, with `polls` polls at most, on an mbarrier that nothing arrives
// at, so the wait runs out and sets the pipeline status word exactly as a
// stage kernel's timed-out wait does.  Nothing else is in flight (no tensor
// memory, MMA or bulk copy), so the kernel just returns.
#include <cuda_runtime.h>

#include "device.h"
#include "tc_stage.cuh"

namespace dgdev {

__global__ void wait_selftest_kernel(int* status, uint32_t polls, unsigned long long* ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
  }
  __syncthreads();
  unsigned long long t0, t1;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  wait_or_flag(&bar, 0, status, polls);          // phase 0 never completes
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
  if (threadIdx.x == 0) *ns = t1 - t0;
}

cudaError_t launch_wait_selftest(int* status, uint32_t polls, unsigned long long* ns,
                                 cudaStream_t s) {
  wait_selftest_kernel<<<1, 32, 0, s>>>(status, polls, ns);
  return cudaGetLastError();
}

}  // namespace dgdev
