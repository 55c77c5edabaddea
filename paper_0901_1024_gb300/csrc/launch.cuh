// Programmatic dependent launch for the stage kernels.
//
// Consecutive stage kernels of a time step run back to back on one stream.
// Each is launched with programmatic stream serialization, and every CTA
// signals griddepcontrol.launch_dependents as it starts: the next kernel may
// then be scheduled while this one drains, run its set-up (tensor memory,
// barriers, constant operators), and block in griddepcontrol.wait -- which
// returns once the previous grid has completed and its writes are visible --
// before it touches a field array.  Each stage grid is at most one persistent
// wave, so every CTA of the previous grid has started before the next grid is
// launched and a waiting CTA never holds resources the previous grid needs.
#pragma once

#include <cuda_runtime.h>

#include "device.h"

namespace dgdev {

__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

inline cudaError_t launch_pdl(void (*kern)(const StageArgs), int grid, int threads, int smem,
                              cudaStream_t s, const StageArgs& a) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

}  // namespace dgdev
