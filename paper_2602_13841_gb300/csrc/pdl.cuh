// Programmatic dependent launch (sm_90 and later) for the kernels of the V-cycle chain.
//
// A kernel launched by launch_pdl may be scheduled while the kernel before it in the stream is
// still draining, which hides the launch gap between the many short, dependent launches of a
// V-cycle (every level runs ten or more of them per smoothing sweep).  Each kernel launched this
// way calls pdl_enter() as its first statement, before it touches global memory:
// griddepcontrol.wait returns once every prerequisite grid has completed and its writes are
// visible (at once for a kernel launched without the attribute), and
// griddepcontrol.launch_dependents then allows the next kernel of the stream to be scheduled.
#pragma once
#include <cuda_runtime.h>

namespace stmg {

__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace stmg
