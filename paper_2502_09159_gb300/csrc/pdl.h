// Programmatic dependent launch (sm_90 and later): a kernel launched with pdl_launch may be
// scheduled while its predecessor in the stream is still finishing.  Every such kernel
// calls pdl_wait() before it reads or writes memory that its predecessor touches (the
// wait returns once the predecessor grid has completed and its writes are visible), and
// pdl_trigger() to let its own successor be scheduled early.  Without a programmatic
// predecessor both are no-ops, so the kernels are also correct under an ordinary launch.
#pragma once

#include <cuda_runtime.h>

namespace stmg {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace stmg
