// pdl.h -- programmatic dependent launch.
//
// A kernel launched with launch_pdl may start while the preceding kernel of
// its stream is still running: it calls grid_dep_wait() before touching
// anything that kernel writes (the wait returns once the preceding kernel has
// completed and its writes are visible; at once for a kernel launched
// without the attribute).  grid_dep_launch() lets the following kernel be
// launched before this one ends.  In a captured graph the attribute becomes a
// programmatic edge between the two kernel nodes.
#pragma once

#include <cuda_runtime.h>

namespace bd {

__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" :::); }

template <typename... Params, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

}  // namespace bd
