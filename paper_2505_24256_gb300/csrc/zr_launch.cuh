// Programmatic dependent launches, shared by the step's kernels and the
// O(T log^2 T) path: a kernel launched with launch_k may become resident while
// the one before it on the stream drains.  Every such kernel first calls
// pdl_enter: griddepcontrol.wait holds it until its predecessors have
// completed and their memory is visible, then griddepcontrol.launch_dependents
// lets its own dependents start launching (they run once all of its CTAs have
// started).  In a kernel launched without the attribute the wait returns at
// once.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace zr {

static __device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <class... P, class... A>
static cudaError_t launch_k(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                            A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

}  // namespace zr
