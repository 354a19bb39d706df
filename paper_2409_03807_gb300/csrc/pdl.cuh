// Programmatic dependent launch: the kernels of one evaluation pass form a
// chain (hidden layers -> output layer -> element -> reduction -> select).
// Each is launched with programmatic stream serialisation and waits for its
// predecessor's completion and memory (griddepcontrol.wait) only after the
// prologue that does not read its predecessor's results (TMEM allocation,
// barrier set-up, tensor-map prefetch), which hides part of the launch
// latency between the dependent kernels.  The predecessors do not signal
// early (launch_dependents): scheduling the successor's CTAs while the
// predecessor runs measured slower.  Without the launch attribute the wait
// is a no-op, so the same kernels run under plain launches.
#pragma once
#include <cuda_runtime.h>

#include <utility>

namespace lsn {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args&&... args) {
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
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace lsn
