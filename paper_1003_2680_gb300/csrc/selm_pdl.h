// Programmatic dependent launch (sm_90 and later).
//
// A kernel launched with programmatic stream serialisation may start while
// the kernel before it on the stream is still running, once every block of
// that kernel has executed griddepcontrol.launch_dependents (or exited).  It
// must execute griddepcontrol.wait before it reads anything the earlier
// kernel writes: the wait returns when that kernel has completed and its
// memory operations are visible.  Its launch latency and whatever it does
// before the wait then overlap the earlier kernel's tail.  In a kernel
// launched the ordinary way both instructions return at once, so a kernel
// with them may be launched either way.
#pragma once

#include <cuda_runtime.h>

namespace selm {

__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// For kernels that read their inputs from the start: wait for the previous
// kernel, then let the next one launch.
__device__ __forceinline__ void pdl_enter() {
  pdl_wait();
  pdl_launch_dependents();
}

// Launches `kernel` on `st` with programmatic stream serialisation (the
// kernel must call pdl_wait() before reading the previous kernel's output).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace selm
