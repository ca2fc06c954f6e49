// Kernel accounting shared by the kernel translation units: every launch is
// counted; with profiling on it is bracketed by CUDA events on its stream.
#pragma once

#include <cuda_runtime.h>

namespace selm {
namespace prof {
struct Scope {
  int kind;
  cudaStream_t st;
  cudaEvent_t a;
  Scope(int k, cudaStream_t s);
  ~Scope();
  Scope(const Scope&) = delete;
  Scope& operator=(const Scope&) = delete;
};
}  // namespace prof
}  // namespace selm
