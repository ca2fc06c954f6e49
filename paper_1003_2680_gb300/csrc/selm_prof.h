// Kernel accounting shared by the kernel translation units: every launch is
// counted; with profiling on it is bracketed by CUDA events on its stream.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

namespace selm {
namespace prof {
// Launches so far (every Scope counts one; replays of captured graphs add
// their captured count) and whether launches are bracketed by events.
extern std::atomic<long long> g_launches;
extern bool g_on;
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
