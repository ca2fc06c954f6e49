// Kernel launchers (defined in selm_kernels.cu, used by the C-ABI layer).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "selm_internal.h"

namespace selm {

struct Key {
  uint32_t k0, k1;
};

// Stage kernels.  `T` is float or double (inner precision); all launches go
// on `st`.  Counters (`cyc`) are read from device memory so that the calls can
// be captured in CUDA graphs.
template <typename T>
cudaError_t launch_smooth(const LevelDev& L, T* v, const T* b, int sweep, bool noise, Key key,
                          const unsigned long long* cyc, cudaStream_t st);
template <typename T>
cudaError_t launch_residual(const LevelDev& L, const T* v, const T* b, T* t, cudaStream_t st);
template <typename T>
cudaError_t launch_restrict(const LevelDev& Lf, const LevelDev& Lc, const T* t, T* bc,
                            cudaStream_t st);
template <typename T>
cudaError_t launch_prolong(const LevelDev& Lf, const LevelDev& Lc, T* v, const T* vc,
                           cudaStream_t st);
// One Galerkin level (L.level >= 1) as a single cooperative launch over the
// GPU.  phase 0: the descending half of the V-cycle at this level (mu1
// sweeps from the zero start in v, residual into t, restriction into bc,
// vc = 0); phase 1: the ascending half (v += P vc, then mu2 sweeps).  `bar`:
// 4 zeroed, 8-byte aligned words of device memory, the launch's grid barrier,
// reserved for the launches of one stream order (two launches that may
// overlap need distinct words).  flow (FP32, levels with L.flow): the colour
// passes run in dataflow order, each update waiting only for its coupled
// neighbours (the parity of their update count in the value's last bit)
// instead of a grid barrier between passes.
// After a barrier wait timed out, bar[2] is non-zero, the level's result is
// undefined and the caller reports the error and zeroes the words.
// level_coop_supported() tells whether the device and the level admit it.
template <typename T>
cudaError_t launch_level_coop(const LevelDev& L, const LevelDev& Lc, int phase, int mu1, int mu2, T* v, const T* b,
                              T* t, T* bc, T* vc, unsigned* bar, bool flow, bool noise, Key key,
                              const unsigned long long* cyc, cudaStream_t st);
template <typename T>
bool level_coop_supported(const LevelDev& L);
template <typename T>
cudaError_t launch_coarsest(const LevelDev& L, T* v, const T* b, bool noise, Key key,
                            const unsigned long long* cyc, cudaStream_t st);
template <typename T>
cudaError_t launch_outer_residual(const LevelDev& L0, const double* z, const double* b, T* r,
                                  double* norm2, cudaStream_t st);
template <typename T>
cudaError_t launch_outer_update(long long n, double* z, const T* d, cudaStream_t st);

cudaError_t launch_norm2(long long n, const double* x, double* out, cudaStream_t st);
cudaError_t launch_axpby(long long n, double a, const double* x, double c, const double* y,
                         double* out, cudaStream_t st);
cudaError_t launch_set_u64(unsigned long long* p, unsigned long long v, cudaStream_t st);
cudaError_t launch_inc_u64(unsigned long long* p, cudaStream_t st);

// Particle coupling (velocity system, level 0).
cudaError_t launch_spread(const LevelDev& L0, int n, int dim, int np, const double* X,
                          const double* F, double* b, cudaStream_t st);
cudaError_t launch_interp(const LevelDev& L0, int n, int dim, int np, const double* X,
                          const double* u, double* U, cudaStream_t st);
cudaError_t launch_em(int np, int dim, double* X, const double* V, cudaStream_t st);

// MAC projection pieces.
cudaError_t launch_divergence(const LevelDev& Lv, const double* w, double* div, double* sum,
                              cudaStream_t st);
cudaError_t launch_sub_mean(long long n, double* x, const double* sum, cudaStream_t st);
cudaError_t launch_grad_sub(const LevelDev& Lv, double* w, const double* phi, cudaStream_t st);

cudaError_t launch_philox(const uint32_t* ctr, Key key, uint32_t* out, int n, cudaStream_t st);

// Spectral inner solve of the uniform channel's Neumann pressure problem
// (selm_spectral.cu): delta = A^-1 r up to FP32 rounding (FFT along x and y,
// Thomas along z); `spectrum`: spectral_pressure_bytes() of scratch.
bool spectral_pressure_supported(const LevelDev& L0);
size_t spectral_pressure_bytes(const LevelDev& L0);
cudaError_t spectral_pressure_solve(const LevelDev& L0, const float* r, float* delta, void* spectrum,
                                    cudaStream_t st);

// ---- batched FAC cycles as one persistent launch ----------------------------
// One system of a batch as the persistent launch sees it (device pointers of
// its handle).
struct BatchSysHost {
  int levels;
  int esize;                     // inner precision bytes (the same for all systems)
  bool cholesky;                 // exact coarsest step (required)
  const LevelDev* lev;           // [levels]
  void* const* v;                // [levels] level fields
  void* const* b;
  void* const* t;
  Key key;
  unsigned long long* cyc;       // [0] chain counter, [1] solve stage counter
  double* u;                     // solve iterate (FP64)
  double* xi;                    // chain state (FP64)
  const double* bvel;            // solve right-hand side (FP64)
};
struct BatchPersist;
bool batch_persist_eligible(int nsys, const BatchSysHost* sys);
// Device plan of the batch (allocates device memory for its tables).
cudaError_t batch_persist_create(int nsys, const BatchSysHost* sys, int mu1, int mu2, BatchPersist** out);
void batch_persist_destroy(BatchPersist* bp);
// Tile shape: level-0 column items of kc z rows; bps co-resident blocks per SM.
cudaError_t batch_persist_configure(BatchPersist* bp, int kc, int bps);
void batch_persist_shape(const BatchPersist* bp, int* kc, int* bps);
// kind 0: one stochastic cycle of every chain (counters advance);
// kind 1: one pipelined solve cycle (V-cycle on the residual already in each
//         system's level-0 rhs with v0 = 0, update of u, next residual and its
//         squared norm into batch_persist_norms()[i], v0 = 0);
// kind 2: one solve cycle from u (residual, V-cycle, update).
// tstamp (optional, device, nphase + 1 words): %globaltimer at the start and
// after each phase's barrier, as block 0 sees it.
cudaError_t batch_persist_launch(BatchPersist* bp, int kind, cudaStream_t st, unsigned long long* tstamp = nullptr);
const double* batch_persist_norms(const BatchPersist* bp);
// Phases of a launch kind (types: BatchPhaseType codes, levels); returns the count.
int batch_persist_phases(const BatchPersist* bp, int kind, int* types, int* levels);
// Grid-barrier words of the launches ([2] != 0: a wait timed out).
const unsigned* batch_persist_bar(const BatchPersist* bp);

}  // namespace selm
