// Handle internals shared by the C-ABI translation units (not public ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/selm_mg.h"
#include "selm_coarse.h"
#include "selm_internal.h"
#include "selm_launch.h"

namespace selm {

struct Sys {
  HostSystem host;
  LevelDev lev[kMaxLevels];
  void* v[kMaxLevels] = {};
  void* b[kMaxLevels] = {};
  void* t[kMaxLevels] = {};
  int levels = 0;
  int ncomp = 0;
  EnginePlanT<float> engf;    // cluster-resident coarse levels (FP32 inner)
  EnginePlanT<double> engd;   // (FP64 inner)
  bool use_engine = true;
  int engine_cluster = 0;     // preferred cluster size of the engine (0 = largest that fits)
  int engine_level = 0;       // first level the engine may take (0 = the first that fits)
  void* eng_dev = nullptr;    // device slot of the engine plan
  bool use_coop = true;       // levels above the engine: cooperative launches (else one per pass)
  bool coop_flow = true;      // FP32 cooperative passes in dataflow order where the level allows it
  unsigned* coop_bar = nullptr;   // grid-barrier words of the system's cooperative launches
};

template <typename T>
inline EnginePlanT<T>& eng_of(Sys& s);
template <>
inline EnginePlanT<float>& eng_of<float>(Sys& s) {
  return s.engf;
}
template <>
inline EnginePlanT<double>& eng_of<double>(Sys& s) {
  return s.engd;
}

// Byte layout of the workspace.
struct Layout {
  size_t total = 0;
  size_t add(size_t bytes) {
    size_t off = (total + 255) & ~(size_t)255;
    total = off + bytes;
    return off;
  }
};

}  // namespace selm

struct selm_mg {
  selm_mg_desc d{};
  int mu1 = 2, mu2 = 2;
  int esize = 8;
  selm::Sys vel, pres;
  bool has_pres = false;
  // The chain's copy of the velocity system: the same operators and launch
  // plans over level fields of its own (with its own coarse-engine plan and
  // grid-barrier words), so that the chain cycles of a step can run on the
  // side stream while the velocity solve runs on the work stream.  Present
  // with the side stream (has_chain).
  selm::Sys chn;
  bool has_chain = false;
  selm::Key key{};
  char* ws = nullptr;
  size_t ws_bytes = 0;
  double* u = nullptr;      // solution of the deterministic solve (FP64)
  double* xi = nullptr;     // chain state (FP64)
  double* bvel = nullptr;   // right-hand side (FP64)
  double* wcomb = nullptr;  // combined field for the particle update (FP64)
  double* phi = nullptr;    // pressure (FP64), 3 slots: warm starts of the projections
                            // of Gamma^T F (0), of the step's combined field (1), of the
                            // sampled field (2)
  double* prhs = nullptr;   // pressure right-hand side (FP64)
  void* spec = nullptr;     // spectral pressure solve scratch (null: not available)
  bool spectral = false;    // projection's inner solves spectral instead of V-cycles
  double* red = nullptr;    // reduction slots
  unsigned long long* cyc = nullptr;  // [0] chain counter, [1] stage-call counter
  double* V = nullptr;      // particle scratch [max_particles][3]
  double* Xs = nullptr;     // device copies of host particle arrays (selm_mg_step_host)
  double* Fs = nullptr;
  double* host_red = nullptr;  // host word for norm read-backs
  // Side stream for the chain cycles of a step, which depend only on the
  // previous chain state: they run on the chain's own level fields beside
  // the spread, the first projection and the velocity solve, and join before
  // the step combines the solve with the chain state.
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // high-priority stream of the step's main path while the chain runs beside
  // it (forked from and joined back to the caller's stream)
  cudaStream_t prio = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // norm read-back beside the work stream: the solve enqueues its next
  // V-cycle before the copy (see fac_solve)
  cudaStream_t xfer = nullptr;
  cudaEvent_t ev_norm = nullptr;
  // CUDA graphs of the internal V-cycles (the handle's level-0 buffers),
  // keyed by system, noise and counter; captured on `cap`, replayed on the
  // work stream.  Dropped whenever the launch plans change.
  struct VGraph {
    cudaGraphExec_t exec = nullptr;
    const selm::Sys* sys = nullptr;
    bool noise = false;
    const unsigned long long* cyc = nullptr;
    int uses = 0;              // direct runs before the capture (first run initialises lazily)
    long long launches = 0;    // kernel launches in the graph
  };
  VGraph vg[4];
  cudaStream_t cap = nullptr;
  bool graphs = true;
  bool speculate = true;      // solves enqueue the next V-cycle before reading the norm
  uint64_t cycle = 0;
  // scratch of the exact Stokes solve (allocated on its first use) and the
  // step counter of the drift directions
  void* stokes = nullptr;
  size_t stokes_bytes = 0;
  uint64_t stokes_step = 0;
  int last_solve_cycles = 0, last_proj_cycles = 0;
  long long total_vcycles = 0;
  std::string err;
};

namespace selm {

// Asynchronous building blocks (no host synchronisation; safe under stream
// capture).  All return SELM_OK or SELM_ECUDA with h->err set.
selm_status vcycle(selm_mg* h, Sys& s, void* v0, const void* b0, bool noise, const unsigned long long* cyc,
                   cudaStream_t st);
selm_status outer_residual(selm_mg* h, Sys& s, const double* z, const double* b, void* r, double* norm2,
                           cudaStream_t st);
selm_status outer_update(selm_mg* h, Sys& s, double* z, const void* d, cudaStream_t st);
// Re-plans the coarse engines with a preferred cluster size (0 = largest that
// fits) and each system's first engine level.
selm_status replan_engine(selm_mg* h, int cluster, cudaStream_t st);

// A handle around a prepared host hierarchy (one system, no projection), with
// V-cycle scratch only plus `extra_bytes` of workspace for the caller at
// *extra_off.  Level rb_level (if >= 0) is smoothed red-black; the engine
// starts at engine_level at the earliest.  The composite form builds on it.
selm_status create_with_host(const selm_mg_desc& d, const HostSystem& host, int engine_level, bool use_coop,
                             int rb_level, size_t extra_bytes, cudaStream_t st, selm_mg** out, size_t* extra_off);
size_t footprint_with_host(const selm_mg_desc& d, const HostSystem& host, size_t extra_bytes);
// One V-cycle (Algorithm 3) of system s from `level` down, on the internal
// level fields: reads s.b[level], writes s.v[level] (which must hold its
// initial value, normally 0).
selm_status vcycle_level(selm_mg* h, Sys& s, int level, bool noise, const unsigned long long* cyc, cudaStream_t st);
// `ncycles` stochastic FAC cycles of the handle's chain xi (b = 0).
selm_status chain_advance(selm_mg* h, int ncycles, cudaStream_t st);
// Frees the Stokes scratch (selm_stokes.cu).
void stokes_release(selm_mg* h);

}  // namespace selm
