// Plan of the cluster-resident coarse-level engine (selm_coarse.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "selm_internal.h"
#include "selm_launch.h"

namespace selm {

// Levels with at most this many sites per component are held by one CTA.
constexpr long long kEngSingleMaxSites = 8192;

template <typename T>
struct EngLevel {
  int nx, ny, nz;
  int mx, my, mz, ncol;
  int comp_id;
  int cluster;        // 1: z-slabs over the cluster's CTAs; 0: held by CTA 0
  int P;              // planes per CTA (cluster levels) or nz (single levels)
  int sv, sb, st;     // shared-memory byte offsets of v (with 2 halo planes per side), b, t
  const T* S;         // [nz][45] stencil
  const int* rz_idx;  // restriction table to the next level
  const T* rz_w;
  const int* pz_idx;  // prolongation table from the next level
  const T* pz_w;
  const double* Linv; // coarsest level
  T* gb;              // global b of this component at this level
  T* gv;              // global v hand-off buffer
  T* gt;              // global residual buffer
};

template <typename T>
struct EngComp {
  EngLevel<T> lev[kMaxLevels];
};

template <typename T>
struct EngParams {
  int l0, L, ncomp;
  int mu1, mu2, coarse_mode;
  int y_off;          // shared-memory byte offset of the FP64 coarsest scratch
  Key key;
  const unsigned long long* cyc;
  EngComp<T> comp[kMaxComps];
};

template <typename T>
struct EnginePlanT {
  bool valid = false;
  int cluster = 1;
  size_t smem_bytes = 0;
  size_t y_off_comp[kMaxComps] = {};
  EngParams<T> params{};
};

// Builds the plan for levels l0..L-1 (l0 >= 1 chosen as the first level whose
// slabs fit in shared memory).  gb/gv/gt: per-level global field pointers.
template <typename T>
bool plan_coarse_engine(const LevelDev* levs, int L, void* const* gb, void* const* gv, void* const* gt,
                        EnginePlanT<T>* plan);

// Runs the V-cycle below level l0-1: reads b at level l0, writes v at level l0.
template <typename T>
cudaError_t launch_coarse_engine(const EnginePlanT<T>& plan, int mu1, int mu2, int coarse_mode, bool noise, Key key,
                                 const unsigned long long* cyc, cudaStream_t st);

}  // namespace selm
