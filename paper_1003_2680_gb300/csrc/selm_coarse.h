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
  int half;           // shared v rows: even x at [0, half), odd x at [half, nx)
  int rp, pp;         // shared v row and plane pitch (elements; padded against bank conflicts)
  int sv, sb, st;     // shared-memory byte offsets of v (with 2 halo planes per side), b, t
  const T* S;         // [nz][45] stencil
  const T* zb;        // [nz][10]: s*Mz row (offsets -2..2), then s*Kz row
  T w1[9];            // Kx (x) My + Mx (x) Ky at (dy, dx) = index (dy+1)*3 + dx+1
  T w2[9];            // Mx (x) My
  float inv_nxc, inv_nyc;  // reciprocals for the colour-class rank decode
  int lx, ly;         // log2 of nx / ny when a power of two (index decode by shifts), else -1
  const int* rz_idx;  // restriction table to the next level
  const T* rz_w;
  const int* pz_idx;  // prolongation table from the next level
  const T* pz_w;
  const double* Linv; // coarsest level
  T* gb;              // global b of this component at this level
  T* gv;              // global v hand-off buffer
  T* gt;              // global residual buffer
};

// Per-colour class data of a level, staged in shared memory per CTA.
struct EngColour {
  int cx, cy, cz;       // class origin
  int nxc, nyc;         // class extents in x and y
  int rank_lo, nsite;   // ranks of the class owned by this CTA: [rank_lo, rank_lo + nsite)
  float inv_nxc, inv_nyc;
  int sx, sy;           // log2 of nxc / nyc when they are powers of two, else -1
};

constexpr int kEngMaxColours = 16;

template <typename T>
struct EngComp {
  EngLevel<T> lev[kMaxLevels];
};

// Plan of one system, uploaded once to device memory (read through L1 and
// staged level by level into shared memory by the kernel).
template <typename T>
struct EngParams {
  int l0, L, ncomp;
  int y_off;          // shared-memory byte offset of the FP64 coarsest scratch
  // Staged once per launch in shared memory, for every level l0..L-1: the
  // level descriptors (lev_off, one EngLevel per level), the colour classes
  // as this CTA sees them (col_off, kEngMaxColours per level) and the row
  // tables (tab_off + tab_row[l] rows of 12 values: 10 z bands, inverse
  // diagonal, noise scale).
  int lev_off, col_off, tab_off;
  int tab_row[kMaxLevels];
  // Transfer tables of level l < L-1, staged at xf_row[l] in a parallel int
  // array (xfi_off) and T array (xfw_off): prolongation from level l+1 by
  // fine row k at [2k, 2k+2), then restriction to level l+1 by coarse row K
  // at [2 nz_l + 4K, 2 nz_l + 4K + 4).
  int xfi_off, xfw_off;
  int xf_row[kMaxLevels];
  EngComp<T> comp[kMaxComps];
};

// Per-launch arguments.
struct EngRun {
  int mu1, mu2, coarse_mode;
  Key key;
  const unsigned long long* cyc;
};

template <typename T>
struct EnginePlanT {
  bool valid = false;
  int cluster = 1;
  size_t smem_bytes = 0;
  size_t y_off_comp[kMaxComps] = {};
  EngParams<T> params{};
  const EngParams<T>* dev = nullptr;   // device copy of params
};

// Bytes of device memory a system's plan occupies (reserved in the workspace).
constexpr size_t kEngParamBytes = 32768;

// Builds the plan for levels l0..L-1 (l0 >= min_level >= 1 chosen as the
// first level whose slabs fit in shared memory).  gb/gv/gt: per-level global
// field pointers.  dev_params: kEngParamBytes of device memory that receives
// the plan (copied on `st`, which is synchronised before returning).
// want_cluster > 0 caps the cluster size (the autotuner's knob).
template <typename T>
bool plan_coarse_engine(const LevelDev* levs, int L, void* const* gb, void* const* gv, void* const* gt,
                        void* dev_params, cudaStream_t st, EnginePlanT<T>* plan, int want_cluster = 0,
                        int min_level = 1);

// Runs the V-cycle below level l0-1: reads b at level l0, writes v at level l0.
template <typename T>
cudaError_t launch_coarse_engine(const EnginePlanT<T>& plan, int mu1, int mu2, int coarse_mode, bool noise, Key key,
                                 const unsigned long long* cyc, cudaStream_t st);

}  // namespace selm
