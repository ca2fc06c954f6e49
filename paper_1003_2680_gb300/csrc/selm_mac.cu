// Staggered composite grid: device plan, kernels and the C ABI.
//
// Every operator of the composite MAC grid (velocity operator, divergence,
// gradient, pressure operator, FAC transfers, Galerkin base operators, the
// extension to the fine lattice) is an explicit sparse matrix built on the
// host (selm_mac_setup.cpp).  On the device each is a sliced ELL matrix:
// slices of 32 consecutive list positions, slice s holding swid[s] entries
// per position at soff[s] + e * 32 + lane, so that a warp reads its 32 rows'
// e-th entries as one coalesced access.  The smoothers use class-ordered
// lists: the rows of each colour class (ascending, padded to a multiple of 32
// with -1), off-diagonal entries only, with the diagonal, its reciprocal and
// its reciprocal square root stored per position; a colour pass is one launch
// over its class's positions (Section 3.1's heat-bath update of Eq.
// equ_R_GS with the noise of Eq. equ_def_Q_GS).

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/selm_mac.h"
#include "../../include/selm_mg.h"
#include "selm_devmath.h"
#include "selm_internal.h"
#include "selm_launch.h"
#include "selm_mac.h"
#include "selm_pdl.h"
#include "selm_prof.h"

namespace selm {
namespace mac {
namespace {

constexpr int kThreads = 256;
constexpr int kRedBlocks = 304;        // 2 x 152 SMs: grid of the reductions

struct SellDev {
  int npos = 0;                        // list positions (multiple of 32)
  const int* row = nullptr;            // position -> row, -1 = padding
  const long long* soff = nullptr;
  const int* swid = nullptr;
  const int* col = nullptr;
  const double* v64 = nullptr;
  const float* v32 = nullptr;
  const double* dg64 = nullptr;        // class-ordered lists: diagonal,
  const float* dg32 = nullptr;
  const double* rd64 = nullptr;        // its reciprocal,
  const float* rd32 = nullptr;
  const double* rs64 = nullptr;        // and reciprocal square root
  const float* rs32 = nullptr;
};

template <typename T>
__device__ __forceinline__ const T* vals(const SellDev& S);
template <>
__device__ __forceinline__ const double* vals<double>(const SellDev& S) { return S.v64; }
template <>
__device__ __forceinline__ const float* vals<float>(const SellDev& S) { return S.v32; }
template <typename T>
__device__ __forceinline__ T dg_at(const SellDev& S, int p);
template <>
__device__ __forceinline__ double dg_at<double>(const SellDev& S, int p) { return S.dg64[p]; }
template <>
__device__ __forceinline__ float dg_at<float>(const SellDev& S, int p) { return S.dg32[p]; }
template <typename T>
__device__ __forceinline__ T rd_at(const SellDev& S, int p);
template <>
__device__ __forceinline__ double rd_at<double>(const SellDev& S, int p) { return S.rd64[p]; }
template <>
__device__ __forceinline__ float rd_at<float>(const SellDev& S, int p) { return S.rd32[p]; }
template <typename T>
__device__ __forceinline__ T rs_at(const SellDev& S, int p);
template <>
__device__ __forceinline__ double rs_at<double>(const SellDev& S, int p) { return S.rs64[p]; }
template <>
__device__ __forceinline__ float rs_at<float>(const SellDev& S, int p) { return S.rs32[p]; }

// sum_e val * x[col] over the entries of list position p (column order).
template <typename T, typename X>
__device__ __forceinline__ T row_dot(const SellDev& S, int p, const X* __restrict__ x) {
  const int s = p >> 5;
  const long long o = S.soff[s] + (p & 31);
  const int w = S.swid[s];
  const T* __restrict__ v = vals<T>(S);
  T acc = T(0);
  for (int e = 0; e < w; ++e) acc += v[o + 32ll * e] * (T)x[S.col[o + 32ll * e]];
  return acc;
}

__device__ __forceinline__ double warp_sum(double a) {
  for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  return a;
}

// Sum over the block (result valid in thread 0); fixed order.
__device__ double block_sum(double a) {
  __shared__ double sh[kThreads / 32];
  a = warp_sum(a);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  __syncthreads();
  return s;
}

// ---- kernels ----------------------------------------------------------------

// mode 0: y = S x;  1: y += S x;  2: y = b - S x.  Grid-stride over positions.
template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) k_sell_mv(SellDev S, const T* __restrict__ x, T* __restrict__ y,
                                                     const T* __restrict__ b) {
  pdl_enter();
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < S.npos; p += gridDim.x * blockDim.x) {
    const int r = S.row[p];
    if (r < 0) continue;
    const T a = row_dot<T>(S, p, x);
    if (MODE == 0) y[r] = a;
    else if (MODE == 1) y[r] += a;
    else y[r] = b[r] - a;
  }
}

// FP64 outer residual r = b - A z of the composite rows (Algorithm 1 step 1),
// stored in the inner precision, with per-block partial sums of ||r||^2.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_outer_resid(SellDev S, const double* __restrict__ z,
                                                         const double* __restrict__ b, T* __restrict__ r,
                                                         double* __restrict__ part) {
  double acc = 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < S.npos; p += gridDim.x * blockDim.x) {
    const int row = S.row[p];
    if (row < 0) continue;
    const double v = b[row] - row_dot<double>(S, p, z);
    r[row] = (T)v;
    acc += v * v;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// part[0..nb) -> out[0] (one block, fixed order).
__global__ void __launch_bounds__(kThreads) k_reduce(const double* __restrict__ part, int nb, double* __restrict__ out) {
  double a = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) a += part[i];
  a = block_sum(a);
  if (threadIdx.x == 0) *out = a;
}

// Per-block partial sums of x . y.
__global__ void __launch_bounds__(kThreads) k_dot_part(long long n, const double* __restrict__ x,
                                                      const double* __restrict__ y, double* __restrict__ part) {
  double a = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    a += x[i] * y[i];
  a = block_sum(a);
  if (threadIdx.x == 0) part[blockIdx.x] = a;
}

// Heat-bath update of one colour class (Eq. equ_R_GS with the noise term of
// Eq. equ_def_Q_GS): v_i = (b_i - sum_{j != i} a_ij v_j) / a_ii
//                          + sigma n_i / sqrt(a_ii).
// NK = 0: no noise; 1: normal of the site's rank in the class; 2: normal of
// the site's row index (slab faces).  kRowLanes lanes share a row: each sums
// every kRowLanes-th stored entry, a shuffle combines them, and the first
// lane updates the site, so a class of a few thousand rows still puts
// several warps on every SM.
constexpr int kRowLanes = 4;

// Programmatic dependent launch: the class passes of a sweep are launched
// with programmatic stream serialisation, and each block lets the next pass
// launch as soon as it starts.  Everything a pass needs that no earlier
// pass writes -- the matrix entries of its rows (the first kPrefetch per
// lane), its row numbers and scales, its normals (the counter word is
// written only by launches that completed before the sweep began) -- is
// loaded and computed before griddepcontrol.wait, which returns once the
// previous pass has completed and its writes are visible; v and b are read
// only after it.  The updates and their order are those of plain launches.
constexpr int kPrefetch = 8;

template <typename T, int NK, int LANES>
__global__ void __launch_bounds__(kThreads) k_colour(SellDev S, int pos0, int cnt, T* __restrict__ v,
                                                    const T* __restrict__ b, T sigma, Key key, uint32_t c1,
                                                    const unsigned long long* __restrict__ cyc) {
  pdl_launch_dependents();
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int t = g / LANES, sub = g % LANES;
  const bool valid = t < cnt;        // every lane stays for the shuffles
  const int p = pos0 + (valid ? t : 0);
  const T* __restrict__ vv = vals<T>(S);
  long long o = 0;
  int w = 0;
  int cidx[kPrefetch];
  T cval[kPrefetch];
  if (valid) {
    const int s = p >> 5;
    o = S.soff[s] + (p & 31);
    w = S.swid[s];
#pragma unroll
    for (int q = 0; q < kPrefetch; ++q) {
      const int e = sub + q * LANES;
      cidx[q] = e < w ? S.col[o + 32ll * e] : 0;
      cval[q] = e < w ? vv[o + 32ll * e] : T(0);
    }
  }
  int row = 0;
  T rd = T(0), ns = T(0), rsv = T(0);
  if (valid && sub == 0) {
    row = S.row[p];
    rd = rd_at<T>(S, p);
    if (NK != 0) {
      const unsigned long long c = *cyc;
      const uint32_t id = NK == 1 ? (uint32_t)t : (uint32_t)row;
      const uint4 wv = philox4x32_10(make_uint4(id >> 2, c1, (uint32_t)c, (uint32_t)(c >> 32)), key.k0, key.k1);
      T gn;
      normal_of(wv, (int)(id & 3), &gn);
      ns = sigma * gn;
      rsv = rs_at<T>(S, p);
    }
  }
  pdl_wait();
  T off = T(0);
  if (valid) {
#pragma unroll
    for (int q = 0; q < kPrefetch; ++q)
      if (sub + q * LANES < w) off += cval[q] * v[cidx[q]];
    for (int e = sub + kPrefetch * LANES; e < w; e += LANES) off += vv[o + 32ll * e] * v[S.col[o + 32ll * e]];
  }
#pragma unroll
  for (int m = 1; m < LANES; m <<= 1) off += __shfl_xor_sync(0xffffffffu, off, m);
  if (!valid || sub != 0) return;
  T nv = (b[row] - off) * rd;
  if (NK != 0) nv += ns * rsv;
  v[row] = nv;
}

// Launch of one class pass with programmatic stream serialisation.  Classes
// of at least kWideClass rows take one lane per row: a warp then reads each
// stored entry of its 32 rows as one coalesced access, and a class that large
// fills the GPU anyway; smaller classes keep kRowLanes lanes per row.
constexpr long long kWideClass = 32768;

template <typename T, int NK>
cudaError_t launch_colour(const SellDev& S, int pos0, int cnt, T* v, const T* b, T sigma, Key key, uint32_t c1,
                          const unsigned long long* cyc, cudaStream_t st) {
  if (cnt >= kWideClass) {
    const unsigned grid = (unsigned)(((long long)cnt + kThreads - 1) / kThreads);
    return launch_pdl(k_colour<T, NK, 1>, grid, kThreads, st, S, pos0, cnt, v, b, sigma, key, c1, cyc);
  }
  const unsigned grid = (unsigned)std::max<long long>(1, ((long long)cnt * kRowLanes + kThreads - 1) / kThreads);
  return launch_pdl(k_colour<T, NK, kRowLanes>, grid, kThreads, st, S, pos0, cnt, v, b, sigma, key, c1, cyc);
}

// ---- all colour passes of a small level's sweeps in one thread block --------
// On levels of a few thousand rows a launch per class is almost all launch
// latency.  One block of kBlockSweep threads runs `nsweeps` sweeps of every
// class with a block barrier between classes: the same updates in the same
// order as the per-class launches.  The level's v and b live in shared
// memory for the whole launch (v is written back at the end), and each
// thread loads the static part of its row lane for the next class -- matrix
// entries, row number, scales and normal -- before the barrier that ends the
// current class, so a class pass costs the barrier, the shared-memory
// gathers and the row's arithmetic.
constexpr int kBlockSweep = 1024;
constexpr long long kBlockSweepRows = 4096;   // levels up to this many rows sweep in one block

template <typename T>
struct BlockPrefetch {
  static constexpr int value = sizeof(T) == 4 ? 4 : 2;
};

// Static part of one row lane of a class pass.
template <typename T>
struct RowLane {
  bool valid;
  int sub, row, w;
  long long o;
  int cidx[BlockPrefetch<T>::value];
  T cval[BlockPrefetch<T>::value];
  T rd, ns, rsv;
};

template <typename T, int NK>
__device__ __forceinline__ void row_lane_load(const SellDev& S, int g, int pos0, int cnt, uint32_t c1, T sigma,
                                              Key key, unsigned long long c64, RowLane<T>& k) {
  constexpr int P = BlockPrefetch<T>::value;
  const int t = g / kRowLanes;
  k.sub = g % kRowLanes;
  k.valid = t < cnt;
  k.w = 0;
  k.o = 0;
  k.row = 0;
  k.rd = k.ns = k.rsv = T(0);
  const int p = pos0 + (k.valid ? t : 0);
  if (k.valid) {
    const int s = p >> 5;
    k.o = S.soff[s] + (p & 31);
    k.w = S.swid[s];
    const T* __restrict__ vv = vals<T>(S);
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const int e = k.sub + q * kRowLanes;
      k.cidx[q] = e < k.w ? S.col[k.o + 32ll * e] : 0;
      k.cval[q] = e < k.w ? vv[k.o + 32ll * e] : T(0);
    }
    if (k.sub == 0) {
      k.row = S.row[p];
      k.rd = rd_at<T>(S, p);
      if (NK != 0) {
        const uint4 wv = philox4x32_10(make_uint4((uint32_t)t >> 2, c1, (uint32_t)c64, (uint32_t)(c64 >> 32)),
                                       key.k0, key.k1);
        T gn;
        normal_of(wv, t & 3, &gn);
        k.ns = sigma * gn;
        k.rsv = rs_at<T>(S, p);
      }
    }
  }
}

// The update of a loaded row lane from the shared v and b (the whole warp
// calls it: every lane takes the shuffles).
template <typename T, int NK>
__device__ __forceinline__ void row_lane_apply(const SellDev& S, const RowLane<T>& k, T* vs, const T* bs) {
  constexpr int P = BlockPrefetch<T>::value;
  T off = T(0);
  if (k.valid) {
#pragma unroll
    for (int q = 0; q < P; ++q)
      if (k.sub + q * kRowLanes < k.w) off += k.cval[q] * vs[k.cidx[q]];
    const T* __restrict__ vv = vals<T>(S);
    for (int e = k.sub + P * kRowLanes; e < k.w; e += kRowLanes) off += vv[k.o + 32ll * e] * vs[S.col[k.o + 32ll * e]];
  }
#pragma unroll
  for (int m = 1; m < kRowLanes; m <<= 1) off += __shfl_xor_sync(0xffffffffu, off, m);
  if (k.valid && k.sub == 0) {
    T nv = (bs[k.row] - off) * k.rd;
    if (NK != 0) nv += k.ns * k.rsv;
    vs[k.row] = nv;
  }
}

__host__ __device__ constexpr uint32_t block_ctr1(int level1, int c, int sweep) {
  return (uint32_t)level1 | ((uint32_t)(c & 15) << 8) | ((uint32_t)sweep << 12) | ((uint32_t)(c >> 4) << 24);
}

template <typename T>
size_t block_sweep_smem(long long N, int ncol) {
  return (size_t)(2 * N) * sizeof(T) + (size_t)(2 * ncol) * sizeof(int);
}

template <typename T, int NK>
__global__ void __launch_bounds__(kBlockSweep) k_colour_block(SellDev S, const int* __restrict__ cstart,
                                                             const int* __restrict__ csize, int ncol, int level1,
                                                             int sweep0, int nsweeps, int N, T* v,
                                                             const T* __restrict__ b, T sigma, Key key,
                                                             const unsigned long long* __restrict__ cyc) {
  extern __shared__ __align__(16) unsigned char block_smem[];
  T* vs = reinterpret_cast<T*>(block_smem);
  T* bs = vs + N;
  int* cs = reinterpret_cast<int*>(bs + N);
  int* cz = cs + ncol;
  const int tid = threadIdx.x;
  const int wbase = tid - (tid & 31);   // warp-uniform lane-task base
  for (int i = tid; i < N; i += kBlockSweep) {
    vs[i] = v[i];
    bs[i] = b[i];
  }
  for (int i = tid; i < ncol; i += kBlockSweep) {
    cs[i] = cstart[i];
    cz[i] = csize[i];
  }
  const unsigned long long c64 = NK ? *cyc : 0ull;
  __syncthreads();
  const int npass = nsweeps * ncol;
  RowLane<T> k;
  if (npass > 0) row_lane_load<T, NK>(S, wbase + (tid & 31), cs[0], cz[0], block_ctr1(level1, 0, sweep0), sigma, key,
                                      c64, k);
  for (int q = 0; q < npass; ++q) {
    const int sw = q / ncol, c = q - sw * ncol;
    const int pos0 = cs[c], cnt = cz[c];
    const uint32_t c1 = block_ctr1(level1, c, sweep0 + sw);
    if (wbase < cnt * kRowLanes) row_lane_apply<T, NK>(S, k, vs, bs);
    // classes of more than kBlockSweep / kRowLanes rows: the further lanes
    for (int base = wbase + kBlockSweep; base < cnt * kRowLanes; base += kBlockSweep) {
      RowLane<T> x;
      row_lane_load<T, NK>(S, base + (tid & 31), pos0, cnt, c1, sigma, key, c64, x);
      row_lane_apply<T, NK>(S, x, vs, bs);
    }
    if (q + 1 < npass) {   // the next class's static data, before the barrier
      const int sw2 = (q + 1) / ncol, c2 = (q + 1) - sw2 * ncol;
      row_lane_load<T, NK>(S, wbase + (tid & 31), cs[c2], cz[c2], block_ctr1(level1, c2, sweep0 + sw2), sigma, key,
                           c64, k);
    }
    __syncthreads();
  }
  for (int i = tid; i < N; i += kBlockSweep) v[i] = vs[i];
}

// Lets both noise variants of the block sweep take `bytes` of dynamic shared
// memory (above the 48 KB default).
template <typename T>
cudaError_t allow_block_smem(size_t bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_colour_block<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_colour_block<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return e;
}

// t = b - A v on every row of a class-ordered level (diagonal included);
// kRowLanes lanes per row as in k_colour.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_cls_resid(SellDev S, const T* __restrict__ v, const T* __restrict__ b,
                                                       T* __restrict__ t) {
  pdl_enter();
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int p = (int)(g / kRowLanes), sub = (int)(g % kRowLanes);
  const bool valid = p < S.npos && S.row[p] >= 0;
  T off = T(0);
  if (valid) {
    const int s = p >> 5;
    const long long o = S.soff[s] + (p & 31);
    const int w = S.swid[s];
    const T* __restrict__ vv = vals<T>(S);
    for (int e = sub; e < w; e += kRowLanes) off += vv[o + 32ll * e] * v[S.col[o + 32ll * e]];
  }
#pragma unroll
  for (int m = 1; m < kRowLanes; m <<= 1) off += __shfl_xor_sync(0xffffffffu, off, m);
  if (!valid || sub != 0) return;
  const int row = S.row[p];
  t[row] = b[row] - dg_at<T>(S, p) * v[row] - off;
}

// Exact draw on the coarsest level (FP64): with A = L L^T,
// v = L^-T (L^-1 b + sigma n), n ~ N(0, I): mean A^-1 b, covariance
// sigma^2 A^-1.  One block; y in shared memory.
// Coarsest level, the exact draw: v = L^-T (L^-1 b + sigma n) with A_c = L L^T
// in FP64, in two launches spread over the GPU.  Forward: one warp per row i
// of L^-1 b (lanes stride over j <= i, then a warp sum), the row's normal
// added by lane 0.  Backward: one warp per row i of L^-T, read from the
// transposed copy of L^-1 so that the lanes' loads are consecutive.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_coarsest_fwd(const double* __restrict__ Linv, int m,
                                                          const T* __restrict__ b, double* __restrict__ y,
                                                          double sigma, Key key, uint32_t c1,
                                                          const unsigned long long* __restrict__ cyc) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (i >= m) return;   // the whole warp
  double a = 0.0;
  for (int j = lane; j <= i; j += 32) a += Linv[(size_t)i * m + j] * (double)b[j];
  a = warp_sum(a);
  if (lane == 0) {
    if (sigma != 0.0) {
      const unsigned long long c = *cyc;
      const uint4 w = philox4x32_10(make_uint4((uint32_t)i >> 2, c1, (uint32_t)c, (uint32_t)(c >> 32)), key.k0,
                                    key.k1);
      double g;
      normal_of(w, i & 3, &g);
      a += sigma * g;
    }
    y[i] = a;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_coarsest_bwd(const double* __restrict__ LinvT, int m,
                                                          const double* __restrict__ y, T* __restrict__ v) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (i >= m) return;   // the whole warp
  double a = 0.0;
  for (int j = i + lane; j < m; j += 32) a += LinvT[(size_t)i * m + j] * y[j];
  a = warp_sum(a);
  if (lane == 0) v[i] = (T)a;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_add_to(long long n, double* __restrict__ z, const T* __restrict__ q) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] += (double)q[i];
}

// y = x * s (elementwise vector s), or x / s with DIV.
template <bool DIV>
__global__ void __launch_bounds__(kThreads) k_scale(long long n, const double* __restrict__ x,
                                                   const double* __restrict__ s, double* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = DIV ? x[i] / s[i] : x[i] * s[i];
}

// Conjugate gradients (Jacobi preconditioned) on diag(vol) L phi = rhs, the
// scalars kept on the device: sc[0], sc[1] = r.z of even / odd iterations,
// sc[2] = the starting r.z, sc[3] = r.r.  An iteration is three launches
// (programmatic dependent launches): q = S p with the partial sums of p.q;
// the update of x, r, z with the partial sums of r.z and r.r; the new
// direction.  Each block of the second and third launch sums the previous
// launch's partials itself, in the order of k_reduce, so every block holds
// the same alpha and beta.
__device__ double block_total(const double* __restrict__ part, int nb) {
  __shared__ double tot;
  double a = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) a += part[i];
  a = block_sum(a);
  if (threadIdx.x == 0) tot = a;
  __syncthreads();
  return tot;
}

__global__ void __launch_bounds__(kThreads) k_cg_mv(SellDev S, const double* __restrict__ p, double* __restrict__ q,
                                                   double* __restrict__ part) {
  pdl_enter();
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < S.npos; i += gridDim.x * blockDim.x) {
    const int r = S.row[i];
    if (r < 0) continue;
    const double a = row_dot<double>(S, i, p);
    q[r] = a;
    acc += a * p[r];
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kThreads) k_cg_update(long long n, int nb, const double* __restrict__ part_pq,
                                                       const double* __restrict__ sc, int old,
                                                       double* __restrict__ x, double* __restrict__ r,
                                                       const double* __restrict__ p, const double* __restrict__ q,
                                                       const double* __restrict__ minv, double* __restrict__ z,
                                                       double* __restrict__ part) {
  pdl_enter();
  const double pq = block_total(part_pq, nb);
  const double alpha = pq != 0.0 ? sc[old] / pq : 0.0;
  double rz = 0.0, rr = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    const double zi = ri * minv[i];
    z[i] = zi;
    rz += ri * zi;
    rr += ri * ri;
  }
  rz = block_sum(rz);
  rr = block_sum(rr);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = rz;
    part[kRedBlocks + blockIdx.x] = rr;
  }
}

__global__ void __launch_bounds__(kThreads) k_cg_reduce2(const double* __restrict__ part, int nb,
                                                        double* __restrict__ sc) {
  double a = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    a += part[i];
    c += part[kRedBlocks + i];
  }
  a = block_sum(a);
  c = block_sum(c);
  if (threadIdx.x == 0) {
    sc[2] = a;
    sc[3] = c;
  }
}

__global__ void __launch_bounds__(kThreads) k_cg_dir(long long n, int nb, const double* __restrict__ part,
                                                    double* __restrict__ sc, int old, const double* __restrict__ z,
                                                    double* __restrict__ p) {
  pdl_enter();
  const double rz = block_total(part, nb);
  const double rr = block_total(part + kRedBlocks, nb);
  const double rz_old = sc[old];
  const double beta = rz_old != 0.0 ? rz / rz_old : 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    sc[old ^ 1] = rz;   // the next iteration's r.z (the other slot: blocks still read sc[old])
    sc[3] = rr;
  }
}

__global__ void k_cg_shift(double* sc) { sc[0] = sc[2]; }

// p = z, sc[0] = r.z (start of the iteration).
__global__ void __launch_bounds__(kThreads) k_cg_start(long long n, const double* __restrict__ r,
                                                      const double* __restrict__ minv, double* __restrict__ z,
                                                      double* __restrict__ p, double* __restrict__ part) {
  double rz = 0.0, rr = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double zi = r[i] * minv[i];
    z[i] = zi;
    p[i] = zi;
    rz += r[i] * zi;
    rr += r[i] * r[i];
  }
  rz = block_sum(rz);
  rr = block_sum(rr);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = rz;
    part[kRedBlocks + blockIdx.x] = rr;
  }
}

// phi -= (vol . phi) / sum(vol): the representative of zero volume mean.
__global__ void __launch_bounds__(kThreads) k_sub_scalar(long long n, double* __restrict__ x, const double* __restrict__ s,
                                                        double inv_total) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] -= s[0] * inv_total;
}

unsigned blocks_for(long long n) { return (unsigned)std::max<long long>(1, (n + kThreads - 1) / kThreads); }
unsigned red_blocks(long long n) { return (unsigned)std::min<long long>(kRedBlocks, std::max<long long>(1, (n + kThreads - 1) / kThreads)); }

// ---- host: sliced ELL from CSR -------------------------------------------------
struct SellHost {
  std::vector<int> row, swid, col;
  std::vector<long long> soff;
  std::vector<double> v, dg, rd, rs;
  int npos = 0;
};

// `order`: list of rows (-1 = padding), length a multiple of 32.  offdiag:
// keep only off-diagonal entries and record the diagonal per position.
SellHost make_sell(const Csr& A, const std::vector<int>& order, bool offdiag) {
  SellHost S;
  S.npos = (int)order.size();
  S.row = order;
  const int nsl = S.npos / 32;
  S.soff.resize(nsl);
  S.swid.resize(nsl);
  long long off = 0;
  for (int s = 0; s < nsl; ++s) {
    int w = 0;
    for (int l = 0; l < 32; ++l) {
      const int r = order[s * 32 + l];
      if (r < 0) continue;
      int len = 0;
      for (long long q = A.ptr[r]; q < A.ptr[r + 1]; ++q)
        if (!offdiag || A.col[q] != r) ++len;
      w = std::max(w, len);
    }
    S.soff[s] = off;
    S.swid[s] = w;
    off += 32ll * w;
  }
  S.col.assign(off, 0);
  S.v.assign(off, 0.0);
  if (offdiag) {
    S.dg.assign(S.npos, 1.0);
    S.rd.assign(S.npos, 1.0);
    S.rs.assign(S.npos, 1.0);
  }
  for (int p = 0; p < S.npos; ++p) {
    const int r = order[p];
    if (r < 0) continue;
    const int s = p >> 5, l = p & 31;
    int e = 0;
    for (long long q = A.ptr[r]; q < A.ptr[r + 1]; ++q) {
      if (offdiag && A.col[q] == r) {
        S.dg[p] = A.val[q];
        S.rd[p] = 1.0 / A.val[q];
        S.rs[p] = 1.0 / std::sqrt(A.val[q]);
        continue;
      }
      S.col[S.soff[s] + 32ll * e + l] = A.col[q];
      S.v[S.soff[s] + 32ll * e + l] = A.val[q];
      ++e;
    }
  }
  return S;
}

std::vector<int> natural_order(int nr) {
  std::vector<int> o((nr + 31) / 32 * 32, -1);
  for (int r = 0; r < nr; ++r) o[r] = r;
  return o;
}

// Class-ordered list: each class's rows, padded to a multiple of 32.
std::vector<int> class_order(const std::vector<std::vector<int>>& classes, std::vector<int>* start,
                             std::vector<int>* size) {
  std::vector<int> o;
  for (const auto& c : classes) {
    start->push_back((int)o.size());
    size->push_back((int)c.size());
    o.insert(o.end(), c.begin(), c.end());
    while (o.size() % 32) o.push_back(-1);
  }
  if (o.empty()) o.assign(32, -1);
  return o;
}

}  // namespace
}  // namespace mac
}  // namespace selm

using namespace selm;
using namespace selm::mac;

struct selm_mac {
  selm_mac_desc d{};
  int esize = 8;
  int levels = 0;
  long long n_faces = 0, n_cells = 0;
  std::string err;
  std::vector<void*> allocs;
  Key key{};
  double total_vol = 0.0;
  // operators
  SellDev A64;                       // composite A, natural rows, diagonal included (FP64)
  SellDev Apatch;                    // slab faces, class-ordered
  std::vector<int> pstart, psize;
  SellDev Pm, Pt;                    // P (composite <- base) and P^T
  struct Level {
    long long N = 0;
    SellDev cls;                     // class-ordered operator (levels above the coarsest)
    std::vector<int> cstart, csize;
    SellDev Pl, Plt;                 // transfers to / from the next coarser level
    void *v = nullptr, *b = nullptr, *t = nullptr;
    // small levels: every class of a sweep set in one thread block
    const int* d_cstart = nullptr;
    const int* d_csize = nullptr;
    bool block_sweeps = false;
  };
  std::vector<Level> lev;
  const double* Linv = nullptr;
  const double* LinvT = nullptr;     // its transpose (rows of L^-T)
  double* ycoarse = nullptr;         // L^-1 b (+ noise) of the coarsest draw
  int mc = 0;
  SellDev D, G, S;                   // divergence, gradient, diag(vol) D G (FP64)
  const double* minv = nullptr;      // 1 / diag(S)
  const double* vol = nullptr;
  const double* weight = nullptr;
  SellDev Et;                        // E^T (composite <- fine lattice), E (fine lattice <- composite)
  SellDev E;
  LevelDev fine{};                   // the uniform fine lattice of the particle kernel
  long long fine_size = 0;
  // buffers
  void *r = nullptr, *q = nullptr;   // composite residual / correction (inner precision)
  double* xi = nullptr;
  unsigned long long* cyc = nullptr; // counter of the chain's next cycle (device)
  unsigned long long* cyc_user = nullptr;
  uint64_t chain_cycle = 0;
  double* part = nullptr;            // reduction partials (2 x kRedBlocks)
  double* part2 = nullptr;           // second set for the CG update's partials
  double* part_rows = nullptr;       // one partial per block of the outer residual's rows
  double* sc = nullptr;              // device scalars
  double* host_sc = nullptr;         // pinned host copy
  double *cg_x = nullptr, *cg_r = nullptr, *cg_z = nullptr, *cg_p = nullptr, *cg_q = nullptr;
  double *fw = nullptr, *fw2 = nullptr, *fine_buf = nullptr, *pv = nullptr;
  int max_np = 0;
  double* pX = nullptr;
  long long total_cycles = 0;
  // the V-cycle part of a FAC cycle replayed from CUDA graphs (noise / plain)
  cudaStream_t cap = nullptr;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  long long glaunch[2] = {0, 0};
  cudaGraphExec_t cg_exec = nullptr;  // a block of conjugate-gradient iterations
  long long cg_launch = 0;
  int gruns[2] = {0, 0};
  bool graphs = true;
};

namespace {

#define MCK(call)                                                          \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) {                                               \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_);         \
      return SELM_ECUDA;                                                   \
    }                                                                      \
  } while (0)

cudaStream_t ST(void* s) { return (cudaStream_t)s; }

template <typename V>
selm_status upload(selm_mac* h, const std::vector<V>& x, const V** out, cudaStream_t st) {
  *out = nullptr;
  if (x.empty()) return SELM_OK;
  void* p = nullptr;
  if (cudaMalloc(&p, x.size() * sizeof(V)) != cudaSuccess) {
    cudaGetLastError();
    h->err = "device allocation failed";
    return SELM_ENOMEM;
  }
  h->allocs.push_back(p);
  MCK(cudaMemcpyAsync(p, x.data(), x.size() * sizeof(V), cudaMemcpyHostToDevice, st));
  *out = (const V*)p;
  return SELM_OK;
}

selm_status alloc(selm_mac* h, size_t bytes, void** out, cudaStream_t st) {
  *out = nullptr;
  if (cudaMalloc(out, std::max<size_t>(bytes, 256)) != cudaSuccess) {
    cudaGetLastError();
    h->err = "device allocation failed";
    return SELM_ENOMEM;
  }
  h->allocs.push_back(*out);
  MCK(cudaMemsetAsync(*out, 0, std::max<size_t>(bytes, 256), st));
  return SELM_OK;
}

#define MRET(x)                        \
  do {                                 \
    selm_status r_ = (x);              \
    if (r_ != SELM_OK) return r_;      \
  } while (0)

// Upload a sliced ELL (FP64 values, plus FP32 copies when f32).
selm_status upload_sell(selm_mac* h, const SellHost& S, bool f32, SellDev* out, cudaStream_t st) {
  out->npos = S.npos;
  MRET(upload(h, S.row, &out->row, st));
  MRET(upload(h, S.soff, &out->soff, st));
  MRET(upload(h, S.swid, &out->swid, st));
  MRET(upload(h, S.col, &out->col, st));
  MRET(upload(h, S.v, &out->v64, st));
  if (!S.dg.empty()) {
    MRET(upload(h, S.dg, &out->dg64, st));
    MRET(upload(h, S.rd, &out->rd64, st));
    MRET(upload(h, S.rs, &out->rs64, st));
  }
  if (f32) {
    auto cvt = [](const std::vector<double>& a) {
      std::vector<float> o(a.size());
      for (size_t i = 0; i < a.size(); ++i) o[i] = (float)a[i];
      return o;
    };
    MRET(upload(h, cvt(S.v), &out->v32, st));
    if (!S.dg.empty()) {
      MRET(upload(h, cvt(S.dg), &out->dg32, st));
      MRET(upload(h, cvt(S.rd), &out->rd32, st));
      MRET(upload(h, cvt(S.rs), &out->rs32, st));
    }
  }
  return SELM_OK;
}

uint32_t ctr1(int level, int comp, int colour, int sweep, int kind) {
  return (uint32_t)level | ((uint32_t)comp << 4) | ((uint32_t)(colour & 15) << 8) | ((uint32_t)sweep << 12) |
         ((uint32_t)kind << 20) | ((uint32_t)(colour >> 4) << 24);
}

// ---- the V-cycle on the base hierarchy (Algorithm 3) -------------------------
template <typename T>
selm_status sweep(selm_mac* h, int l, int s, double sigma, const unsigned long long* cyc, cudaStream_t st) {
  selm_mac::Level& L = h->lev[l];
  for (size_t c = 0; c < L.cstart.size(); ++c) {
    const int cnt = L.csize[c];
    prof::Scope ps(SELM_K_COARSE_SWEEP, st);
    if (sigma != 0.0)
      MCK((launch_colour<T, 1>(L.cls, L.cstart[c], cnt, (T*)L.v, (const T*)L.b, (T)sigma, h->key,
                              ctr1(l + 1, 0, (int)c, s, 0), cyc, st)));
    else
      MCK((launch_colour<T, 0>(L.cls, L.cstart[c], cnt, (T*)L.v, (const T*)L.b, (T)0, h->key, 0, cyc, st)));
  }
  return SELM_OK;
}

// `n` sweeps of level l from sweep index s0: one block launch on the small
// levels, one launch per class on the others.
template <typename T>
selm_status sweeps(selm_mac* h, int l, int s0, int n, double sigma, const unsigned long long* cyc, cudaStream_t st) {
  selm_mac::Level& L = h->lev[l];
  if (n <= 0) return SELM_OK;
  if (!L.block_sweeps) {
    for (int s = 0; s < n; ++s) MRET(sweep<T>(h, l, s0 + s, sigma, cyc, st));
    return SELM_OK;
  }
  prof::Scope ps(SELM_K_COARSE_SWEEP, st);
  const int ncol = (int)L.cstart.size();
  const size_t smem = block_sweep_smem<T>(L.N, ncol);
  if (sigma != 0.0)
    k_colour_block<T, 1><<<1, kBlockSweep, smem, st>>>(L.cls, L.d_cstart, L.d_csize, ncol, l + 1, s0, n, (int)L.N,
                                                       (T*)L.v, (const T*)L.b, (T)sigma, h->key, cyc);
  else
    k_colour_block<T, 0><<<1, kBlockSweep, smem, st>>>(L.cls, L.d_cstart, L.d_csize, ncol, l + 1, s0, n, (int)L.N,
                                                       (T*)L.v, (const T*)L.b, (T)0, h->key, cyc);
  MCK(cudaGetLastError());
  return SELM_OK;
}

template <typename T>
selm_status vcycle(selm_mac* h, int l, double sigma, const unsigned long long* cyc, cudaStream_t st) {
  selm_mac::Level& L = h->lev[l];
  if (l == h->levels - 1) {
    prof::Scope ps(SELM_K_COARSEST, st);
    const unsigned grid = (unsigned)(((long long)h->mc * 32 + kThreads - 1) / kThreads);
    MCK((launch_pdl(k_coarsest_fwd<T>, grid, kThreads, st, h->Linv, h->mc, (const T*)L.b, h->ycoarse, sigma, h->key,
                    ctr1(l + 1, 0, 0, 0, 1), cyc)));
    MCK((launch_pdl(k_coarsest_bwd<T>, grid, kThreads, st, h->LinvT, h->mc, (const double*)h->ycoarse, (T*)L.v)));
    return SELM_OK;
  }
  const int mu1 = h->d.nu_pre, mu2 = h->d.nu_post;
  MRET(sweeps<T>(h, l, 0, mu1, sigma, cyc, st));
  selm_mac::Level& C = h->lev[l + 1];
  {
    prof::Scope ps(SELM_K_RESIDUAL, st);
    MCK((launch_pdl(k_cls_resid<T>, blocks_for((long long)L.cls.npos * kRowLanes), kThreads, st, L.cls,
                    (const T*)L.v, (const T*)L.b, (T*)L.t)));
  }
  {
    prof::Scope ps(SELM_K_RESTRICT, st);
    MCK((launch_pdl(k_sell_mv<T, 0>, blocks_for(L.Plt.npos), kThreads, st, L.Plt, (const T*)L.t, (T*)C.b, nullptr)));
  }
  MCK(cudaMemsetAsync(C.v, 0, (size_t)C.N * sizeof(T), st));
  MRET(vcycle<T>(h, l + 1, sigma, cyc, st));
  {
    prof::Scope ps(SELM_K_PROLONG, st);
    MCK((launch_pdl(k_sell_mv<T, 1>, blocks_for(L.Pl.npos), kThreads, st, L.Pl, (const T*)C.v, (T*)L.v, nullptr)));
  }
  MRET(sweeps<T>(h, l, mu1, mu2, sigma, cyc, st));
  return SELM_OK;
}

// From the residual r (inner precision): q = P V-cycle(P^T r), then the slab
// sweeps of A q = r (Algorithm 2 with the patch sweeps of Algorithm 1).
template <typename T>
selm_status correction(selm_mac* h, double sigma, const unsigned long long* cyc, cudaStream_t st) {
  selm_mac::Level& B = h->lev[0];
  {
    prof::Scope ps(SELM_K_RESTRICT, st);
    MCK((launch_pdl(k_sell_mv<T, 0>, blocks_for(h->Pt.npos), kThreads, st, h->Pt, (const T*)h->r, (T*)B.b, nullptr)));
  }
  MCK(cudaMemsetAsync(B.v, 0, (size_t)B.N * sizeof(T), st));
  MRET(vcycle<T>(h, 0, sigma, cyc, st));
  {
    prof::Scope ps(SELM_K_PROLONG, st);
    MCK((launch_pdl(k_sell_mv<T, 0>, blocks_for(h->Pm.npos), kThreads, st, h->Pm, (const T*)B.v, (T*)h->q, nullptr)));
  }
  for (int s = 0; s < h->d.nu_patch; ++s)
    for (size_t c = 0; c < h->pstart.size(); ++c) {
      const int cnt = h->psize[c];
      prof::Scope ps(SELM_K_FINE_SWEEP, st);
      if (sigma != 0.0)
        MCK((launch_colour<T, 2>(h->Apatch, h->pstart[c], cnt, (T*)h->q, (const T*)h->r, (T)sigma, h->key,
                                ctr1(0, 0, (int)c, s, 2), cyc, st)));
      else
        MCK((launch_colour<T, 0>(h->Apatch, h->pstart[c], cnt, (T*)h->q, (const T*)h->r, (T)0, h->key, 0, cyc, st)));
    }
  return SELM_OK;
}

selm_status correction_any(selm_mac* h, double sigma, const unsigned long long* cyc, cudaStream_t st) {
  return h->esize == 4 ? correction<float>(h, sigma, cyc, st) : correction<double>(h, sigma, cyc, st);
}

// The correction as a replay of a captured graph (sigma 0 or 1 with the
// handle's counter words); other sigmas and counters run directly.
selm_status correction_graph(selm_mac* h, double sigma, const unsigned long long* cyc, cudaStream_t st) {
  const int g = sigma != 0.0 ? 1 : 0;
  if (!h->graphs || prof::g_on || (sigma != 0.0 && sigma != 1.0) || (g == 1 && cyc != h->cyc))
    return correction_any(h, sigma, cyc, st);
  if (!h->gexec[g]) {
    if (h->gruns[g]++ == 0) return correction_any(h, sigma, cyc, st);   // lazy set-up outside the capture
    const long long l0 = prof::g_launches.load();
    if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      h->graphs = false;
      return correction_any(h, sigma, cyc, st);
    }
    const selm_status r = correction_any(h, sigma, cyc, h->cap);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
    h->glaunch[g] = prof::g_launches.load() - l0;
    prof::g_launches.fetch_sub(h->glaunch[g]);
    if (r != SELM_OK || e != cudaSuccess || !graph || cudaGraphInstantiate(&h->gexec[g], graph, 0) != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      h->gexec[g] = nullptr;
      h->graphs = false;
      return correction_any(h, sigma, cyc, st);
    }
    cudaGraphDestroy(graph);
  }
  MCK(cudaGraphLaunch(h->gexec[g], st));
  prof::g_launches.fetch_add(h->glaunch[g]);
  return SELM_OK;
}

// r = b - A z (FP64, stored in the inner precision); ||r||^2 into sc[slot].
selm_status outer_residual(selm_mac* h, const double* z, const double* b, int slot, cudaStream_t st) {
  // one list position per thread (each row's FP64 dot in a latency chain of
  // its own), the block partials summed by one block in a fixed order
  const unsigned nb = blocks_for(h->A64.npos);
  {
    prof::Scope ps(SELM_K_OUTER_RESIDUAL, st);
    if (h->esize == 4)
      k_outer_resid<float><<<nb, kThreads, 0, st>>>(h->A64, z, b, (float*)h->r, h->part_rows);
    else
      k_outer_resid<double><<<nb, kThreads, 0, st>>>(h->A64, z, b, (double*)h->r, h->part_rows);
    MCK(cudaGetLastError());
  }
  prof::Scope ps(SELM_K_OTHER, st);
  k_reduce<<<1, kThreads, 0, st>>>(h->part_rows, (int)nb, h->sc + slot);
  MCK(cudaGetLastError());
  return SELM_OK;
}

selm_status update(selm_mac* h, double* z, cudaStream_t st) {
  prof::Scope ps(SELM_K_OUTER_UPDATE, st);
  if (h->esize == 4)
    k_add_to<float><<<blocks_for(h->n_faces), kThreads, 0, st>>>(h->n_faces, z, (const float*)h->q);
  else
    k_add_to<double><<<blocks_for(h->n_faces), kThreads, 0, st>>>(h->n_faces, z, (const double*)h->q);
  MCK(cudaGetLastError());
  return SELM_OK;
}

selm_status fac_cycle(selm_mac* h, double* z, const double* b, double sigma, const unsigned long long* cyc,
                      cudaStream_t st) {
  MRET(outer_residual(h, z, b, 4, st));
  MRET(correction_graph(h, sigma, cyc, st));
  MRET(update(h, z, st));
  h->total_cycles += 1;
  return SELM_OK;
}

selm_status norm2(selm_mac* h, long long n, const double* x, int slot, cudaStream_t st) {
  const unsigned nb = red_blocks(n);
  prof::Scope ps(SELM_K_OTHER, st);
  k_dot_part<<<nb, kThreads, 0, st>>>(n, x, x, h->part);
  k_reduce<<<1, kThreads, 0, st>>>(h->part, (int)nb, h->sc + slot);
  MCK(cudaGetLastError());
  return SELM_OK;
}

selm_status read_scalars(selm_mac* h, cudaStream_t st) {
  MCK(cudaMemcpyAsync(h->host_sc, h->sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
  MCK(cudaStreamSynchronize(st));
  return SELM_OK;
}

selm_status solve(selm_mac* h, double* z, const double* b, double tol, int max_cycles, int* cycles, double* rel,
                  cudaStream_t st) {
  MRET(norm2(h, h->n_faces, b, 5, st));
  MRET(outer_residual(h, z, b, 4, st));
  MRET(read_scalars(h, st));
  const double bn = std::sqrt(h->host_sc[5]);
  double rn = std::sqrt(h->host_sc[4]);
  int k = 0;
  const double target = tol * (bn > 0.0 ? bn : 1.0);
  while (rn > target && k < max_cycles) {
    MRET(correction_graph(h, 0.0, h->cyc, st));
    MRET(update(h, z, st));
    h->total_cycles += 1;
    ++k;
    MRET(outer_residual(h, z, b, 4, st));
    MRET(read_scalars(h, st));
    rn = std::sqrt(h->host_sc[4]);
  }
  if (cycles) *cycles = k;
  if (rel) *rel = bn > 0.0 ? rn / bn : rn;
  if (rn > target) {
    h->err = "FAC solve did not reach tol";
    return SELM_ENOCONV;
  }
  return SELM_OK;
}

// phi with L phi = rhs (cells), zero volume mean, by PCG on diag(vol) L.
selm_status pressure_solve(selm_mac* h, const double* rhs, int* iters, double* resid, cudaStream_t st) {
  const long long n = h->n_cells;
  const unsigned nb = red_blocks(n), eb = blocks_for(n);
  {
    prof::Scope ps(SELM_K_PROJECTION, st);
    k_scale<false><<<eb, kThreads, 0, st>>>(n, rhs, h->vol, h->cg_r);      // r = vol rhs (x = 0)
    MCK(cudaMemsetAsync(h->cg_x, 0, n * sizeof(double), st));
    k_cg_start<<<nb, kThreads, 0, st>>>(n, h->cg_r, h->minv, h->cg_z, h->cg_p, h->part);
    k_cg_reduce2<<<1, kThreads, 0, st>>>(h->part, (int)nb, h->sc);
    k_cg_shift<<<1, 1, 0, st>>>(h->sc);
    MCK(cudaGetLastError());
  }
  MCK(cudaMemcpyAsync(h->host_sc, h->sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
  MCK(cudaStreamSynchronize(st));
  const double bn = std::sqrt(h->host_sc[3]);
  const double tol = h->d.proj_tol;
  double rn = bn;
  int it = 0;
  const int max_it = 20000;
  constexpr int check = 16;
  // `check` iterations (three launches each) on the handle's fixed buffers;
  // iteration k reads its r.z from sc[k & 1] (check is even, so every block
  // of iterations starts from sc[0])
  static_assert(check % 2 == 0, "the r.z slots alternate");
  auto block = [&](cudaStream_t s2) -> cudaError_t {
    for (int k = 0; k < check; ++k) {
      prof::Scope ps(SELM_K_PROJECTION, s2);
      const int old = k & 1;
      cudaError_t e = launch_pdl(k_cg_mv, nb, kThreads, s2, h->S, (const double*)h->cg_p, h->cg_q, h->part);
      if (e == cudaSuccess)
        e = launch_pdl(k_cg_update, nb, kThreads, s2, n, (int)nb, (const double*)h->part, (const double*)h->sc, old,
                       h->cg_x, h->cg_r, (const double*)h->cg_p, (const double*)h->cg_q, h->minv, h->cg_z,
                       h->part2);
      if (e == cudaSuccess)
        e = launch_pdl(k_cg_dir, nb, kThreads, s2, n, (int)nb, (const double*)h->part2, h->sc, old,
                       (const double*)h->cg_z, h->cg_p);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  // replayed from a captured graph (captured once per handle) unless
  // profiling or capture is off
  if (!h->cg_exec && h->graphs && !prof::g_on) {
    const long long l0 = prof::g_launches.load();
    if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const cudaError_t e1 = block(h->cap);
      cudaGraph_t graph = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(h->cap, &graph);
      h->cg_launch = prof::g_launches.load() - l0;
      prof::g_launches.fetch_sub(h->cg_launch);
      if (e1 != cudaSuccess || e2 != cudaSuccess || !graph ||
          cudaGraphInstantiate(&h->cg_exec, graph, 0) != cudaSuccess)
        h->cg_exec = nullptr;
      if (graph) cudaGraphDestroy(graph);
    }
    cudaGetLastError();
  }
  while (bn > 0.0 && rn > tol * bn && it < max_it) {
    if (h->cg_exec && !prof::g_on) {
      MCK(cudaGraphLaunch(h->cg_exec, st));
      prof::g_launches.fetch_add(h->cg_launch);
    } else {
      MCK(block(st));
    }
    it += check;
    MCK(cudaMemcpyAsync(h->host_sc, h->sc, 8 * sizeof(double), cudaMemcpyDeviceToHost, st));
    MCK(cudaStreamSynchronize(st));
    rn = std::sqrt(h->host_sc[3]);
  }
  {
    prof::Scope ps(SELM_K_PROJECTION, st);
    k_dot_part<<<nb, kThreads, 0, st>>>(n, h->cg_x, h->vol, h->part);
    k_reduce<<<1, kThreads, 0, st>>>(h->part, (int)nb, h->sc + 6);
    k_sub_scalar<<<eb, kThreads, 0, st>>>(n, h->cg_x, h->sc + 6, 1.0 / h->total_vol);
    MCK(cudaGetLastError());
  }
  if (iters) *iters = it;
  if (resid) *resid = bn > 0.0 ? rn / bn : 0.0;
  if (bn > 0.0 && rn > tol * bn) {
    h->err = "pressure solve of the projection did not reach proj_tol";
    return SELM_ENOCONV;
  }
  return SELM_OK;
}

// out = P~ u (adjoint 0) or W P~ W^-1 u (adjoint 1); out may equal u.
selm_status project(selm_mac* h, const double* u, double* out, int adjoint, int* iters, double* resid,
                    cudaStream_t st) {
  const long long nf = h->n_faces;
  const double* src = u;
  if (adjoint) {
    prof::Scope ps(SELM_K_PROJECTION, st);
    k_scale<true><<<blocks_for(nf), kThreads, 0, st>>>(nf, u, h->weight, h->fw);
    MCK(cudaGetLastError());
    src = h->fw;
  }
  double* div = h->cg_q;   // the divergence (cells) as the pressure right-hand side
  {
    prof::Scope ps(SELM_K_PROJECTION, st);
    k_sell_mv<double, 0><<<blocks_for(h->D.npos), kThreads, 0, st>>>(h->D, src, div, nullptr);
    MCK(cudaGetLastError());
  }
  MCK(cudaMemcpyAsync(h->pv, div, h->n_cells * sizeof(double), cudaMemcpyDeviceToDevice, st));
  MRET(pressure_solve(h, h->pv, iters, resid, st));
  {
    prof::Scope ps(SELM_K_PROJECTION, st);
    // out = src - G phi
    k_sell_mv<double, 2><<<blocks_for(h->G.npos), kThreads, 0, st>>>(h->G, h->cg_x, adjoint ? h->fw2 : out, src);
    MCK(cudaGetLastError());
    if (adjoint) {
      k_scale<false><<<blocks_for(nf), kThreads, 0, st>>>(nf, h->fw2, h->weight, out);
      MCK(cudaGetLastError());
    }
  }
  return SELM_OK;
}

selm_status chain_cycles(selm_mac* h, int ncycles, cudaStream_t st) {
  for (int k = 0; k < ncycles; ++k) {
    MRET(outer_residual(h, h->xi, h->fw2, 4, st));
    MRET(correction_graph(h, 1.0, h->cyc, st));
    MRET(update(h, h->xi, st));
    MCK(launch_inc_u64(h->cyc, st));
    h->chain_cycle += 1;
    h->total_cycles += 1;
  }
  return SELM_OK;
}

selm_status interp(selm_mac* h, int np, const double* X, const double* u, double* U, cudaStream_t st) {
  {
    prof::Scope ps(SELM_K_INTERP, st);
    k_sell_mv<double, 0><<<blocks_for(h->E.npos), kThreads, 0, st>>>(h->E, u, h->fine_buf, nullptr);
    MCK(cudaGetLastError());
  }
  MCK(launch_interp(h->fine, 2 * h->d.n, h->d.dim, np, X, h->fine_buf, U, st));
  return SELM_OK;
}

selm_status spread(selm_mac* h, int np, const double* X, const double* F, double* f, cudaStream_t st) {
  MCK(cudaMemsetAsync(h->fine_buf, 0, h->fine_size * sizeof(double), st));
  MCK(launch_spread(h->fine, 2 * h->d.n, h->d.dim, np, X, F, h->fine_buf, st));
  prof::Scope ps(SELM_K_SPREAD, st);
  k_sell_mv<double, 0><<<blocks_for(h->Et.npos), kThreads, 0, st>>>(h->Et, h->fine_buf, f, nullptr);
  MCK(cudaGetLastError());
  return SELM_OK;
}

std::string fill_defaults(selm_mac_desc* d) {
  if (d->mu == 0.0) d->mu = 1.0;
  if (d->nu_pre == 0) d->nu_pre = 2;
  if (d->nu_post == 0) d->nu_post = 2;
  if (d->nu_patch == 0) d->nu_patch = 2;
  if (d->tol == 0.0) d->tol = 1e-10;
  if (d->max_cycles == 0) d->max_cycles = 100;
  if (d->proj_tol == 0.0) d->proj_tol = 1e-13;
  if (d->dim != 2 && d->dim != 3) return "dim must be 2 or 3";
  if (!(d->mu > 0.0) || d->kT < 0.0) return "mu must be positive and kT non-negative";
  if (d->nu_pre < 0 || d->nu_post < 0 || d->nu_patch < 0 || d->nu_pre + d->nu_post > 255 || d->nu_patch > 255)
    return "sweep counts out of range";
  if (d->precision != SELM_FP64 && d->precision != SELM_FP32_REFINE64) return "unknown precision";
  if (d->projection != SELM_PROJ_NONE && d->projection != SELM_PROJ_MAC) return "unknown projection";
  if (d->max_cycles < 0 || d->tol < 0.0 || d->proj_tol < 0.0) return "negative tolerance or cycle cap";
  return "";
}

}  // namespace

extern "C" {

selm_status selm_mac_create(const selm_mac_desc* desc, void* stream, selm_mac** out) {
  if (!desc || !out) return SELM_EINVAL;
  *out = nullptr;
  selm_mac_desc d = *desc;
  std::string e = fill_defaults(&d);
  Plan plan;
  if (e.empty()) e = build_plan(d.dim, d.n, d.K, d.levels, d.mu, &plan);
  if (e.empty() && plan.levels > 15) e = "too many levels";
  if (!e.empty()) {
    std::fprintf(stderr, "selm_mac_create: %s\n", e.c_str());
    return SELM_EINVAL;
  }
  for (const auto& cl : plan.colours)
    if (cl.size() > 4095) return SELM_EINVAL;
  selm_mac* h = new (std::nothrow) selm_mac();
  if (!h) return SELM_ENOMEM;
  h->d = d;
  h->esize = d.precision == SELM_FP32_REFINE64 ? 4 : 8;
  h->levels = plan.levels;
  h->n_faces = plan.n_faces;
  h->n_cells = plan.n_cells;
  h->key.k0 = (uint32_t)(d.seed & 0xffffffffu) ^ (uint32_t)(d.instance >> 32);
  h->key.k1 = (uint32_t)(d.seed >> 32) ^ (uint32_t)(d.instance & 0xffffffffu);
  cudaStream_t st = ST(stream);
  const bool f32 = h->esize == 4;
  auto fail = [&](selm_status s) {
    if (s != SELM_OK) {
      std::fprintf(stderr, "selm_mac_create: %s\n", h->err.c_str());
      selm_mac_destroy(h);
    }
    return s;
  };
  selm_status r = SELM_OK;
#define CREATE_STEP(x)          \
  do {                          \
    r = (x);                    \
    if (r != SELM_OK) return fail(r); \
  } while (0)
  CREATE_STEP(upload_sell(h, make_sell(plan.A, natural_order(plan.A.nr), false), false, &h->A64, st));
  {
    std::vector<int> slab_order = class_order(plan.patch_colours, &h->pstart, &h->psize);
    CREATE_STEP(upload_sell(h, make_sell(plan.A, slab_order, true), f32, &h->Apatch, st));
  }
  CREATE_STEP(upload_sell(h, make_sell(plan.P, natural_order(plan.P.nr), false), f32, &h->Pm, st));
  {
    Csr Pt;
    // P^T by rows of the base level
    Pt.nr = plan.P.nc;
    Pt.nc = plan.P.nr;
    std::vector<std::vector<std::pair<int, double>>> rows(Pt.nr);
    for (int rr = 0; rr < plan.P.nr; ++rr)
      for (long long q = plan.P.ptr[rr]; q < plan.P.ptr[rr + 1]; ++q) rows[plan.P.col[q]].push_back({rr, plan.P.val[q]});
    Pt.ptr.assign(Pt.nr + 1, 0);
    for (int rr = 0; rr < Pt.nr; ++rr) {
      for (auto& x : rows[rr]) {
        Pt.col.push_back(x.first);
        Pt.val.push_back(x.second);
      }
      Pt.ptr[rr + 1] = (long long)Pt.col.size();
    }
    CREATE_STEP(upload_sell(h, make_sell(Pt, natural_order(Pt.nr), false), f32, &h->Pt, st));
  }
  h->lev.resize(plan.levels);
  for (int l = 0; l < plan.levels; ++l) {
    selm_mac::Level& L = h->lev[l];
    L.N = plan.ops[l].nr;
    CREATE_STEP(alloc(h, (size_t)L.N * h->esize, &L.v, st));
    CREATE_STEP(alloc(h, (size_t)L.N * h->esize, &L.b, st));
    if (l + 1 < plan.levels) {
      CREATE_STEP(alloc(h, (size_t)L.N * h->esize, &L.t, st));
      std::vector<int> ord = class_order(plan.colours[l], &L.cstart, &L.csize);
      CREATE_STEP(upload_sell(h, make_sell(plan.ops[l], ord, true), f32, &L.cls, st));
      if (L.N <= kBlockSweepRows) {   // small level: its sweeps run in one block
        CREATE_STEP(upload(h, L.cstart, &L.d_cstart, st));
        CREATE_STEP(upload(h, L.csize, &L.d_csize, st));
        const int ncol = (int)L.cstart.size();
        const cudaError_t ce = f32 ? allow_block_smem<float>(block_sweep_smem<float>(L.N, ncol))
                                   : allow_block_smem<double>(block_sweep_smem<double>(L.N, ncol));
        if (ce != cudaSuccess) {
          h->err = std::string("block sweep shared memory: ") + cudaGetErrorString(ce);
          return fail(SELM_ECUDA);
        }
        L.block_sweeps = true;
      }
      const Csr& pl = plan.Pl[l];
      CREATE_STEP(upload_sell(h, make_sell(pl, natural_order(pl.nr), false), f32, &L.Pl, st));
      Csr plt;
      {
        plt.nr = pl.nc;
        plt.nc = pl.nr;
        std::vector<std::vector<std::pair<int, double>>> rows(plt.nr);
        for (int rr = 0; rr < pl.nr; ++rr)
          for (long long q = pl.ptr[rr]; q < pl.ptr[rr + 1]; ++q) rows[pl.col[q]].push_back({rr, pl.val[q]});
        plt.ptr.assign(plt.nr + 1, 0);
        for (int rr = 0; rr < plt.nr; ++rr) {
          for (auto& x : rows[rr]) {
            plt.col.push_back(x.first);
            plt.val.push_back(x.second);
          }
          plt.ptr[rr + 1] = (long long)plt.col.size();
        }
      }
      CREATE_STEP(upload_sell(h, make_sell(plt, natural_order(plt.nr), false), f32, &L.Plt, st));
    }
  }
  h->mc = plan.ops.back().nr;
  CREATE_STEP(upload(h, plan.Linv, &h->Linv, st));
  // (the host copy lives to the end of the set-up, like the plan's own arrays)
  std::vector<double> linv_t((size_t)h->mc * h->mc);
  for (int i = 0; i < h->mc; ++i)
    for (int j = 0; j < h->mc; ++j) linv_t[(size_t)j * h->mc + i] = plan.Linv[(size_t)i * h->mc + j];
  CREATE_STEP(upload(h, linv_t, &h->LinvT, st));
  CREATE_STEP(alloc(h, (size_t)h->mc * sizeof(double), (void**)&h->ycoarse, st));
  CREATE_STEP(upload_sell(h, make_sell(plan.D, natural_order(plan.D.nr), false), false, &h->D, st));
  CREATE_STEP(upload_sell(h, make_sell(plan.G, natural_order(plan.G.nr), false), false, &h->G, st));
  CREATE_STEP(upload_sell(h, make_sell(plan.S, natural_order(plan.S.nr), false), false, &h->S, st));
  {
    std::vector<double> minv(plan.n_cells, 0.0);
    for (int rr = 0; rr < plan.S.nr; ++rr)
      for (long long q = plan.S.ptr[rr]; q < plan.S.ptr[rr + 1]; ++q)
        if (plan.S.col[q] == rr && plan.S.val[q] != 0.0) minv[rr] = 1.0 / plan.S.val[q];
    CREATE_STEP(upload(h, minv, &h->minv, st));
  }
  CREATE_STEP(upload(h, plan.vol, &h->vol, st));
  CREATE_STEP(upload(h, plan.weight, &h->weight, st));
  h->total_vol = 0.0;
  for (double v : plan.vol) h->total_vol += v;
  CREATE_STEP(upload_sell(h, make_sell(plan.E, natural_order(plan.E.nr), false), false, &h->E, st));
  {
    Csr Et;
    Et.nr = plan.E.nc;
    Et.nc = plan.E.nr;
    std::vector<std::vector<std::pair<int, double>>> rows(Et.nr);
    for (int rr = 0; rr < plan.E.nr; ++rr)
      for (long long q = plan.E.ptr[rr]; q < plan.E.ptr[rr + 1]; ++q) rows[plan.E.col[q]].push_back({rr, plan.E.val[q]});
    Et.ptr.assign(Et.nr + 1, 0);
    for (int rr = 0; rr < Et.nr; ++rr) {
      for (auto& x : rows[rr]) {
        Et.col.push_back(x.first);
        Et.val.push_back(x.second);
      }
      Et.ptr[rr + 1] = (long long)Et.col.size();
    }
    CREATE_STEP(upload_sell(h, make_sell(Et, natural_order(Et.nr), false), false, &h->Et, st));
  }
  // the uniform fine lattice of the particle kernel
  h->fine.level = 0;
  h->fine.ncomp = plan.fine_ncomp;
  h->fine.size = plan.fine_size;
  for (int c = 0; c < plan.fine_ncomp; ++c) {
    CompDev& cd = h->fine.c[c];
    std::memset(&cd, 0, sizeof(cd));
    cd.nx = plan.fine_dims[c][0];
    cd.ny = plan.fine_dims[c][1];
    cd.nz = plan.fine_dims[c][2];
    cd.off = plan.fine_off[c];
    const bool normal = c == plan.fine_ncomp - 1;
    cd.comp_id = d.dim == 3 ? c : (c == 0 ? 0 : 2);
    cd.zkind = normal ? kAxisVertex : kAxisCellDir;
  }
  h->fine_size = plan.fine_size;
  // buffers
  const long long nf = plan.n_faces, nc = plan.n_cells;
  CREATE_STEP(alloc(h, (size_t)nf * h->esize, &h->r, st));
  CREATE_STEP(alloc(h, (size_t)nf * h->esize, &h->q, st));
  void* p = nullptr;
  CREATE_STEP(alloc(h, (size_t)nf * 8, &p, st));
  h->xi = (double*)p;
  CREATE_STEP(alloc(h, (size_t)nf * 8, &p, st));
  h->fw = (double*)p;
  CREATE_STEP(alloc(h, (size_t)nf * 8, &p, st));
  h->fw2 = (double*)p;
  CREATE_STEP(alloc(h, (size_t)plan.fine_size * 8, &p, st));
  h->fine_buf = (double*)p;
  for (double** b : {&h->cg_x, &h->cg_r, &h->cg_z, &h->cg_p, &h->cg_q, &h->pv}) {
    CREATE_STEP(alloc(h, (size_t)nc * 8, &p, st));
    *b = (double*)p;
  }
  CREATE_STEP(alloc(h, 2 * kRedBlocks * sizeof(double), &p, st));
  h->part = (double*)p;
  CREATE_STEP(alloc(h, 2 * kRedBlocks * sizeof(double), &p, st));
  h->part2 = (double*)p;
  CREATE_STEP(alloc(h, (size_t)blocks_for(h->A64.npos) * sizeof(double), &p, st));
  h->part_rows = (double*)p;
  CREATE_STEP(alloc(h, 16 * sizeof(double), &p, st));
  h->sc = (double*)p;
  CREATE_STEP(alloc(h, 2 * sizeof(unsigned long long), &p, st));
  h->cyc = (unsigned long long*)p;
  h->cyc_user = h->cyc + 1;
  if (cudaMallocHost(&p, 16 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    h->err = "pinned allocation failed";
    return fail(SELM_ENOMEM);
  }
  h->host_sc = (double*)p;
  if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    h->cap = nullptr;
    h->graphs = false;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    h->err = "set-up copies failed";
    return fail(SELM_ECUDA);
  }
#undef CREATE_STEP
  *out = h;
  return SELM_OK;
}

selm_status selm_mac_destroy(selm_mac* h) {
  if (!h) return SELM_EINVAL;
  for (auto& g : h->gexec)
    if (g) cudaGraphExecDestroy(g);
  if (h->cg_exec) cudaGraphExecDestroy(h->cg_exec);
  if (h->cap) cudaStreamDestroy(h->cap);
  for (void* p : h->allocs) cudaFree(p);
  if (h->host_sc) cudaFreeHost(h->host_sc);
  delete h;
  return SELM_OK;
}

const char* selm_mac_last_error(const selm_mac* h) { return h ? h->err.c_str() : "null handle"; }
long long selm_mac_faces(const selm_mac* h) { return h ? h->n_faces : -1; }
long long selm_mac_cells(const selm_mac* h) { return h ? h->n_cells : -1; }
int selm_mac_levels(const selm_mac* h) { return h ? h->levels : -1; }
int selm_mac_colours(const selm_mac* h, int level) {
  if (!h) return -1;
  if (level == -1) return (int)h->pstart.size();
  if (level < 0 || level >= h->levels) return -1;
  return (int)h->lev[level].cstart.size();
}
int selm_mac_inner_bytes(const selm_mac* h) { return h ? h->esize : -1; }
long long selm_mac_total_cycles(const selm_mac* h) { return h ? h->total_cycles : -1; }

selm_status selm_mac_apply(selm_mac* h, const double* u, double* Au, void* stream) {
  if (!h || !u || !Au) return SELM_EINVAL;
  cudaStream_t st = ST(stream);
  prof::Scope ps(SELM_K_OTHER, st);
  k_sell_mv<double, 0><<<blocks_for(h->A64.npos), kThreads, 0, st>>>(h->A64, u, Au, nullptr);
  MCK(cudaGetLastError());
  return SELM_OK;
}

selm_status selm_mac_divergence(selm_mac* h, const double* u, double* div, void* stream) {
  if (!h || !u || !div) return SELM_EINVAL;
  cudaStream_t st = ST(stream);
  prof::Scope ps(SELM_K_PROJECTION, st);
  k_sell_mv<double, 0><<<blocks_for(h->D.npos), kThreads, 0, st>>>(h->D, u, div, nullptr);
  MCK(cudaGetLastError());
  return SELM_OK;
}

selm_status selm_mac_gradient(selm_mac* h, const double* p, double* grad, void* stream) {
  if (!h || !p || !grad) return SELM_EINVAL;
  cudaStream_t st = ST(stream);
  prof::Scope ps(SELM_K_PROJECTION, st);
  k_sell_mv<double, 0><<<blocks_for(h->G.npos), kThreads, 0, st>>>(h->G, p, grad, nullptr);
  MCK(cudaGetLastError());
  return SELM_OK;
}

selm_status selm_mac_project(selm_mac* h, const double* u, double* out, int adjoint, int* iters, double* resid,
                             void* stream) {
  if (!h || !u || !out || (adjoint != 0 && adjoint != 1)) return SELM_EINVAL;
  return project(h, u, out, adjoint, iters, resid, ST(stream));
}

selm_status selm_mac_fac_cycle(selm_mac* h, double* z, const double* b, double sigma, uint64_t cycle, void* stream) {
  if (!h || !z || !b || !(sigma >= 0.0)) return SELM_EINVAL;
  cudaStream_t st = ST(stream);
  MCK(launch_set_u64(h->cyc_user, cycle, st));
  return fac_cycle(h, z, b, sigma, h->cyc_user, st);
}

selm_status selm_mac_solve(selm_mac* h, double* z, const double* b, double tol, int max_cycles, int* cycles,
                           double* rel, void* stream) {
  if (!h || !z || !b || tol < 0.0 || max_cycles < 0) return SELM_EINVAL;
  return solve(h, z, b, tol > 0.0 ? tol : h->d.tol, max_cycles > 0 ? max_cycles : h->d.max_cycles, cycles, rel,
               ST(stream));
}

selm_status selm_mac_sample(selm_mac* h, int ncycles, double* xi_out, void* stream) {
  if (!h || ncycles < 0) return SELM_EINVAL;
  cudaStream_t st = ST(stream);
  MCK(cudaMemsetAsync(h->fw2, 0, h->n_faces * sizeof(double), st));   // b = 0
  MRET(chain_cycles(h, ncycles, st));
  if (xi_out) MCK(cudaMemcpyAsync(xi_out, h->xi, h->n_faces * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return SELM_OK;
}

selm_status selm_mac_chain(selm_mac* h, double** xi, uint64_t* cycle) {
  if (!h) return SELM_EINVAL;
  if (xi) *xi = h->xi;
  if (cycle) *cycle = h->chain_cycle;
  return SELM_OK;
}

selm_status selm_mac_set_chain(selm_mac* h, uint64_t cycle, void* stream) {
  if (!h) return SELM_EINVAL;
  cudaStream_t st = ST(stream);
  MCK(cudaMemsetAsync(h->xi, 0, h->n_faces * sizeof(double), st));
  MCK(launch_set_u64(h->cyc, cycle, st));
  h->chain_cycle = cycle;
  return SELM_OK;
}

selm_status selm_mac_interp(selm_mac* h, int np, const double* X, const double* u, double* U, void* stream) {
  if (!h || np < 0 || (np > 0 && (!X || !u || !U))) return SELM_EINVAL;
  if (np == 0) return SELM_OK;
  return interp(h, np, X, u, U, ST(stream));
}

selm_status selm_mac_spread(selm_mac* h, int np, const double* X, const double* F, double* f, void* stream) {
  if (!h || np < 0 || !f || (np > 0 && (!X || !F))) return SELM_EINVAL;
  cudaStream_t st = ST(stream);
  if (np == 0) {
    MCK(cudaMemsetAsync(f, 0, h->n_faces * sizeof(double), st));
    return SELM_OK;
  }
  return spread(h, np, X, F, f, st);
}

selm_status selm_mac_mobility(selm_mac* h, int np, const double* X, const double* F, double* U, int* cycles,
                              void* stream) {
  if (!h || np < 0 || (np > 0 && (!X || !F || !U))) return SELM_EINVAL;
  if (np == 0) return SELM_OK;
  cudaStream_t st = ST(stream);
  const bool proj = h->d.projection == SELM_PROJ_MAC;
  MRET(spread(h, np, X, F, h->fw, st));
  if (proj) MRET(project(h, h->fw, h->fw, 1, nullptr, nullptr, st));
  // u = A^-1 f in fw2 (from zero)
  MCK(cudaMemsetAsync(h->fw2, 0, h->n_faces * sizeof(double), st));
  MRET(solve(h, h->fw2, h->fw, h->d.tol, h->d.max_cycles, cycles, nullptr, st));
  if (proj) MRET(project(h, h->fw2, h->fw2, 0, nullptr, nullptr, st));
  return interp(h, np, X, h->fw2, U, st);
}

selm_status selm_mac_thermal(selm_mac* h, int np, const double* X, int ncycles, double* g, void* stream) {
  if (!h || np < 0 || ncycles < 0 || (np > 0 && (!X || !g))) return SELM_EINVAL;
  cudaStream_t st = ST(stream);
  MCK(cudaMemsetAsync(h->fw2, 0, h->n_faces * sizeof(double), st));
  MRET(chain_cycles(h, ncycles, st));
  if (np == 0) return SELM_OK;
  const double* w = h->xi;
  if (h->d.projection == SELM_PROJ_MAC) {
    MRET(project(h, h->xi, h->fw, 0, nullptr, nullptr, st));
    w = h->fw;
  }
  MRET(interp(h, np, X, w, g, st));
  const double c = std::sqrt(2.0 * h->d.kT);
  MCK(launch_axpby((long long)np * h->d.dim, c, g, 0.0, g, g, st));
  return SELM_OK;
}

selm_status selm_mac_step(selm_mac* h, int np, double* X, const double* F, double dt, int nsteps, int ncycles,
                          void* stream) {
  if (!h || np < 0 || nsteps < 0 || ncycles < 0 || !(dt >= 0.0) || (np > 0 && (!X || !F))) return SELM_EINVAL;
  if (np == 0) return SELM_OK;
  cudaStream_t st = ST(stream);
  if (np > h->max_np) {
    void* p = nullptr;
    MRET(alloc(h, (size_t)np * h->d.dim * 2 * sizeof(double), &p, st));
    h->pX = (double*)p;
    h->max_np = np;
  }
  double* V = h->pX;
  const bool proj = h->d.projection == SELM_PROJ_MAC;
  const long long nf = h->n_faces;
  for (int s = 0; s < nsteps; ++s) {
    // u = A^-1 P~^T Gamma^T F (fw: right-hand side, then the field of the step)
    MRET(spread(h, np, X, F, h->fw, st));
    if (proj) MRET(project(h, h->fw, h->fw, 1, nullptr, nullptr, st));
    // the solve writes into fw2 (from zero), then the chain runs with b = 0
    MCK(cudaMemcpyAsync(h->fw2, h->fw, nf * sizeof(double), cudaMemcpyDeviceToDevice, st));
    MCK(cudaMemsetAsync(h->fw, 0, nf * sizeof(double), st));
    MRET(solve(h, h->fw, h->fw2, h->d.tol, h->d.max_cycles, nullptr, nullptr, st));
    MCK(cudaMemsetAsync(h->fw2, 0, nf * sizeof(double), st));
    MRET(chain_cycles(h, ncycles, st));
    // w = dt u + sqrt(2 kT dt) xi; V = Gamma P~ w
    MCK(launch_axpby(nf, dt, h->fw, std::sqrt(2.0 * h->d.kT * dt), h->xi, h->fw, st));
    if (proj) MRET(project(h, h->fw, h->fw, 0, nullptr, nullptr, st));
    MRET(interp(h, np, X, h->fw, V, st));
    MCK(launch_em(np, h->d.dim, X, V, st));
  }
  return SELM_OK;
}

selm_status selm_mac_host_matrix(const selm_mac_desc* desc, int which, int level, int* nr, int* nc, long long* nnz,
                                 long long** ptr, int** col, double** val) {
  if (!desc || !nr || !nc || !nnz || !ptr || !col || !val) return SELM_EINVAL;
  selm_mac_desc d = *desc;
  std::string e = fill_defaults(&d);
  Plan plan;
  if (e.empty()) e = build_plan(d.dim, d.n, d.K, d.levels, d.mu, &plan);
  if (!e.empty()) return SELM_EINVAL;
  const Csr* m = nullptr;
  switch (which) {
    case SELM_MAC_MAT_A: m = &plan.A; break;
    case SELM_MAC_MAT_D: m = &plan.D; break;
    case SELM_MAC_MAT_G: m = &plan.G; break;
    case SELM_MAC_MAT_S: m = &plan.S; break;
    case SELM_MAC_MAT_P: m = &plan.P; break;
    case SELM_MAC_MAT_E: m = &plan.E; break;
    case SELM_MAC_MAT_OPS:
      if (level >= 0 && level < (int)plan.ops.size()) m = &plan.ops[level];
      break;
    case SELM_MAC_MAT_PL:
      if (level >= 0 && level < (int)plan.Pl.size()) m = &plan.Pl[level];
      break;
    default: break;
  }
  if (!m) return SELM_EINVAL;
  *nr = m->nr;
  *nc = m->nc;
  *nnz = m->nnz();
  *ptr = (long long*)std::malloc(sizeof(long long) * (m->nr + 1));
  *col = (int*)std::malloc(sizeof(int) * std::max<long long>(1, m->nnz()));
  *val = (double*)std::malloc(sizeof(double) * std::max<long long>(1, m->nnz()));
  if (!*ptr || !*col || !*val) {
    std::free(*ptr);
    std::free(*col);
    std::free(*val);
    return SELM_ENOMEM;
  }
  std::memcpy(*ptr, m->ptr.data(), sizeof(long long) * (m->nr + 1));
  std::memcpy(*col, m->col.data(), sizeof(int) * m->nnz());
  std::memcpy(*val, m->val.data(), sizeof(double) * m->nnz());
  return SELM_OK;
}

selm_status selm_mac_host_colours(const selm_mac_desc* desc, int level, int* n, int** colour) {
  if (!desc || !n || !colour) return SELM_EINVAL;
  selm_mac_desc d = *desc;
  std::string e = fill_defaults(&d);
  Plan plan;
  if (e.empty()) e = build_plan(d.dim, d.n, d.K, d.levels, d.mu, &plan);
  if (!e.empty()) return SELM_EINVAL;
  const std::vector<std::vector<int>>* cl = nullptr;
  int rows = 0;
  if (level == -1) {
    cl = &plan.patch_colours;
    rows = plan.n_faces;
  } else if (level >= 0 && level < (int)plan.colours.size()) {
    cl = &plan.colours[level];
    rows = plan.ops[level].nr;
  }
  if (!cl) return SELM_EINVAL;
  *n = rows;
  *colour = (int*)std::malloc(sizeof(int) * std::max(1, rows));
  if (!*colour) return SELM_ENOMEM;
  for (int i = 0; i < rows; ++i) (*colour)[i] = -1;
  for (size_t c = 0; c < cl->size(); ++c)
    for (int r : (*cl)[c]) (*colour)[r] = (int)c;
  return SELM_OK;
}

void selm_mac_host_free(void* p) { std::free(p); }

}  // extern "C"
