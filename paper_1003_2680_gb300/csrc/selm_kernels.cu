// CUDA kernels of the stochastic multigrid SELM path (sm_103a).
//
// Every hot-path step is an HBM-bound stencil; none is a dense contraction,
// so the tensor cores are not used.  Step -> kernel:
//   Gibbs sweep, level 0 (Section 3.1, red-black)      k_fine_colour
//   Gibbs sweep, Galerkin levels (multicolour)         k_coarse_site, k_level_coop, coarse engine
//   residual (Alg. 3 step 3)                           k_residual
//   restriction P^T (Eq. equ_restr_prolong_variation)  k_restrict
//   prolongation + correction (Alg. 3 step 4)          k_prolong
//   coarsest exact step (reading of Alg. 3 step 2)     k_coarsest
//   FP64 outer residual / update (Alg. 1 steps 1, 4)   k_outer_residual, k_outer_update
//   Peskin spread / interpolation (Section 2.1)        k_spread, k_interp
//   MAC divergence / gradient (Section 4)              k_divergence, k_grad_sub
//   Euler-Maruyama update (Alg. 4 step 4)              k_em

#include <cuda_runtime.h>

#include <atomic>
#include <type_traits>
#include <cstdint>
#include <cstring>
#include <new>
#include <mutex>
#include <vector>

#include "../../include/selm_mg.h"
#include "selm_internal.h"
#include "selm_launch.h"
#include "selm_devmath.h"
#include "selm_pdl.h"
#include "selm_prof.h"

// Returns the error of a launch from the enclosing launcher.
#define LTRY(call)                            \
  do {                                        \
    const cudaError_t e_ = (call);            \
    if (e_ != cudaSuccess) return e_;         \
  } while (0)

namespace selm {

// ---------------------------------------------------------------------------
// Kernel accounting: a launch counter and optional event timing per kernel
// class (events recorded on the launching stream).
// ---------------------------------------------------------------------------
namespace prof {
std::atomic<long long> g_launches{0};
std::mutex g_mu;
bool g_on = false;
std::vector<cudaEvent_t> g_pool;
struct Pending {
  int kind;
  cudaEvent_t a, b;
};
std::vector<Pending> g_pending;
double g_ms[SELM_K_NCLASSES] = {};
long long g_count[SELM_K_NCLASSES] = {};

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void drain() {
  for (auto& p : g_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      g_ms[p.kind] += ms;
      g_count[p.kind] += 1;
    }
    g_pool.push_back(p.a);
    g_pool.push_back(p.b);
  }
  g_pending.clear();
}

Scope::Scope(int k, cudaStream_t s) : kind(k), st(s), a(nullptr) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (g_on) {
    std::lock_guard<std::mutex> lk(g_mu);
    a = take_event();
    if (a) cudaEventRecord(a, st);
  }
}

Scope::~Scope() {
  if (!a) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = take_event();
  if (!b) return;
  cudaEventRecord(b, st);
  g_pending.push_back({kind, a, b});
  if (g_pending.size() > 4096) drain();
}
}  // namespace prof

namespace {

constexpr int kBlock = 256;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Box-Muller.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) { return philox4x32_10(c, k0, k1); }

__device__ __forceinline__ uint32_t ctr1_of(int level, int comp, int colour, int sweep, int kind) {
  return (uint32_t)level | ((uint32_t)comp << 4) | ((uint32_t)colour << 8) | ((uint32_t)sweep << 12) |
         ((uint32_t)kind << 20);
}

template <typename T>
__device__ __forceinline__ const T* stencil_of(const CompDev& c);
template <>
__device__ __forceinline__ const double* stencil_of<double>(const CompDev& c) {
  return c.S64;
}
template <>
__device__ __forceinline__ const float* stencil_of<float>(const CompDev& c) {
  return c.S32;
}

template <typename T>
__device__ __forceinline__ T rz_w(const CompDev& c, int q);
template <>
__device__ __forceinline__ double rz_w<double>(const CompDev& c, int q) {
  return c.rz_w64[q];
}
template <>
__device__ __forceinline__ float rz_w<float>(const CompDev& c, int q) {
  return c.rz_w32[q];
}
template <typename T>
__device__ __forceinline__ T pz_w(const CompDev& c, int q);
template <>
__device__ __forceinline__ double pz_w<double>(const CompDev& c, int q) {
  return c.pz_w64[q];
}
template <>
__device__ __forceinline__ float pz_w<float>(const CompDev& c, int q) {
  return c.pz_w32[q];
}

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Level-0 operator: s * sum over axes of (2 v - v_left - v_right), with the
// wall ghost rules folded into the diagonal.  Returns the off-diagonal part
// sum_{j != i} A_ij v_j and the diagonal A_ii.
template <typename T, typename V>
__device__ __forceinline__ void fine_row(const CompDev& c, const V* __restrict__ v, int i, int j, int k,
                                         T* off, T* diag) {
  const long long plane = (long long)c.nx * c.ny;
  const long long row = c.off + (long long)k * plane + (long long)j * c.nx;
  T sum = (T)v[row + wrapi(i - 1, c.nx)] + (T)v[row + wrapi(i + 1, c.nx)];
  T d = (T)2;
  if (c.ny > 1) {
    const long long base = c.off + (long long)k * plane + i;
    sum += (T)v[base + (long long)wrapi(j - 1, c.ny) * c.nx] + (T)v[base + (long long)wrapi(j + 1, c.ny) * c.nx];
    d += (T)2;
  }
  const long long idx = row + i;
  if (k > 0) sum += (T)v[idx - plane];
  if (k < c.nz - 1) sum += (T)v[idx + plane];
  int edges = (k == 0) + (k == c.nz - 1);
  T dz = (T)2;
  if (c.zkind == kAxisCellDir) dz += (T)edges;
  if (c.zkind == kAxisCellNeu) dz -= (T)edges;
  const T s = (T)c.s;
  *off = -s * sum;
  *diag = s * (d + dz);
}

// Galerkin-level operator: full 3x3x5 stencil row k (periodic wrap in x, y).
template <typename T>
__device__ __forceinline__ T coarse_diag(const CompDev& c, int k) {
  return stencil_of<T>(c)[(long long)k * kStencil + 22];
}

__device__ __forceinline__ int comp_of(const long long* start, int ncomp, long long g) {
  int c = 0;
  while (c + 1 < ncomp && g >= start[c + 1]) ++c;
  return c;
}

// ---------------------------------------------------------------------------
// Gibbs sweeps
// ---------------------------------------------------------------------------
struct ColourPass {
  long long gstart[kMaxComps + 1];  // first noise group of each component
  long long nsites[kMaxComps];
  int cx[kMaxComps], cy[kMaxComps], cz[kMaxComps];     // colour tuple (levels >= 1)
  int nxc[kMaxComps], nyc[kMaxComps], nzc[kMaxComps];  // extents of the colour class
  int lxc[kMaxComps], lyc[kMaxComps];                  // log2 of nxc / nyc when powers of two, else -1
  int colour_id[kMaxComps];
};

// Level 0, red-black: one thread updates the four consecutive-rank sites of
// one noise group (one Philox call).  Sites of colour `colour` satisfy
// (i + j + k) % 2 == colour; rank = (k ny + j) nx/2 + i/2.
template <typename T, bool NOISE>
__global__ void __launch_bounds__(kBlock) k_fine_colour(LevelDev L, ColourPass cp, T* __restrict__ v,
                                                       const T* __restrict__ b, int colour, int sweep,
                                                       Key key, const unsigned long long* __restrict__ cyc) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= cp.gstart[L.ncomp]) return;
  const int ci = comp_of(cp.gstart, L.ncomp, g);
  const CompDev& c = L.c[ci];
  const long long gl = g - cp.gstart[ci];
  T nz4[4] = {(T)0, (T)0, (T)0, (T)0};
  if (NOISE) {
    const unsigned long long cy = *cyc;
    uint4 ctr = make_uint4((uint32_t)gl, ctr1_of(L.level, c.comp_id, colour, sweep, 0), (uint32_t)cy,
                           (uint32_t)(cy >> 32));
    Normals<T>::get(philox10(ctr, key.k0, key.k1), nz4);
  }
  const int half = c.nx >> 1;
#pragma unroll
  for (int lane = 0; lane < 4; ++lane) {
    const long long rank = gl * 4 + lane;
    if (rank >= cp.nsites[ci]) break;
    const int m = (int)(rank % half);
    const long long rw = rank / half;
    const int j = (int)(rw % c.ny), k = (int)(rw / c.ny);
    const int i = 2 * m + ((j + k + colour) & 1);
    T off, diag;
    fine_row<T, T>(c, v, i, j, k, &off, &diag);
    const long long idx = c.off + ((long long)k * c.ny + j) * c.nx + i;
    T nv = (b[idx] - off) / diag;
    if (NOISE) nv += nz4[lane] / tsqrt(diag);
    v[idx] = nv;
  }
}

__device__ __forceinline__ double block_sum(double x) {
  __shared__ double red[kBlock / 32];
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = x;
  __syncthreads();
  x = (threadIdx.x < blockDim.x / 32) ? red[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// Level 0, red-black, vectorised: one thread owns the 8 consecutive x
// positions [8g, 8g+8) of one row (requires nx % 8 == 0).  These hold exactly
// the four sites of colour `colour` of one noise group (ranks 4g'..4g'+3 of
// the class), so one Philox call serves the thread.  Centre, y+-1, z+-1 and b
// rows are read with 16-byte vector loads; the x neighbours at the segment
// ends are scalar loads.  The whole segment is written back: its
// other-colour entries are unchanged and are the only entries other threads
// read during this pass.
// Updates the four sites of parity P in an 8-wide segment (compile-time
// indices keep the arrays in registers).
template <typename T, bool NOISE, int P>
__device__ __forceinline__ void fine_update8(T cen[8], const T bb[8], const T acc[8], T left, T right, const T n4[4],
                                             T s, T rdiag, T rsd) {
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    const int e = 2 * l + P;
    const T xl = e == 0 ? left : cen[e - 1];
    const T xr = e == 7 ? right : cen[e + 1];
    T nv = (bb[e] + s * (acc[e] + xl + xr)) * rdiag;   // rdiag = 1 / A_ii of the row
    if (NOISE) nv += n4[l] * rsd;
    cen[e] = nv;
  }
}

struct RowPass {
  int rstart[kMaxComps + 1];   // first row of each component (rows = ny * nz)
};

// FP64 outer residual, vectorised over 4 consecutive x positions (nx % 4 == 0).
template <typename T, bool NORM>
__global__ void __launch_bounds__(kBlock) k_outer_residual_v4(LevelDev L, RowPass rp, const double* __restrict__ z,
                                                             const double* __restrict__ b, T* __restrict__ r,
                                                             double* __restrict__ norm2) {
  pdl_enter();
  const int segs = L.c[0].nx >> 2;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int row_all = gt / segs;
  double rr = 0.0;
  if (row_all < rp.rstart[L.ncomp]) {
    const int seg = gt - row_all * segs;
    int ci = 0;
    while (ci + 1 < L.ncomp && row_all >= rp.rstart[ci + 1]) ++ci;
    const CompDev& c = L.c[ci];
    const int row = row_all - rp.rstart[ci];
    const int j = row % c.ny, k = row / c.ny;
    const int nx = c.nx;
    const long long plane = (long long)nx * c.ny;
    const long long rbase = c.off + (long long)row * nx;
    const int x0 = seg << 2;
    double cen[4], acc[4];
    {
      const double2 a = *reinterpret_cast<const double2*>(z + rbase + x0);
      const double2 d = *reinterpret_cast<const double2*>(z + rbase + x0 + 2);
      cen[0] = a.x; cen[1] = a.y; cen[2] = d.x; cen[3] = d.y;
    }
    const double left = z[rbase + (x0 == 0 ? nx - 1 : x0 - 1)];
    const double right = z[rbase + (x0 + 4 == nx ? 0 : x0 + 4)];
    acc[0] = left + cen[1];
    acc[1] = cen[0] + cen[2];
    acc[2] = cen[1] + cen[3];
    acc[3] = cen[2] + right;
    auto add4 = [&](long long off) {
      const double2 a = *reinterpret_cast<const double2*>(z + off);
      const double2 d = *reinterpret_cast<const double2*>(z + off + 2);
      acc[0] += a.x; acc[1] += a.y; acc[2] += d.x; acc[3] += d.y;
    };
    if (c.ny > 1) {
      add4(c.off + ((long long)k * c.ny + (j == 0 ? c.ny - 1 : j - 1)) * nx + x0);
      add4(c.off + ((long long)k * c.ny + (j == c.ny - 1 ? 0 : j + 1)) * nx + x0);
    }
    if (k > 0) add4(rbase - plane + x0);
    if (k < c.nz - 1) add4(rbase + plane + x0);
    const int edges = (k == 0) + (k == c.nz - 1);
    double dz = 2.0;
    if (c.zkind == kAxisCellDir) dz += (double)edges;
    if (c.zkind == kAxisCellNeu) dz -= (double)edges;
    const double dg = (c.ny > 1 ? 4.0 : 2.0) + dz;
    const double sdg = c.s * dg;
    double bv[4] = {0.0, 0.0, 0.0, 0.0};
    if (b) {
      const double2 a = *reinterpret_cast<const double2*>(b + rbase + x0);
      const double2 d = *reinterpret_cast<const double2*>(b + rbase + x0 + 2);
      bv[0] = a.x; bv[1] = a.y; bv[2] = d.x; bv[3] = d.y;
    }
    T out[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      // b - s (dg z - sum) as two FMAs: GB300's FP64 rate bounds this kernel
      const double res = fma(c.s, acc[e], fma(-sdg, cen[e], bv[e]));
      out[e] = (T)res;
      if (NORM) rr = fma(res, res, rr);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) r[rbase + x0 + e] = out[e];
  }
  if (NORM) {
    rr = block_sum(rr);
    if (threadIdx.x == 0) atomicAdd(norm2, rr);
  }
}

// ---- the FP64 outer residual without the FP64 pipe ---------------------------
// GB300 issues FP64 arithmetic and conversions at about two per SM clock, so
// the nine FP64 operations per unknown of the plain residual bound it at
// several times its memory time.  With an FP32 output the residual is formed
// instead in exact integer arithmetic: the level-0 stencil's coefficients are
// integers times s (A z = s (dg z_c - sum of the neighbours)), so with every
// z of a thread's window written as a fixed-point integer Z = m 2^(e - emax)
// 2^5 relative to the window's largest exponent emax (|Z| < 2^58, the bits
// dropped from smaller values lie below 2^-58 of the window's largest value,
// far under FP64's own rounding of the sum), S = dg Z_c - sum Z_nb is exact in
// 64-bit integers, is rounded once to FP64 by integer operations, and
// r = b - s S 2^(emax - 1080) is one FP64 FMA (its square for the norm a
// second); the FP32 rounding of r is done by integer operations too.  The result is the exact residual up to two
// roundings (the plain form accumulates nine), so it satisfies the FP64
// residual's accuracy.  Windows outside the guarded exponent range (zero,
// tiny, huge, non-finite values) take the plain FP64 arithmetic.

__device__ __forceinline__ int fx_exp(long long bits) { return (int)((unsigned long long)bits >> 52) & 0x7ff; }

// z (as bits) -> Z = m 32 2^-(emax - e), m the signed 53-bit significand.
__device__ __forceinline__ long long fx_align(long long bits, int emax) {
  const int ex = fx_exp(bits);
  long long m = (bits & 0x000FFFFFFFFFFFFFll) | (ex ? 0x0010000000000000ll : 0ll);
  if (bits < 0) m = -m;
  const int d = emax - (ex ? ex : 1);
  return d >= 63 ? (m < 0 ? -1ll : 0ll) : ((m * 32) >> d);
}

// S 2^e2 rounded to nearest even as FP64 (S != 0 and the result normal,
// which the caller's exponent guard ensures).
__device__ __forceinline__ double fx_to_double(long long S, int e2) {
  const unsigned long long sign = S < 0 ? 0x8000000000000000ull : 0ull;
  unsigned long long a = S < 0 ? (unsigned long long)(-S) : (unsigned long long)S;
  const int lz = __clzll((long long)a);
  a <<= lz;
  unsigned long long mant = a >> 11;
  const unsigned long long rem = a & 0x7ffull;
  int E = 63 - lz + e2;
  if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) {
    ++mant;
    if (mant >> 53) {
      mant >>= 1;
      ++E;
    }
  }
  return __longlong_as_double((long long)(sign | ((unsigned long long)(E + 1023) << 52) | (mant & 0x000FFFFFFFFFFFFFull)));
}

// FP64 -> FP32, round to nearest even, by integer operations on the normal
// FP32 range; other values through the conversion instruction.
__device__ __forceinline__ float fx_to_float(double x) {
  const long long b = __double_as_longlong(x);
  const int ex = fx_exp(b);
  if (ex < 1023 - 126 || ex > 1023 + 127) return __double2float_rn(x);
  const unsigned long long mant = (unsigned long long)b & 0x000FFFFFFFFFFFFFull;
  const unsigned m23 = (unsigned)(mant >> 29);
  const unsigned long long rem = mant & 0x1FFFFFFFull;
  unsigned f = ((unsigned)((unsigned long long)b >> 32) & 0x80000000u) | ((unsigned)(ex - 1023 + 127) << 23) | m23;
  if (rem > 0x10000000ull || (rem == 0x10000000ull && (m23 & 1u))) f += 1u;
  return __uint_as_float(f);
}

// The FP32-output residual of k_outer_residual_v4 in the exact form above.
template <bool NORM>
__global__ void __launch_bounds__(kBlock) k_outer_residual_fx(LevelDev L, RowPass rp, const double* __restrict__ z,
                                                             const double* __restrict__ b, float* __restrict__ r,
                                                             double* __restrict__ norm2) {
  pdl_enter();
  const int segs = L.c[0].nx >> 2;
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  const int row_all = gt / segs;
  double rr = 0.0;
  if (row_all < rp.rstart[L.ncomp]) {
    const int seg = gt - row_all * segs;
    int ci = 0;
    while (ci + 1 < L.ncomp && row_all >= rp.rstart[ci + 1]) ++ci;
    const CompDev& c = L.c[ci];
    const int row = row_all - rp.rstart[ci];
    const int j = row % c.ny, k = row / c.ny;
    const int nx = c.nx;
    const long long plane = (long long)nx * c.ny;
    const long long rbase = c.off + (long long)row * nx;
    const int x0 = seg << 2;
    // the window as FP64 bit patterns: the centre row (4, left, right), then
    // the rows y-1, y+1, z-1, z+1 in fixed slots, an absent row as zeros
    // (which add nothing and do not raise the window's exponent)
    long long w[22];
    auto ld4 = [&](bool present, long long off, long long* dst) {
      if (present) {
        const longlong2 a = *reinterpret_cast<const longlong2*>(z + off);
        const longlong2 d = *reinterpret_cast<const longlong2*>(z + off + 2);
        dst[0] = a.x; dst[1] = a.y; dst[2] = d.x; dst[3] = d.y;
      } else {
        dst[0] = 0; dst[1] = 0; dst[2] = 0; dst[3] = 0;
      }
    };
    ld4(true, rbase + x0, w);
    w[4] = __double_as_longlong(z[rbase + (x0 == 0 ? nx - 1 : x0 - 1)]);
    w[5] = __double_as_longlong(z[rbase + (x0 + 4 == nx ? 0 : x0 + 4)]);
    const bool ys = c.ny > 1;
    ld4(ys, c.off + ((long long)k * c.ny + (j == 0 ? c.ny - 1 : j - 1)) * nx + x0, w + 6);
    ld4(ys, c.off + ((long long)k * c.ny + (j == c.ny - 1 ? 0 : j + 1)) * nx + x0, w + 10);
    ld4(k > 0, rbase - plane + x0, w + 14);
    ld4(k < c.nz - 1, rbase + plane + x0, w + 18);
    int emax = 0;
#pragma unroll
    for (int q = 0; q < 22; ++q) emax = max(emax, fx_exp(w[q]));
    const int edges = (k == 0) + (k == c.nz - 1);
    int dz = 2;
    if (c.zkind == kAxisCellDir) dz += edges;
    if (c.zkind == kAxisCellNeu) dz -= edges;
    const long long dg = (c.ny > 1 ? 4 : 2) + dz;
    double bv[4] = {0.0, 0.0, 0.0, 0.0};
    if (b) {
      const double2 a = *reinterpret_cast<const double2*>(b + rbase + x0);
      const double2 d = *reinterpret_cast<const double2*>(b + rbase + x0 + 2);
      bv[0] = a.x; bv[1] = a.y; bv[2] = d.x; bv[3] = d.y;
    }
    float out[4];
    double res[4];                         // the FP64 residual (its norm is FP64 too)
    if (emax == 0) {                       // z = 0 on the window: r = b
#pragma unroll
      for (int e = 0; e < 4; ++e) res[e] = bv[e];
    } else if (emax >= 64 && emax <= 2000) {
      long long Z[22];
#pragma unroll
      for (int q = 0; q < 22; ++q) Z[q] = fx_align(w[q], emax);
      long long S[4];
      S[0] = Z[4] + Z[1];
      S[1] = Z[0] + Z[2];
      S[2] = Z[1] + Z[3];
      S[3] = Z[2] + Z[5];
#pragma unroll
      for (int q = 6; q < 22; q += 4) {
        S[0] += Z[q]; S[1] += Z[q + 1]; S[2] += Z[q + 2]; S[3] += Z[q + 3];
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const long long t = dg * Z[e] - S[e];
        const double az = t == 0 ? 0.0 : fx_to_double(t, emax - 1080);
        res[e] = fma(-c.s, az, bv[e]);
      }
    } else {                               // the plain FP64 arithmetic
      double cz[22];
#pragma unroll
      for (int q = 0; q < 22; ++q) cz[q] = __longlong_as_double(w[q]);
      double acc[4];
      acc[0] = cz[4] + cz[1];
      acc[1] = cz[0] + cz[2];
      acc[2] = cz[1] + cz[3];
      acc[3] = cz[2] + cz[5];
#pragma unroll
      for (int q = 6; q < 22; q += 4) {
        acc[0] += cz[q]; acc[1] += cz[q + 1]; acc[2] += cz[q + 2]; acc[3] += cz[q + 3];
      }
      const double sdg = c.s * (double)dg;
#pragma unroll
      for (int e = 0; e < 4; ++e) res[e] = fma(c.s, acc[e], fma(-sdg, cz[e], bv[e]));
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      out[e] = fx_to_float(res[e]);
      if (NORM) rr = fma(res[e], res[e], rr);
    }
    *reinterpret_cast<float4*>(r + rbase + x0) = make_float4(out[0], out[1], out[2], out[3]);
  }
  if (NORM) {
    rr = block_sum(rr);
    if (threadIdx.x == 0) atomicAdd(norm2, rr);
  }
}

// FP32 -> FP64 (exact) by integer operations for normal values; zero,
// subnormal and non-finite values through the conversion instruction.
__device__ __forceinline__ double fx_widen(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xffu;
  if (ex == 0u || ex == 0xffu) return (double)f;
  return __longlong_as_double((long long)(((unsigned long long)(u & 0x80000000u) << 32) |
                                          ((unsigned long long)(ex - 127u + 1023u) << 52) |
                                          ((unsigned long long)(u & 0x7fffffu) << 29)));
}
__device__ __forceinline__ double fx_widen(double f) { return f; }

// z += d: one FP64 add per unknown (the widening of an FP32 d is done by
// integer operations, off GB300's narrow FP64 pipe).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_outer_update_v4(long long n4, double* __restrict__ z,
                                                           const T* __restrict__ d) {
  pdl_enter();
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n4) return;
  double2 a = *reinterpret_cast<double2*>(z + 4 * q);
  double2 c = *reinterpret_cast<double2*>(z + 4 * q + 2);
  a.x += fx_widen(d[4 * q]);
  a.y += fx_widen(d[4 * q + 1]);
  c.x += fx_widen(d[4 * q + 2]);
  c.y += fx_widen(d[4 * q + 3]);
  *reinterpret_cast<double2*>(z + 4 * q) = a;
  *reinterpret_cast<double2*>(z + 4 * q + 2) = c;
}

// Load policies for the per-site functions below: LdNC reads through the
// read-only path (data no block of the launch writes), LdCG reads from L2
// only (data written by other blocks of the same launch before a grid
// barrier, which another SM's L1 may hold stale), LdPlain is a plain load.
struct LdNC {
  template <typename T>
  __device__ __forceinline__ static T ld(const T* p) { return __ldg(p); }
};
struct LdCG {
  template <typename T>
  __device__ __forceinline__ static T ld(const T* p) { return __ldcg(p); }
};
struct LdPlain {
  template <typename T>
  __device__ __forceinline__ static T ld(const T* p) { return *p; }
};

// 8 consecutive values (16-byte aligned); CG: from L2 only (data that other
// blocks of the same launch wrote before a grid barrier).
template <typename T, bool CG>
__device__ __forceinline__ void ldv8(const T* p, T o[8]) {
  if constexpr (!CG) {
    Vec<T>::load8(p, o);
  } else if constexpr (sizeof(T) == 4) {
    const float4 a = __ldcg(reinterpret_cast<const float4*>(p)), c = __ldcg(reinterpret_cast<const float4*>(p + 4));
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = c.x; o[5] = c.y; o[6] = c.z; o[7] = c.w;
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double2 a = __ldcg(reinterpret_cast<const double2*>(p + 2 * q));
      o[2 * q] = a.x;
      o[2 * q + 1] = a.y;
    }
  }
}
template <typename T, bool CG>
__device__ __forceinline__ T ld1(const T* p) {
  if constexpr (CG) return __ldcg(p);
  return *p;
}

// Row k of a Galerkin operator applied to vc (one component's field) in the
// separable form of the stencil,
//   sum_dz (s Mz)_dz (w1 . v_plane(k+dz)) + (s Kz)_dz (w2 . v_plane(k+dz)),
// with w1 = Kx(x)My + Mx(x)Ky and w2 = Mx(x)My on the periodic x/y axes.
// CENTRE == false leaves out the diagonal term.
// Separable x/y weights in the kernel's precision (read by value: the level
// descriptor is a by-value kernel parameter).
template <typename T>
__device__ __forceinline__ T sep_w1(const CompDev& c, int q);
template <>
__device__ __forceinline__ float sep_w1<float>(const CompDev& c, int q) {
  return c.w1f[q];
}
template <>
__device__ __forceinline__ double sep_w1<double>(const CompDev& c, int q) {
  return c.w1[q];
}
template <typename T>
__device__ __forceinline__ T sep_w2(const CompDev& c, int q);
template <>
__device__ __forceinline__ float sep_w2<float>(const CompDev& c, int q) {
  return c.w2f[q];
}
template <>
__device__ __forceinline__ double sep_w2<double>(const CompDev& c, int q) {
  return c.w2[q];
}

template <typename T, typename LD, bool CENTRE>
__device__ __forceinline__ T sep_apply(const CompDev& c, const T* vc, int i, int j, int k) {
  const int nx = c.nx, ny = c.ny, nz = c.nz;
  const int xm = i == 0 ? nx - 1 : i - 1, xp = i == nx - 1 ? 0 : i + 1;
  const int jm = j == 0 ? ny - 1 : j - 1, jp = j == ny - 1 ? 0 : j + 1;
  const T* zb = (sizeof(T) == 4 ? (const T*)c.zb32 : (const T*)c.zb64) + k * 10;
  T w1[9], w2[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    w1[q] = sep_w1<T>(c, q);
    w2[q] = sep_w2<T>(c, q);
  }
  // Planes beyond a wall carry zero band weights (a Galerkin band row has no
  // entry outside the level): their loads are clamped to a valid plane and
  // multiplied by 0, so all 45 loads are issued without a branch between
  // planes and overlap in one round trip.
  T acc = (T)0;
#pragma unroll
  for (int dz = -2; dz <= 2; ++dz) {
    const int kk = min(max(k + dz, 0), nz - 1);
    const T* vp = vc + kk * ny * nx;
    T p1, p2;
    if (ny == 1) {
      const T a = LD::ld(vp + xm), cc = LD::ld(vp + xp);
      p1 = w1[3] * a + w1[5] * cc;
      p2 = w2[3] * a + w2[5] * cc;
      if (CENTRE || dz != 0) {
        const T bb = LD::ld(vp + i);
        p1 += w1[4] * bb;
        p2 += w2[4] * bb;
      }
    } else {
      const T* r0 = vp + jm * nx;
      const T* r1 = vp + j * nx;
      const T* r2 = vp + jp * nx;
      const T a0 = LD::ld(r0 + xm), b0 = LD::ld(r0 + i), c0 = LD::ld(r0 + xp);
      const T a1 = LD::ld(r1 + xm), c1 = LD::ld(r1 + xp);
      const T a2 = LD::ld(r2 + xm), b2 = LD::ld(r2 + i), c2 = LD::ld(r2 + xp);
      p1 = w1[0] * a0 + w1[1] * b0 + w1[2] * c0 + w1[3] * a1 + w1[5] * c1 + w1[6] * a2 + w1[7] * b2 + w1[8] * c2;
      p2 = w2[0] * a0 + w2[1] * b0 + w2[2] * c0 + w2[3] * a1 + w2[5] * c1 + w2[6] * a2 + w2[7] * b2 + w2[8] * c2;
      if (CENTRE || dz != 0) {
        const T b1 = LD::ld(r1 + i);
        p1 += w1[4] * b1;
        p2 += w2[4] * b1;
      }
    }
    acc += zb[dz + 2] * p1 + zb[5 + dz + 2] * p2;
  }
  return acc;
}

// t = b - A v on W consecutive x sites [x0, x0 + W) of row j, z rows
// [k0, k1), of one component of a Galerkin level (vc, bc, tc: the
// component's fields).  The x-y partial sums w1 * v and w2 * v of each plane
// are computed once and kept in registers for the five rows that read it;
// each row then combines them with its z bands.  Per row the arithmetic and
// order are sep_apply<CENTRE = true>'s (a plane beyond a wall contributes 0).
template <typename T, int W, typename LD>
__device__ __forceinline__ void galerkin_residual_seg(const CompDev& c, const T* vc, const T* bc, T* tc, int j, int x0,
                                                      int k0, int k1) {
  const int nx = c.nx, ny = c.ny, nz = c.nz;
  const int jm = j == 0 ? ny - 1 : j - 1, jp = j == ny - 1 ? 0 : j + 1;
  const T* zbt = sizeof(T) == 4 ? (const T*)c.zb32 : (const T*)c.zb64;
  T w1[9], w2[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    w1[q] = sep_w1<T>(c, q);
    w2[q] = sep_w2<T>(c, q);
  }
  int xs[W + 2];
#pragma unroll
  for (int e = 0; e < W + 2; ++e) {
    const int x = x0 - 1 + e;
    xs[e] = x < 0 ? x + nx : (x >= nx ? x - nx : x);
  }
  T P1[5][W], P2[5][W];
  auto sums = [&](int kk, T* p1, T* p2) {
    if (kk < 0 || kk >= nz) {
#pragma unroll
      for (int e = 0; e < W; ++e) p1[e] = p2[e] = (T)0;
      return;
    }
    const T* vp = vc + (long long)kk * ny * nx;
    if (ny == 1) {
      T r[W + 2];
#pragma unroll
      for (int e = 0; e < W + 2; ++e) r[e] = LD::ld(vp + xs[e]);
#pragma unroll
      for (int e = 0; e < W; ++e) {
        p1[e] = w1[3] * r[e] + w1[5] * r[e + 2];
        p2[e] = w2[3] * r[e] + w2[5] * r[e + 2];
        p1[e] += w1[4] * r[e + 1];
        p2[e] += w2[4] * r[e + 1];
      }
      return;
    }
    T r0[W + 2], r1[W + 2], r2[W + 2];
    const T* q0 = vp + (long long)jm * nx;
    const T* q1 = vp + (long long)j * nx;
    const T* q2 = vp + (long long)jp * nx;
#pragma unroll
    for (int e = 0; e < W + 2; ++e) {
      r0[e] = LD::ld(q0 + xs[e]);
      r1[e] = LD::ld(q1 + xs[e]);
      r2[e] = LD::ld(q2 + xs[e]);
    }
#pragma unroll
    for (int e = 0; e < W; ++e) {
      p1[e] = w1[0] * r0[e] + w1[1] * r0[e + 1] + w1[2] * r0[e + 2] + w1[3] * r1[e] + w1[5] * r1[e + 2] +
              w1[6] * r2[e] + w1[7] * r2[e + 1] + w1[8] * r2[e + 2];
      p2[e] = w2[0] * r0[e] + w2[1] * r0[e + 1] + w2[2] * r0[e + 2] + w2[3] * r1[e] + w2[5] * r1[e + 2] +
              w2[6] * r2[e] + w2[7] * r2[e + 1] + w2[8] * r2[e + 2];
      p1[e] += w1[4] * r1[e + 1];
      p2[e] += w2[4] * r1[e + 1];
    }
  };
#pragma unroll
  for (int d = 0; d < 4; ++d) sums(k0 - 2 + d, P1[d], P2[d]);
  for (int k = k0; k < k1; ++k) {
    sums(k + 2, P1[4], P2[4]);
    const T* zb = zbt + k * 10;
    const long long row = ((long long)k * ny + j) * nx + x0;
#pragma unroll
    for (int e = 0; e < W; ++e) {
      T acc = (T)0;
#pragma unroll
      for (int d = 0; d < 5; ++d) acc += zb[d] * P1[d][e] + zb[5 + d] * P2[d][e];
      tc[row + e] = LD::ld(bc + row + e) - acc;
    }
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
      for (int e = 0; e < W; ++e) {
        P1[d][e] = P1[d + 1][e];
        P2[d][e] = P2[d + 1][e];
      }
  }
}

// Heat-bath update of site g of a Galerkin colour pass (g runs over the
// class sites of all components, component ci from cp.gstart):
// v_i = (b_i - sum_{j != i} A_ij v_j) / A_ii + n / sqrt(A_ii).  The four
// sites of a noise group each recompute the group's Philox block and keep
// their own lane.  Neighbours are of other colours.
template <typename T, bool NOISE, typename LD>
__device__ __forceinline__ void coarse_site_at(const LevelDev& L, const ColourPass& cp, T* v, const T* b, int sweep,
                                               Key key, unsigned long long cy, long long g) {
  const int ci = comp_of(cp.gstart, L.ncomp, g);
  const CompDev& c = L.c[ci];
  const unsigned rank = (unsigned)(g - cp.gstart[ci]);
  const unsigned nxc = (unsigned)cp.nxc[ci], nyc = (unsigned)cp.nyc[ci];
  const unsigned t = rank / nxc;
  const int i = cp.cx[ci] + c.mx * (int)(rank - t * nxc);
  const int j = cp.cy[ci] + c.my * (int)(t % nyc);
  const int k = cp.cz[ci] + c.mz * (int)(t / nyc);
  const T off = sep_apply<T, LD, false>(c, v + c.off, i, j, k);
  const T diag = coarse_diag<T>(c, k);
  const long long idx = c.off + (long long)((k * c.ny + j) * c.nx + i);
  T nv = (LD::ld(b + idx) - off) / diag;
  if (NOISE) {
    T nn;
    normal_of(philox10(make_uint4(rank >> 2, ctr1_of(L.level, c.comp_id, cp.colour_id[ci], sweep, 0), (uint32_t)cy,
                                  (uint32_t)(cy >> 32)),
                       key.k0, key.k1),
              (int)(rank & 3), &nn);
    nv += nn / tsqrt(diag);
  }
  v[idx] = nv;
}

// Row k of a banded red-black level in its 7-point form: x-y weight a_k
// (the z band's mass entry), z coefficients below / above (the stiffness band's
// off-diagonal entries), diagonal from the tabulated stencil.  The level's x-y
// weights w1 (5-point) and w2 (centre only) complete the row.
template <typename T>
struct Band7 {
  T a, dn, up, diag;
};

template <typename T>
__device__ __forceinline__ Band7<T> band7_row(const CompDev& c, int k) {
  const T* zb = (sizeof(T) == 4 ? (const T*)c.zb32 : (const T*)c.zb64) + k * 10;
  const T w2c = sep_w2<T>(c, 4);
  Band7<T> r;
  r.a = zb[2];
  r.dn = zb[6] * w2c;
  r.up = zb[8] * w2c;
  r.diag = coarse_diag<T>(c, k);
  return r;
}

// Work items of a z-marching pass: per component ny * (nx / 8) columns times
// ceil(nz / kc) chunks of kc rows.
struct ColumnPass {
  long long start[kMaxComps + 1];
  int kc;
};

// Red-black colour pass of a banded 7-point level, marching along z: one
// thread per (component, y row, 8-wide x segment, chunk of kc z rows).  The
// z neighbours of row k come from registers (row k-1 after its update: its
// sites of the other colour, the ones row k reads, are unchanged by the
// pass), and the next row's loads are issued before the current row is
// computed (two rows of loads in flight).  Values read across threads are
// always of the other colour, which no thread writes in the pass; the
// vector loads also carry same-colour lanes, which are not used.
// Blocks per SM the z-marching colour passes are compiled for (register
// budget 65536 / (256 x this)): more resident warps keep more row loads in
// flight.
#ifndef SELM_ZM_MIN_BLOCKS
#define SELM_ZM_MIN_BLOCKS 3
#endif

template <typename T, bool NOISE>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? SELM_ZM_MIN_BLOCKS : 1) k_band7_rb_zm(LevelDev L, ColumnPass cp, T* __restrict__ v,
                                                       const T* __restrict__ b, int colour, int sweep, Key key,
                                                       const unsigned long long* __restrict__ cyc) {
  pdl_enter();
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= cp.start[L.ncomp]) return;
  int ci = 0;
  while (ci + 1 < L.ncomp && g >= cp.start[ci + 1]) ++ci;
  const CompDev& c = L.c[ci];
  const int nx = c.nx, ny = c.ny, nz = c.nz, segs = nx >> 3;
  const long long item = g - cp.start[ci];
  const long long col = item % ((long long)ny * segs);
  const int chunk = (int)(item / ((long long)ny * segs));
  const int j = (int)(col / segs), seg = (int)(col - (long long)j * segs);
  const int k0 = chunk * cp.kc, k1 = min(k0 + cp.kc, nz);
  const long long plane = (long long)nx * ny;
  const int x0 = seg << 3;
  const long long base = c.off + (long long)j * nx + x0;   // (k = 0, j, x0)
  const long long ym0 = c.off + (long long)(j == 0 ? ny - 1 : j - 1) * nx + x0;
  const long long yp0 = c.off + (long long)(j == ny - 1 ? 0 : j + 1) * nx + x0;
  const long long rowx = c.off + (long long)j * nx;
  const int xl_i = x0 == 0 ? nx - 1 : x0 - 1, xr_i = x0 + 8 == nx ? 0 : x0 + 8;
  const T wxm = sep_w1<T>(c, 3), wxp = sep_w1<T>(c, 5), wym = sep_w1<T>(c, 1), wyp = sep_w1<T>(c, 7);
  const unsigned long long cy = NOISE ? *cyc : 0ull;
  const uint32_t c1 = ctr1_of(L.level, c.comp_id, colour, sweep, 0);
  T prev[8], cur[8], nxt[8], bb[8], ty[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) prev[e] = (T)0;
  if (k0 > 0) Vec<T>::load8(v + base + (long long)(k0 - 1) * plane, prev);
  Vec<T>::load8(v + base + (long long)k0 * plane, cur);
  for (int k = k0; k < k1; ++k) {
    const long long kp = (long long)k * plane;
    if (k + 1 < nz)
      Vec<T>::load8(v + base + kp + plane, nxt);
    else {
#pragma unroll
      for (int e = 0; e < 8; ++e) nxt[e] = (T)0;
    }
    Vec<T>::load8(b + base + kp, bb);
    const Band7<T> R = band7_row<T>(c, k);
    T acc[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[e] = (k > 0 ? R.dn * prev[e] : (T)0) + (k + 1 < nz ? R.up * nxt[e] : (T)0);
    if (ny > 1) {
      Vec<T>::load8(v + ym0 + kp, ty);
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[e] += R.a * wym * ty[e];
      Vec<T>::load8(v + yp0 + kp, ty);
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[e] += R.a * wyp * ty[e];
    }
    const T left = v[rowx + kp + xl_i], right = v[rowx + kp + xr_i];
    T n4[4] = {(T)0, (T)0, (T)0, (T)0};
    if (NOISE) {
      const uint32_t grp = (uint32_t)((long long)k * ny + j) * (uint32_t)segs + (uint32_t)seg;
      Normals<T>::get(philox4x32_10(make_uint4(grp, c1, (uint32_t)cy, (uint32_t)(cy >> 32)), key.k0, key.k1), n4);
    }
    const T rsd = NOISE ? (T)1 / tsqrt(R.diag) : (T)0;
    const T rdiag = (T)1 / R.diag;   // one division per row instead of one per site
    const int par = (j + k + colour) & 1;
#pragma unroll
    for (int l = 0; l < 4; ++l) {
#pragma unroll
      for (int pp = 0; pp < 2; ++pp) {
        if (pp != par) continue;
        const int e = 2 * l + pp;
        const T xl = e == 0 ? left : cur[e - 1];
        const T xr = e == 7 ? right : cur[e + 1];
        T nv = (bb[e] - (acc[e] + R.a * (wxm * xl + wxp * xr))) * rdiag;
        if (NOISE) nv += n4[l] * rsd;
        cur[e] = nv;
      }
    }
    Vec<T>::store8(v + base + kp, cur);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      prev[e] = cur[e];
      cur[e] = nxt[e];
    }
  }
}

// t = b - A v on a Galerkin level (levels >= 1, not banded red-black; nx % 4
// == 0): one thread per (component, y row, 4-wide x segment, chunk of kc z
// rows), galerkin_residual_seg's separable form.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_galerkin_residual_zm(LevelDev L, ColumnPass cp, const T* __restrict__ v,
                                                                const T* __restrict__ b, T* __restrict__ t) {
  pdl_enter();
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= cp.start[L.ncomp]) return;
  int ci = 0;
  while (ci + 1 < L.ncomp && g >= cp.start[ci + 1]) ++ci;
  const CompDev& c = L.c[ci];
  const int segs = c.nx >> 2;
  const long long item = g - cp.start[ci];
  const long long col = item % ((long long)c.ny * segs);
  const int chunk = (int)(item / ((long long)c.ny * segs));
  const int j = (int)(col / segs), seg = (int)(col - (long long)j * segs);
  const int k0 = chunk * cp.kc, k1 = min(k0 + cp.kc, c.nz);
  galerkin_residual_seg<T, 4, LdPlain>(c, v + c.off, b + c.off, t + c.off, j, seg << 2, k0, k1);
}

// Level-0 red-black colour pass marching along z: one thread per (component,
// y row, 8-wide x segment, chunk of kc z rows); one Philox block per segment
// and row gives the normals of its four sites of the colour.  Row k's z
// neighbours come from registers (row k-1 after this thread's update of it:
// its sites of the other colour, the ones row k reads, are not written by the
// pass) and the next row's loads are issued before the current row is
// computed.
template <typename T, bool NOISE, bool CG>
__device__ __forceinline__ void fine_colour_zm_item(const LevelDev& L, const ColumnPass& cp, T* __restrict__ v,
                                                    const T* __restrict__ b, int colour, int sweep, Key key,
                                                    unsigned long long cy, long long g) {
  if (g >= cp.start[L.ncomp]) return;
  int ci = 0;
  while (ci + 1 < L.ncomp && g >= cp.start[ci + 1]) ++ci;
  const CompDev& c = L.c[ci];
  const int nx = c.nx, ny = c.ny, nz = c.nz, segs = nx >> 3;
  const long long item = g - cp.start[ci];
  const long long col = item % ((long long)ny * segs);
  const int chunk = (int)(item / ((long long)ny * segs));
  const int j = (int)(col / segs), seg = (int)(col - (long long)j * segs);
  const int k0 = chunk * cp.kc, k1 = min(k0 + cp.kc, nz);
  const long long plane = (long long)nx * ny;
  const int x0 = seg << 3;
  const long long base = c.off + (long long)j * nx + x0;
  const long long ym0 = c.off + (long long)(j == 0 ? ny - 1 : j - 1) * nx + x0;
  const long long yp0 = c.off + (long long)(j == ny - 1 ? 0 : j + 1) * nx + x0;
  const long long rowx = c.off + (long long)j * nx;
  const int xl_i = x0 == 0 ? nx - 1 : x0 - 1, xr_i = x0 + 8 == nx ? 0 : x0 + 8;
  const uint32_t c1 = ctr1_of(L.level, c.comp_id, colour, sweep, 0);
  const T s = (T)c.s;
  T prev[8], cur[8], nxt[8], bb[8], ty[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) prev[e] = (T)0;
  if (k0 > 0) ldv8<T, CG>(v + base + (long long)(k0 - 1) * plane, prev);
  ldv8<T, CG>(v + base + (long long)k0 * plane, cur);
  for (int k = k0; k < k1; ++k) {
    const long long kp = (long long)k * plane;
    if (k + 1 < nz)
      ldv8<T, CG>(v + base + kp + plane, nxt);
    else {
#pragma unroll
      for (int e = 0; e < 8; ++e) nxt[e] = (T)0;
    }
    ldv8<T, CG>(b + base + kp, bb);
    // neighbour sums: y-, y+, z-, z+
    T acc[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[e] = (T)0;
    if (ny > 1) {
      ldv8<T, CG>(v + ym0 + kp, ty);
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[e] += ty[e];
      ldv8<T, CG>(v + yp0 + kp, ty);
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[e] += ty[e];
    }
    if (k > 0) {
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[e] += prev[e];
    }
    if (k + 1 < nz) {
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[e] += nxt[e];
    }
    const T left = ld1<T, CG>(v + rowx + kp + xl_i), right = ld1<T, CG>(v + rowx + kp + xr_i);
    T n4[4] = {(T)0, (T)0, (T)0, (T)0};
    if (NOISE) {
      const uint32_t grp = (uint32_t)((long long)k * ny + j) * (uint32_t)segs + (uint32_t)seg;
      Normals<T>::get(philox10(make_uint4(grp, c1, (uint32_t)cy, (uint32_t)(cy >> 32)), key.k0, key.k1), n4);
    }
    const int edges = (k == 0) + (k == nz - 1);
    T dz = (T)2;
    if (c.zkind == kAxisCellDir) dz += (T)edges;
    if (c.zkind == kAxisCellNeu) dz -= (T)edges;
    const T diag = s * ((ny > 1 ? (T)4 : (T)2) + dz);
    const T rdiag = (T)1 / diag;   // one division per row instead of one per site
    const T rsd = NOISE ? (T)1 / tsqrt(diag) : (T)0;
    if (((j + k + colour) & 1) == 0)
      fine_update8<T, NOISE, 0>(cur, bb, acc, left, right, n4, s, rdiag, rsd);
    else
      fine_update8<T, NOISE, 1>(cur, bb, acc, left, right, n4, s, rdiag, rsd);
    Vec<T>::store8(v + base + kp, cur);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      prev[e] = cur[e];
      cur[e] = nxt[e];
    }
  }
}

template <typename T, bool NOISE>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? SELM_ZM_MIN_BLOCKS : 1) k_fine_colour_zm(LevelDev L, ColumnPass cp, T* __restrict__ v,
                                                          const T* __restrict__ b, int colour, int sweep, Key key,
                                                          const unsigned long long* __restrict__ cyc) {
  pdl_enter();
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= cp.start[L.ncomp]) return;
  fine_colour_zm_item<T, NOISE, false>(L, cp, v, b, colour, sweep, key, NOISE ? *cyc : 0ull, g);
}

// t = b - A v on level 0, marching along z like k_fine_colour_zm (every site
// of a segment): fine_row's sum order (x-, x+, y-, y+, z-, z+) and
// t = b - (-s sum + diag v).
template <typename T, bool CG>
__device__ __forceinline__ void fine_residual_zm_item(const LevelDev& L, const ColumnPass& cp, const T* __restrict__ v,
                                                      const T* __restrict__ b, T* __restrict__ t, long long g) {
  if (g >= cp.start[L.ncomp]) return;
  int ci = 0;
  while (ci + 1 < L.ncomp && g >= cp.start[ci + 1]) ++ci;
  const CompDev& c = L.c[ci];
  const int nx = c.nx, ny = c.ny, nz = c.nz, segs = nx >> 3;
  const long long item = g - cp.start[ci];
  const long long col = item % ((long long)ny * segs);
  const int chunk = (int)(item / ((long long)ny * segs));
  const int j = (int)(col / segs), seg = (int)(col - (long long)j * segs);
  const int k0 = chunk * cp.kc, k1 = min(k0 + cp.kc, nz);
  const long long plane = (long long)nx * ny;
  const int x0 = seg << 3;
  const long long base = c.off + (long long)j * nx + x0;
  const long long ym0 = c.off + (long long)(j == 0 ? ny - 1 : j - 1) * nx + x0;
  const long long yp0 = c.off + (long long)(j == ny - 1 ? 0 : j + 1) * nx + x0;
  const long long rowx = c.off + (long long)j * nx;
  const int xl_i = x0 == 0 ? nx - 1 : x0 - 1, xr_i = x0 + 8 == nx ? 0 : x0 + 8;
  const T s = (T)c.s;
  T prev[8], cur[8], nxt[8], bb[8], ty[8], sum[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) prev[e] = (T)0;
  if (k0 > 0) ldv8<T, CG>(v + base + (long long)(k0 - 1) * plane, prev);
  ldv8<T, CG>(v + base + (long long)k0 * plane, cur);
  for (int k = k0; k < k1; ++k) {
    const long long kp = (long long)k * plane;
    if (k + 1 < nz)
      ldv8<T, CG>(v + base + kp + plane, nxt);
    else {
#pragma unroll
      for (int e = 0; e < 8; ++e) nxt[e] = (T)0;
    }
    ldv8<T, CG>(b + base + kp, bb);
    const T left = ld1<T, CG>(v + rowx + kp + xl_i), right = ld1<T, CG>(v + rowx + kp + xr_i);
#pragma unroll
    for (int e = 0; e < 8; ++e) sum[e] = (e == 0 ? left : cur[e - 1]) + (e == 7 ? right : cur[e + 1]);
    if (ny > 1) {
      ldv8<T, CG>(v + ym0 + kp, ty);
#pragma unroll
      for (int e = 0; e < 8; ++e) sum[e] += ty[e];
      ldv8<T, CG>(v + yp0 + kp, ty);
#pragma unroll
      for (int e = 0; e < 8; ++e) sum[e] += ty[e];
    }
    if (k > 0) {
#pragma unroll
      for (int e = 0; e < 8; ++e) sum[e] += prev[e];
    }
    if (k + 1 < nz) {
#pragma unroll
      for (int e = 0; e < 8; ++e) sum[e] += nxt[e];
    }
    const int edges = (k == 0) + (k == nz - 1);
    T dz = (T)2;
    if (c.zkind == kAxisCellDir) dz += (T)edges;
    if (c.zkind == kAxisCellNeu) dz -= (T)edges;
    const T diag = s * ((ny > 1 ? (T)4 : (T)2) + dz);
    T out[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) out[e] = bb[e] - (-s * sum[e] + diag * cur[e]);
    Vec<T>::store8(t + base + kp, out);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      prev[e] = cur[e];
      cur[e] = nxt[e];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_fine_residual_zm(LevelDev L, ColumnPass cp, const T* __restrict__ v,
                                                            const T* __restrict__ b, T* __restrict__ t) {
  pdl_enter();
  fine_residual_zm_item<T, false>(L, cp, v, b, t, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// t = b - A v on a banded 7-point level, marching along z like
// k_band7_rb_zm (every site of a segment, no colour).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_band7_residual_zm(LevelDev L, ColumnPass cp, const T* __restrict__ v,
                                                             const T* __restrict__ b, T* __restrict__ t) {
  pdl_enter();
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= cp.start[L.ncomp]) return;
  int ci = 0;
  while (ci + 1 < L.ncomp && g >= cp.start[ci + 1]) ++ci;
  const CompDev& c = L.c[ci];
  const int nx = c.nx, ny = c.ny, nz = c.nz, segs = nx >> 3;
  const long long item = g - cp.start[ci];
  const long long col = item % ((long long)ny * segs);
  const int chunk = (int)(item / ((long long)ny * segs));
  const int j = (int)(col / segs), seg = (int)(col - (long long)j * segs);
  const int k0 = chunk * cp.kc, k1 = min(k0 + cp.kc, nz);
  const long long plane = (long long)nx * ny;
  const int x0 = seg << 3;
  const long long base = c.off + (long long)j * nx + x0;
  const long long ym0 = c.off + (long long)(j == 0 ? ny - 1 : j - 1) * nx + x0;
  const long long yp0 = c.off + (long long)(j == ny - 1 ? 0 : j + 1) * nx + x0;
  const long long rowx = c.off + (long long)j * nx;
  const int xl_i = x0 == 0 ? nx - 1 : x0 - 1, xr_i = x0 + 8 == nx ? 0 : x0 + 8;
  const T wxm = sep_w1<T>(c, 3), wxp = sep_w1<T>(c, 5), wym = sep_w1<T>(c, 1), wyp = sep_w1<T>(c, 7);
  T prev[8], cur[8], nxt[8], bb[8], ty[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) prev[e] = (T)0;
  if (k0 > 0) Vec<T>::load8(v + base + (long long)(k0 - 1) * plane, prev);
  Vec<T>::load8(v + base + (long long)k0 * plane, cur);
  for (int k = k0; k < k1; ++k) {
    const long long kp = (long long)k * plane;
    if (k + 1 < nz)
      Vec<T>::load8(v + base + kp + plane, nxt);
    else {
#pragma unroll
      for (int e = 0; e < 8; ++e) nxt[e] = (T)0;
    }
    Vec<T>::load8(b + base + kp, bb);
    const Band7<T> R = band7_row<T>(c, k);
    T acc[8];
#pragma unroll
    for (int e = 0; e < 8; ++e)
      acc[e] = R.diag * cur[e] + (k > 0 ? R.dn * prev[e] : (T)0) + (k + 1 < nz ? R.up * nxt[e] : (T)0);
    if (ny > 1) {
      Vec<T>::load8(v + ym0 + kp, ty);
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[e] += R.a * wym * ty[e];
      Vec<T>::load8(v + yp0 + kp, ty);
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[e] += R.a * wyp * ty[e];
    }
    const T left = v[rowx + kp + xl_i], right = v[rowx + kp + xr_i];
    T out[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const T xl = e == 0 ? left : cur[e - 1];
      const T xr = e == 7 ? right : cur[e + 1];
      out[e] = bb[e] - (acc[e] + R.a * (wxm * xl + wxp * xr));
    }
    Vec<T>::store8(t + base + kp, out);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      prev[e] = cur[e];
      cur[e] = nxt[e];
    }
  }
}

// A banded (Galerkin-form) level whose operator is the 7-point stencil (the
// composite base grid), smoothed in red-black order like level 0: colour =
// (i + j + k) mod 2, rank = (k ny + j) nx/2 + i/2 within the colour, one
// thread per site.  The row uses the level's separable stencil tables.
template <typename T, bool NOISE>
__global__ void __launch_bounds__(kBlock) k_band_rb(LevelDev L, ColourPass cp, T* __restrict__ v,
                                                   const T* __restrict__ b, int colour, int sweep, Key key,
                                                   const unsigned long long* __restrict__ cyc) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= cp.gstart[L.ncomp]) return;
  const int ci = comp_of(cp.gstart, L.ncomp, g);
  const CompDev& c = L.c[ci];
  const unsigned rank = (unsigned)(g - cp.gstart[ci]);
  const unsigned hx = (unsigned)(c.nx >> 1);
  const unsigned t = rank / hx;
  const int j = (int)(t % (unsigned)c.ny), k = (int)(t / (unsigned)c.ny);
  const int i = 2 * (int)(rank - t * hx) + ((j + k + colour) & 1);
  const T off = sep_apply<T, LdNC, false>(c, v + c.off, i, j, k);
  const T diag = coarse_diag<T>(c, k);
  const long long idx = c.off + (long long)((k * c.ny + j) * c.nx + i);
  T nv = (__ldg(b + idx) - off) / diag;
  if (NOISE) {
    const unsigned long long cy = *cyc;
    T nn;
    normal_of(philox10(make_uint4(rank >> 2, ctr1_of(L.level, c.comp_id, colour, sweep, 0), (uint32_t)cy,
                                  (uint32_t)(cy >> 32)),
                       key.k0, key.k1),
              (int)(rank & 3), &nn);
    nv += nn / tsqrt(diag);
  }
  v[idx] = nv;
}

// Galerkin levels, one thread per site of the colour class.
template <typename T, bool NOISE>
__global__ void __launch_bounds__(kBlock) k_coarse_site(LevelDev L, ColourPass cp, T* __restrict__ v,
                                                       const T* __restrict__ b, int sweep, Key key,
                                                       const unsigned long long* __restrict__ cyc) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= cp.gstart[L.ncomp]) return;
  coarse_site_at<T, NOISE, LdNC>(L, cp, v, b, sweep, key, NOISE ? *cyc : 0ull, g);
}

// One colour pass of a Galerkin level with 8-wide rows (nx % 8 == 0, x
// modulus 2): one thread per (component, class row, class plane, 8-wide x
// segment) updates the segment's four class sites x = x0 + CX + 2e, which are
// one Philox group (ranks 4s .. 4s + 3).  The 15 rows of the window are read
// as 8-wide vectors plus their two edge values; per site the arithmetic and
// order are coarse_site_at's.  Every value used is of another colour (rows
// j +- 1 and planes k +- 1, +- 2 belong to other classes, and in row j only
// x +- 1 are read), so in-place updates are safe.  sp.start: first item of
// each component.
template <typename T, bool NOISE, int CX, bool CG>
__device__ __forceinline__ void coarse_colour_v8_item(const LevelDev& L, const ColourPass& cp, const ColumnPass& sp,
                                                      T* __restrict__ v, const T* __restrict__ b, int sweep, Key key,
                                                      unsigned long long cy, long long g) {
  if (g >= sp.start[L.ncomp]) return;
  int ci = 0;
  while (ci + 1 < L.ncomp && g >= sp.start[ci + 1]) ++ci;
  const CompDev& c = L.c[ci];
  const int nx = c.nx, ny = c.ny, nz = c.nz, segs = nx >> 3;
  const long long item = g - sp.start[ci];
  const int seg = (int)(item % segs);
  const long long t = item / segs;
  const int jj = (int)(t % cp.nyc[ci]), kk = (int)(t / cp.nyc[ci]);
  const int j = cp.cy[ci] + c.my * jj, k = cp.cz[ci] + c.mz * kk;
  const int x0 = seg << 3;
  const int jm = j == 0 ? ny - 1 : j - 1, jp = j == ny - 1 ? 0 : j + 1;
  const int xl = x0 == 0 ? nx - 1 : x0 - 1, xr = x0 + 8 == nx ? 0 : x0 + 8;
  const T* vc = v + c.off;
  const T* zb = (sizeof(T) == 4 ? (const T*)c.zb32 : (const T*)c.zb64) + k * 10;
  T w1[9], w2[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    w1[q] = sep_w1<T>(c, q);
    w2[q] = sep_w2<T>(c, q);
  }
  auto row = [&](const T* rp, T r[10]) {
    if constexpr (CG) {
      r[0] = __ldcg(rp + xl);
      ldv8<T, true>(rp + x0, r + 1);
      r[9] = __ldcg(rp + xr);
    } else {
      r[0] = LdNC::ld(rp + xl);
      Vec<T>::load8(rp + x0, r + 1);
      r[9] = LdNC::ld(rp + xr);
    }
  };
  T acc[4] = {(T)0, (T)0, (T)0, (T)0};
#pragma unroll
  for (int dz = -2; dz <= 2; ++dz) {
    const T* vp = vc + (long long)min(max(k + dz, 0), nz - 1) * ny * nx;
    T r0[10], r1[10], r2[10];
    row(vp + (long long)j * nx, r1);
    if (ny > 1) {
      row(vp + (long long)jm * nx, r0);
      row(vp + (long long)jp * nx, r2);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int x = CX + 2 * e;   // r[x], r[x + 1], r[x + 2] hold x0 + x - 1 .. x0 + x + 1
      T p1, p2;
      if (ny == 1) {
        p1 = w1[3] * r1[x] + w1[5] * r1[x + 2];
        p2 = w2[3] * r1[x] + w2[5] * r1[x + 2];
      } else {
        p1 = w1[0] * r0[x] + w1[1] * r0[x + 1] + w1[2] * r0[x + 2] + w1[3] * r1[x] + w1[5] * r1[x + 2] +
             w1[6] * r2[x] + w1[7] * r2[x + 1] + w1[8] * r2[x + 2];
        p2 = w2[0] * r0[x] + w2[1] * r0[x + 1] + w2[2] * r0[x + 2] + w2[3] * r1[x] + w2[5] * r1[x + 2] +
             w2[6] * r2[x] + w2[7] * r2[x + 1] + w2[8] * r2[x + 2];
      }
      if (dz != 0) {
        p1 += w1[4] * r1[x + 1];
        p2 += w2[4] * r1[x + 1];
      }
      acc[e] += zb[dz + 2] * p1 + zb[5 + dz + 2] * p2;
    }
  }
  const T diag = coarse_diag<T>(c, k);
  T n4[4] = {(T)0, (T)0, (T)0, (T)0};
  if (NOISE) {
    const unsigned grp = (unsigned)seg + (unsigned)(cp.nxc[ci] >> 2) * (unsigned)(jj + cp.nyc[ci] * kk);
    Normals<T>::get(philox10(make_uint4(grp, ctr1_of(L.level, c.comp_id, cp.colour_id[ci], sweep, 0), (uint32_t)cy,
                                        (uint32_t)(cy >> 32)),
                             key.k0, key.k1),
                    n4);
  }
  const long long rowi = c.off + ((long long)k * ny + j) * nx + x0 + CX;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    T nv = ((CG ? __ldcg(b + rowi + 2 * e) : LdNC::ld(b + rowi + 2 * e)) - acc[e]) / diag;
    if (NOISE) nv += n4[e] / tsqrt(diag);
    v[rowi + 2 * e] = nv;
  }
}

template <typename T, bool NOISE, int CX>
__global__ void __launch_bounds__(kBlock) k_coarse_colour_v8(LevelDev L, ColourPass cp, ColumnPass sp,
                                                            T* __restrict__ v, const T* __restrict__ b, int sweep,
                                                            Key key, const unsigned long long* __restrict__ cyc) {
  pdl_enter();
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= sp.start[L.ncomp]) return;
  coarse_colour_v8_item<T, NOISE, CX, false>(L, cp, sp, v, b, sweep, key, NOISE ? *cyc : 0ull, g);
}

// ---------------------------------------------------------------------------
// Residual, restriction, prolongation
// ---------------------------------------------------------------------------
// Level fields are below 2^31 elements (checked at create), so the site
// decomposition uses 32-bit arithmetic.
__device__ __forceinline__ void site_of(const LevelDev& L, long long s, int* ci, int* i, int* j, int* k) {
  int c = 0;
  while (c + 1 < L.ncomp && s >= L.c[c + 1].off) ++c;
  const CompDev& cd = L.c[c];
  const unsigned loc = (unsigned)(s - cd.off);
  const unsigned t = loc / (unsigned)cd.nx;
  *i = (int)(loc - t * (unsigned)cd.nx);
  *j = (int)(t % (unsigned)cd.ny);
  *k = (int)(t / (unsigned)cd.ny);
  *ci = c;
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_residual(LevelDev L, const T* __restrict__ v, const T* __restrict__ b,
                                                    T* __restrict__ t) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= L.size) return;
  int ci, i, j, k;
  site_of(L, s, &ci, &i, &j, &k);
  const CompDev& c = L.c[ci];
  T Av;
  if (L.level == 0) {
    T off, diag;
    fine_row<T, T>(c, v, i, j, k, &off, &diag);
    Av = off + diag * v[s];
  } else if (L.rb) {   // banded 7-point level
    const Band7<T> R = band7_row<T>(c, k);
    const long long plane = (long long)c.nx * c.ny;
    const long long row = c.off + (long long)k * plane + (long long)j * c.nx;
    T xy = sep_w1<T>(c, 3) * v[row + wrapi(i - 1, c.nx)] + sep_w1<T>(c, 5) * v[row + wrapi(i + 1, c.nx)];
    if (c.ny > 1)
      xy += sep_w1<T>(c, 1) * v[c.off + (long long)k * plane + (long long)wrapi(j - 1, c.ny) * c.nx + i] +
            sep_w1<T>(c, 7) * v[c.off + (long long)k * plane + (long long)wrapi(j + 1, c.ny) * c.nx + i];
    Av = R.diag * v[s] + R.a * xy;
    if (k > 0) Av += R.dn * v[row - plane + i];
    if (k < c.nz - 1) Av += R.up * v[row + plane + i];
  } else {
    Av = sep_apply<T, LdPlain, true>(c, v + c.off, i, j, k);
  }
  t[s] = b[s] - Av;
}

// b_c(I,J,K) = sum_f P(f, (I,J,K)) t(f): periodic axes (1/2, 1, 1/2) around
// fine node 2I; the wall axis from the tabulated columns of P.
template <typename T, typename LD>
__device__ __forceinline__ void restrict_at(const LevelDev& Lf, const LevelDev& Lc, const T* t, T* bc, long long s) {
  int ci, I, J, K;
  site_of(Lc, s, &ci, &I, &J, &K);
  const CompDev& f = Lf.c[ci];
  const CompDev& cf = f;  // transfer tables live on the fine level
  const long long plane = (long long)f.nx * f.ny;
  T acc = (T)0;
#pragma unroll
  for (int qz = 0; qz < 4; ++qz) {
    // an unused tap (index -1) reads row 0 with weight 0: no branch between taps
    const int kr = cf.rz_idx[K * 4 + qz];
    const int kf = kr < 0 ? 0 : kr;
    const T wz = kr < 0 ? (T)0 : rz_w<T>(cf, K * 4 + qz);
    for (int qy = -1; qy <= 1; ++qy) {
      T wy;
      int jf;
      if (f.ny == 1) {
        if (qy != 0) continue;
        wy = (T)1;
        jf = 0;
      } else {
        wy = qy == 0 ? (T)1 : (T)0.5;
        jf = wrapi(2 * J + qy, f.ny);
      }
      const long long rowb = f.off + (long long)kf * plane + (long long)jf * f.nx;
#pragma unroll
      for (int qx = -1; qx <= 1; ++qx) {
        const T wx = qx == 0 ? (T)1 : (T)0.5;
        acc += wz * wy * wx * LD::ld(t + rowb + wrapi(2 * I + qx, f.nx));
      }
    }
  }
  bc[s] = acc;
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_restrict(LevelDev Lf, LevelDev Lc, const T* __restrict__ t,
                                                    T* __restrict__ bc) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < Lc.size) restrict_at<T, LdPlain>(Lf, Lc, t, bc, s);
}

// 8 consecutive values, read through L2 only (data written by other SMs
// earlier in the same launch).
template <typename T>
__device__ __forceinline__ void load8_cg(const T* p, T o[8]);
template <>
__device__ __forceinline__ void load8_cg<float>(const float* p, float o[8]) {
  const float4 a = __ldcg(reinterpret_cast<const float4*>(p)), b = __ldcg(reinterpret_cast<const float4*>(p + 4));
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
}
template <>
__device__ __forceinline__ void load8_cg<double>(const double* p, double o[8]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double2 a = __ldcg(reinterpret_cast<const double2*>(p + 2 * q));
    o[2 * q] = a.x;
    o[2 * q + 1] = a.y;
  }
}

// restrict_at for four consecutive coarse x sites (item gt: coarse row, 4-wide
// segment; fine nx % 8 == 0, the same nx in every component): each
// contributing fine row is read as one 8-wide vector (fine x 2I0 .. 2I0+7) and
// its left neighbour; the terms are added in restrict_at's order.  CG: reads
// through L2 only.
template <typename T, bool CG>
__device__ __forceinline__ void restrict_seg4(const LevelDev& Lf, const LevelDev& Lc, const RowPass& rp,
                                              const T* __restrict__ t, T* __restrict__ bc, long long gt) {
  const int segs = Lc.c[0].nx >> 2;
  const long long row_all = gt / segs;
  if (row_all >= rp.rstart[Lc.ncomp]) return;
  const int seg = (int)(gt - row_all * segs);
  int ci = 0;
  while (ci + 1 < Lc.ncomp && row_all >= rp.rstart[ci + 1]) ++ci;
  const CompDev& f = Lf.c[ci];
  const CompDev& c = Lc.c[ci];
  const int row = (int)(row_all - rp.rstart[ci]);
  const int J = row % c.ny, K = row / c.ny;
  const int I0 = seg << 2, xf0 = 2 * I0;
  const long long plane = (long long)f.nx * f.ny;
  T acc[4] = {(T)0, (T)0, (T)0, (T)0};
#pragma unroll
  for (int qz = 0; qz < 4; ++qz) {
    const int kr = f.rz_idx[K * 4 + qz];   // an unused tap reads row 0 with weight 0
    const int kf = kr < 0 ? 0 : kr;
    const T wz = kr < 0 ? (T)0 : rz_w<T>(f, K * 4 + qz);
    for (int qy = -1; qy <= 1; ++qy) {
      T wy;
      int jf;
      if (f.ny == 1) {
        if (qy != 0) continue;
        wy = (T)1;
        jf = 0;
      } else {
        wy = qy == 0 ? (T)1 : (T)0.5;
        jf = wrapi(2 * J + qy, f.ny);
      }
      const long long rowb = f.off + (long long)kf * plane + (long long)jf * f.nx;
      T r[8];
      if (CG)
        load8_cg<T>(t + rowb + xf0, r);
      else
        Vec<T>::load8(t + rowb + xf0, r);
      const T lft = CG ? __ldcg(t + rowb + wrapi(xf0 - 1, f.nx)) : t[rowb + wrapi(xf0 - 1, f.nx)];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        acc[e] += wz * wy * (T)0.5 * (e == 0 ? lft : r[2 * e - 1]);
        acc[e] += wz * wy * (T)1 * r[2 * e];
        acc[e] += wz * wy * (T)0.5 * r[2 * e + 1];
      }
    }
  }
  T* out = bc + c.off + ((long long)K * c.ny + J) * c.nx + I0;
#pragma unroll
  for (int e = 0; e < 4; ++e) out[e] = acc[e];
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_restrict_v4(LevelDev Lf, LevelDev Lc, RowPass rp, const T* __restrict__ t,
                                                       T* __restrict__ bc) {
  pdl_enter();
  restrict_seg4<T, false>(Lf, Lc, rp, t, bc, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// v_f += P v_c: periodic axes: even fine node = coarse node, odd = mean of two.
template <typename T, typename LD = LdPlain>
__device__ __forceinline__ T prolong_val(const LevelDev& Lf, const LevelDev& Lc, const T* vc, long long s) {
  int ci, i, j, k;
  site_of(Lf, s, &ci, &i, &j, &k);
  const CompDev& f = Lf.c[ci];
  const CompDev& c = Lc.c[ci];
  // fixed 2 x 2 x 2 taps: an unused one reads a valid coarse value with weight
  // 0, so the loads issue without branches (the sum is unchanged)
  const bool xo = (i & 1) != 0;
  const int xi0 = i >> 1, xi1 = xo ? wrapi((i >> 1) + 1, c.nx) : xi0;
  const T xw0 = xo ? (T)0.5 : (T)1, xw1 = xo ? (T)0.5 : (T)0;
  const bool yo = f.ny > 1 && (j & 1) != 0;
  const int yi0 = f.ny == 1 ? 0 : j >> 1, yi1 = yo ? wrapi((j >> 1) + 1, c.ny) : yi0;
  const T yw0 = yo ? (T)0.5 : (T)1, yw1 = yo ? (T)0.5 : (T)0;
  const int xi[2] = {xi0, xi1}, yi[2] = {yi0, yi1};
  const T xw[2] = {xw0, xw1}, yw[2] = {yw0, yw1};
  const long long cplane = (long long)c.nx * c.ny;
  T acc = (T)0;
#pragma unroll
  for (int qz = 0; qz < 2; ++qz) {
    const int kr = f.pz_idx[k * 2 + qz];
    const int kc = kr < 0 ? 0 : kr;
    const T wz = kr < 0 ? (T)0 : pz_w<T>(f, k * 2 + qz);
#pragma unroll
    for (int qy = 0; qy < 2; ++qy)
#pragma unroll
      for (int qx = 0; qx < 2; ++qx)
        acc += wz * yw[qy] * xw[qx] * LD::ld(vc + c.off + (long long)kc * cplane + (long long)yi[qy] * c.nx + xi[qx]);
  }
  return acc;
}

template <typename T>
__device__ __forceinline__ void prolong_at(const LevelDev& Lf, const LevelDev& Lc, T* v, const T* vc, long long s) {
  v[s] += prolong_val<T>(Lf, Lc, vc, s);
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_prolong(LevelDev Lf, LevelDev Lc, T* __restrict__ v,
                                                   const T* __restrict__ vc) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < Lf.size) prolong_at<T>(Lf, Lc, v, vc, s);
}

template <typename T>
__device__ __forceinline__ void load4(const T* p, T o[4]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) o[q] = p[q];
}
template <>
__device__ __forceinline__ void load4<float>(const float* p, float o[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  o[0] = a.x;
  o[1] = a.y;
  o[2] = a.z;
  o[3] = a.w;
}

// v_f += P v_c on one 8-wide segment of a fine row (item gt; nx % 8 == 0;
// periodic x and y with vertex coarsening, so a segment reads coarse
// x0/2 .. x0/2 + 4 of each contributing coarse row; wall axis from the
// prolongation table).  TAG0 (FP32): the results' last mantissa bit is
// cleared (update count 0 of a following dataflow-ordered smoothing).
template <typename T, bool TAG0, bool CG = false>
__device__ __forceinline__ void prolong_seg8(const LevelDev& Lf, const LevelDev& Lc, const RowPass& rp,
                                             T* __restrict__ v, const T* __restrict__ vc, long long gt) {
  const int segs = Lf.c[0].nx >> 3;
  const long long row_all = gt / segs;
  if (row_all >= rp.rstart[Lf.ncomp]) return;
  const int seg = (int)(gt - row_all * segs);
  int ci = 0;
  while (ci + 1 < Lf.ncomp && row_all >= rp.rstart[ci + 1]) ++ci;
  const CompDev& f = Lf.c[ci];
  const CompDev& c = Lc.c[ci];
  const int row = (int)(row_all - rp.rstart[ci]);
  const int j = row % f.ny, k = row / f.ny;
  const int x0 = seg << 3, cx0 = x0 >> 1;
  int yi[2] = {0, 0};
  T yw[2] = {(T)1, (T)0};
  int nyp = 1;
  if (f.ny > 1) {
    yi[0] = j >> 1;
    if (j & 1) {
      yi[1] = (j >> 1) + 1 == c.ny ? 0 : (j >> 1) + 1;
      yw[0] = yw[1] = (T)0.5;
      nyp = 2;
    }
  }
  T acc[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) acc[e] = (T)0;
  const long long cplane = (long long)c.nx * c.ny;
#pragma unroll
  for (int qz = 0; qz < 2; ++qz) {
    const int kr = f.pz_idx[k * 2 + qz];
    const int kc = kr < 0 ? 0 : kr;   // an unused tap reads row 0 with weight 0
    const T wz = kr < 0 ? (T)0 : pz_w<T>(f, k * 2 + qz);
    for (int a = 0; a < nyp; ++a) {
      const T* crow = vc + c.off + (long long)kc * cplane + (long long)yi[a] * c.nx;
      T cx[5];
      if constexpr (CG) {
#pragma unroll
        for (int q = 0; q < 4; ++q) cx[q] = __ldcg(crow + cx0 + q);
        cx[4] = __ldcg(crow + (cx0 + 4 == c.nx ? 0 : cx0 + 4));
      } else {
        load4<T>(crow + cx0, cx);
        cx[4] = crow[cx0 + 4 == c.nx ? 0 : cx0 + 4];
      }
      const T w = wz * yw[a];
#pragma unroll
      for (int e = 0; e < 8; ++e)
        acc[e] += w * ((e & 1) ? (T)0.5 * (cx[e >> 1] + cx[(e >> 1) + 1]) : cx[e >> 1]);
    }
  }
  T* out = v + f.off + (long long)row * f.nx + x0;
  T cur[8];
  ldv8<T, CG>(out, cur);
#pragma unroll
  for (int e = 0; e < 8; ++e) cur[e] += acc[e];
  if constexpr (TAG0 && sizeof(T) == 4) {
#pragma unroll
    for (int e = 0; e < 8; ++e) cur[e] = __uint_as_float(__float_as_uint(cur[e]) & ~1u);
  }
  Vec<T>::store8(out, cur);
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_prolong_v8(LevelDev Lf, LevelDev Lc, RowPass rp, T* __restrict__ v,
                                                      const T* __restrict__ vc) {
  pdl_enter();
  prolong_seg8<T, false>(Lf, Lc, rp, v, vc, (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------------
// One Galerkin level as a cooperative launch (all blocks co-resident; grid
// barriers between colour passes).  Phase 0 (descending half of the V-cycle
// at this level): mu1 sweeps from the zero start, residual t = b - A v,
// restriction b_c = P^T t and v_c = 0.  Phase 1 (ascending half):
// v += P v_c, then mu2 sweeps.  Same arithmetic, counters and order as the
// per-pass launches; the GPU-wide launch suits a level too large for one
// thread-block cluster per component yet too small to hide a launch per pass.
// ---------------------------------------------------------------------------
constexpr int kMaxCoopColours = 16;
constexpr unsigned long long kCoopWaitNs = 1000000000ull;   // 1 s bound on one barrier wait

// 512 threads of at most 64 registers: half an SM's register file, so that a
// block of the launch can share an SM with work of another stream.
template <typename T>
struct CoopThreads {
  static constexpr int value = 512;
};

template <typename T>
struct CoopLevel {
  LevelDev L, Lc;                        // this level and the next coarser one
  ColourPass cp[kMaxCoopColours];        // colour q of this level
  int ncolour;
  int flow;                              // 1: passes in dataflow order (FP32), else grid barriers
  // Dataflow order, per colour and component, bit o = ((dz+2)*3 + dy+1)*3 + dx+1
  // of the 3x3x5 window: check = neighbours coupled through the x-y weights
  // (the centre excluded; planes without band entries are removed per row at
  // run time), early = neighbours of a colour updated before this one in a sweep.
  unsigned long long fcheck[kMaxCoopColours][kMaxComps];
  unsigned long long fearly[kMaxCoopColours][kMaxComps];
  ColumnPass rcp;                        // residual items (2-wide x segments); kc == 0: one site per item
  int vec;                               // 1: transfers on 8-wide fine / 4-wide coarse segments
  RowPass frp, crp;                      // rows of this level and of the coarser one
  T* v;
  const T* b;
  T* t;
  T* bc;
  T* vc;
  unsigned* bar;                         // [0..1] 64-bit arrival count, [2] timeout flag
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier.  bar[0..1] hold a 64-bit arrival count that only grows
// and is a multiple of the grid size when a launch starts (every launch has
// the same grid and passes all its barriers); bar[2] is the timeout flag.
// Thread 0 of each block adds its arrival with release semantics (after the
// block barrier, so the block's writes are ordered before it), takes the
// barrier's target from the count it saw, and polls with acquire loads.
// Every wait is bounded: a block that waits longer than kCoopWaitNs, or sees
// the flag set by another block, sets the flag and returns false; the
// kernel then returns.
__device__ __forceinline__ bool coop_barrier(unsigned* bar) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long* count = reinterpret_cast<unsigned long long*>(bar);
    volatile unsigned* flag = bar + 2;
    int good = *flag == 0u;
    unsigned long long old, cur;
    asm volatile("atom.add.release.gpu.u64 %0, [%1], 1;" : "=l"(old) : "l"(count) : "memory");
    const unsigned long long nb = gridDim.x;
    const unsigned long long target = (old / nb + 1ull) * nb;
    const unsigned long long t0 = global_ns();
    for (;;) {
      asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(cur) : "l"(count) : "memory");
      if (cur >= target) break;
      if (!good || *flag != 0u || global_ns() - t0 > kCoopWaitNs) {
        good = 0;
        break;
      }
    }
    if (!good) atomicExch(bar + 2, 1u);
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// ---- Dataflow order of the colour passes (FP32 levels) ----------------------
// Each stored value carries the parity of its update count in the least
// significant mantissa bit (at most 1 ulp away from the rounded update).
// Within one smoothing phase the counts start at 0 (the phase clears the bit
// of every site behind a grid barrier).  A site of colour c updated in sweep q
// needs its coupled neighbours at count q + 1 (colours before c) or q
// (colours after c); because the operator couples the neighbour back to the
// site, the neighbour's count is then one of {q, q + 1}, resp. {q - 1, q}, so
// the parity alone tells whether it is ready.  A thread updates its sites
// pass after pass as soon as their neighbours are ready, without grid
// barriers, and reads exactly the values the coloured sweep reads.
// Values and tags travel in one 32-bit word with relaxed GPU-scope accesses,
// so no fence is needed.  Every wait is bounded (kCoopWaitNs, or the timeout
// flag set by another thread).
__device__ __forceinline__ float ld_tagged(const float* p) {
  float v;
  asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ void st_tagged(float* p, float v) {
  asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

__device__ __forceinline__ float with_parity(float v, unsigned par) {
  return __uint_as_float((__float_as_uint(v) & ~1u) | par);
}

constexpr unsigned long long kWindowBits = (1ull << kStencil) - 1ull;

// Off-diagonal part of row k (sep_apply's arithmetic, same order) from tagged
// loads; *tags receives the parity bit of every loaded neighbour at its
// window position.
__device__ __forceinline__ float sep_apply_tagged(const CompDev& c, const float* vc, int i, int j, int k,
                                                  const int kk[5], unsigned long long* tags) {
  const int nx = c.nx, ny = c.ny;
  const int xm = i == 0 ? nx - 1 : i - 1, xp = i == nx - 1 ? 0 : i + 1;
  const int jm = j == 0 ? ny - 1 : j - 1, jp = j == ny - 1 ? 0 : j + 1;
  const float* zb = c.zb32 + k * 10;
  unsigned long long tg = 0ull;
  float acc = 0.f;
#pragma unroll
  for (int dz = -2; dz <= 2; ++dz) {
    const float* vp = vc + kk[dz + 2] * ny * nx;
    const int o = (dz + 2) * 9;
    float p1, p2;
    if (ny == 1) {
      const float a = ld_tagged(vp + xm), cc = ld_tagged(vp + xp);
      tg |= ((unsigned long long)(__float_as_uint(a) & 1u) << (o + 3)) |
            ((unsigned long long)(__float_as_uint(cc) & 1u) << (o + 5));
      p1 = c.w1f[3] * a + c.w1f[5] * cc;
      p2 = c.w2f[3] * a + c.w2f[5] * cc;
      if (dz != 0) {
        const float bb = ld_tagged(vp + i);
        tg |= (unsigned long long)(__float_as_uint(bb) & 1u) << (o + 4);
        p1 += c.w1f[4] * bb;
        p2 += c.w2f[4] * bb;
      }
    } else {
      const float* r0 = vp + jm * nx;
      const float* r1 = vp + j * nx;
      const float* r2 = vp + jp * nx;
      const float a0 = ld_tagged(r0 + xm), b0 = ld_tagged(r0 + i), c0 = ld_tagged(r0 + xp);
      const float a1 = ld_tagged(r1 + xm), c1 = ld_tagged(r1 + xp);
      const float a2 = ld_tagged(r2 + xm), b2 = ld_tagged(r2 + i), c2 = ld_tagged(r2 + xp);
      tg |= ((unsigned long long)(__float_as_uint(a0) & 1u) << (o + 0)) |
            ((unsigned long long)(__float_as_uint(b0) & 1u) << (o + 1)) |
            ((unsigned long long)(__float_as_uint(c0) & 1u) << (o + 2)) |
            ((unsigned long long)(__float_as_uint(a1) & 1u) << (o + 3)) |
            ((unsigned long long)(__float_as_uint(c1) & 1u) << (o + 5)) |
            ((unsigned long long)(__float_as_uint(a2) & 1u) << (o + 6)) |
            ((unsigned long long)(__float_as_uint(b2) & 1u) << (o + 7)) |
            ((unsigned long long)(__float_as_uint(c2) & 1u) << (o + 8));
      p1 = c.w1f[0] * a0 + c.w1f[1] * b0 + c.w1f[2] * c0 + c.w1f[3] * a1 + c.w1f[5] * c1 + c.w1f[6] * a2 +
           c.w1f[7] * b2 + c.w1f[8] * c2;
      p2 = c.w2f[0] * a0 + c.w2f[1] * b0 + c.w2f[2] * c0 + c.w2f[3] * a1 + c.w2f[5] * c1 + c.w2f[6] * a2 +
           c.w2f[7] * b2 + c.w2f[8] * c2;
      if (dz != 0) {
        const float b1 = ld_tagged(r1 + i);
        tg |= (unsigned long long)(__float_as_uint(b1) & 1u) << (o + 4);
        p1 += c.w1f[4] * b1;
        p2 += c.w2f[4] * b1;
      }
    }
    acc += zb[dz + 2] * p1 + zb[5 + dz + 2] * p2;
  }
  *tags = tg;
  return acc;
}

__device__ __forceinline__ const float* window_ptr(int nx, int ny, int nz, const float* vc, int i, int j, int k,
                                                   int o) {
  const int dz = o / 9 - 2, dy = (o / 3) % 3 - 1, dx = o % 3 - 1;
  const int ii = i + dx < 0 ? nx - 1 : (i + dx >= nx ? 0 : i + dx);
  const int jj = ny == 1 ? 0 : (j + dy < 0 ? ny - 1 : (j + dy >= ny ? 0 : j + dy));
  const int kk = min(max(k + dz, 0), nz - 1);
  return vc + ((long long)kk * ny + jj) * nx + ii;
}

// Waits until the neighbour at window position o shows parity par (after a
// full read found it not yet updated).  False when the wait timed out or
// another thread raised the timeout flag.
__device__ __noinline__ bool flow_wait1(int nx, int ny, int nz, const float* p0, int i, int j, int k, int o, unsigned par,
                                        const unsigned* flag) {
  const float* p = window_ptr(nx, ny, nz, p0, i, j, k, o);
  const unsigned long long t0 = global_ns();
  for (unsigned it = 1;; ++it) {
    if ((__float_as_uint(ld_tagged(p)) & 1u) == par) return true;
    if ((it & 31u) == 0u && (*(volatile const unsigned*)flag != 0u || global_ns() - t0 > kCoopWaitNs)) return false;
  }
}

// Heat-bath update of site g of colour col in local sweep q (noise counter
// sweep), dataflow order.  False when a wait gave up.
template <bool NOISE>
__device__ __forceinline__ bool flow_site(const CoopLevel<float>& P, const ColourPass& cp, int col, int q, int sweep,
                                          Key key, unsigned long long cy, long long g) {
  const LevelDev& L = P.L;
  const int ci = comp_of(cp.gstart, L.ncomp, g);
  const CompDev& c = L.c[ci];
  const unsigned rank = (unsigned)(g - cp.gstart[ci]);
  const unsigned nxc = (unsigned)cp.nxc[ci], nyc = (unsigned)cp.nyc[ci];
  // shifts for power-of-two class extents (the 64^3 level: 32 x 32)
  const int lx = cp.lxc[ci], ly = cp.lyc[ci];
  const unsigned t = lx >= 0 ? rank >> lx : rank / nxc;
  const int i = cp.cx[ci] + c.mx * (int)(rank - t * nxc);
  const int j = cp.cy[ci] + c.my * (int)(ly >= 0 ? t & (nyc - 1u) : t % nyc);
  const int k = cp.cz[ci] + c.mz * (int)(ly >= 0 ? t >> ly : t / nyc);
  float* vc = P.v + c.off;
  const float* zb = c.zb32 + k * 10;
  int kk[5];
  unsigned long long check = P.fcheck[col][ci];
#pragma unroll
  for (int dz = -2; dz <= 2; ++dz) {
    kk[dz + 2] = min(max(k + dz, 0), c.nz - 1);
    if (zb[dz + 2] == 0.f && zb[5 + dz + 2] == 0.f) check &= ~(0x1FFull << (9 * (dz + 2)));
  }
  const unsigned long long expect = P.fearly[col][ci] ^ ((q & 1) ? kWindowBits : 0ull);
  const long long idx = (long long)((k * c.ny + j) * c.nx + i);
  const float bb = __ldcg(P.b + c.off + idx);
  const float diag = coarse_diag<float>(c, k);
  float off;
  for (;;) {
    unsigned long long tags;
    off = sep_apply_tagged(c, vc, i, j, k, kk, &tags);
    const unsigned long long bad = (tags ^ expect) & check;
    if (bad == 0ull) break;
    const int o = __ffsll((long long)bad) - 1;
    if (!flow_wait1(c.nx, c.ny, c.nz, vc, i, j, k, o, (unsigned)((expect >> o) & 1ull), P.bar + 2)) return false;
  }
  float nv = (bb - off) / diag;
  if (NOISE) {
    float nn;
    normal_of(philox10(make_uint4(rank >> 2, ctr1_of(L.level, c.comp_id, cp.colour_id[ci], sweep, 0), (uint32_t)cy,
                                  (uint32_t)(cy >> 32)),
                       key.k0, key.k1),
              (int)(rank & 3), &nn);
    nv += nn / tsqrt(diag);
  }
  st_tagged(vc + idx, with_parity(nv, (unsigned)((q + 1) & 1)));
  return true;
}

template <typename T, bool NOISE>
__global__ void __launch_bounds__(CoopThreads<T>::value, 2)
    k_level_coop(const __grid_constant__ CoopLevel<T> P, int phase, int mu1, int mu2, Key key,
                 const unsigned long long* __restrict__ cyc) {
  // Logical thread index with the warps interleaved across the blocks: warp
  // w of block b is logical warp w * gridDim.x + b, so a pass with fewer sites
  // than threads still spreads its warps over every SM (each warp keeps 32
  // consecutive sites).
  const long long tid = ((long long)(threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32 + (threadIdx.x & 31);
  const long long nth = (long long)gridDim.x * blockDim.x;
  const unsigned long long cy = NOISE ? *cyc : 0ull;
  const int ncomp = P.L.ncomp;
  constexpr bool kFlowType = std::is_same<T, float>::value;
  const bool flow = kFlowType && P.flow != 0;
  auto sweeps = [&](int first, int count) -> bool {
    if constexpr (kFlowType) {
      if (flow) {
        bool ok = true;
        for (int q = 0; q < count && ok; ++q)
          for (int col = 0; col < P.ncolour && ok; ++col) {
            const ColourPass& cp = P.cp[col];
            for (long long g = tid; g < cp.gstart[ncomp] && ok; g += nth)
              ok = flow_site<NOISE>(P, cp, col, q, first + q, key, cy, g);
          }
        if (!ok) atomicExch(P.bar + 2, 1u);
        return ok;
      }
    }
    for (int q = 0; q < count; ++q)
      for (int col = 0; col < P.ncolour; ++col) {
        const ColourPass& cp = P.cp[col];
        for (long long g = tid; g < cp.gstart[ncomp]; g += nth)
          coarse_site_at<T, NOISE, LdCG>(P.L, cp, P.v, P.b, first + q, key, cy, g);
        if (!coop_barrier(P.bar)) return false;
      }
    return true;
  };
  // Dataflow order: every update count of a phase starts at 0, parity bit
  // clear: phase 0 starts from v = 0 (the launch contract), phase 1 clears the
  // bit as it adds the prolonged correction.
  if (phase == 0) {
    if (flow) {
      sweeps(0, mu1);   // a failed wait raised the flag: the barrier below returns false
      if (!coop_barrier(P.bar)) return;
    } else if (!sweeps(0, mu1)) {
      return;
    }
    // The residual's loads go through L1: no L1 line of v can be stale here,
    // since every read of v earlier in the launch bypassed L1 (GPU-scope
    // relaxed loads in dataflow order, .cg loads between grid barriers) and L1
    // starts empty at launch.
    if (P.rcp.kc > 0) {   // separable form along z columns of 2-wide segments
      for (long long g = tid; g < P.rcp.start[ncomp]; g += nth) {
        int ci = 0;
        while (ci + 1 < ncomp && g >= P.rcp.start[ci + 1]) ++ci;
        const CompDev& c = P.L.c[ci];
        const int segs = c.nx >> 1;
        const long long item = g - P.rcp.start[ci];
        const long long col = item % ((long long)c.ny * segs);
        const int chunk = (int)(item / ((long long)c.ny * segs));
        const int j = (int)(col / segs), seg = (int)(col - (long long)j * segs);
        const int k0 = chunk * P.rcp.kc, k1 = min(k0 + P.rcp.kc, c.nz);
        galerkin_residual_seg<T, 2, LdPlain>(c, P.v + c.off, P.b + c.off, P.t + c.off, j, seg << 1, k0, k1);
      }
    } else {
      for (long long s = tid; s < P.L.size; s += nth) {
        int ci, i, j, k;
        site_of(P.L, s, &ci, &i, &j, &k);
        const CompDev& c = P.L.c[ci];
        P.t[s] = P.b[s] - sep_apply<T, LdPlain, true>(c, P.v + c.off, i, j, k);
      }
    }
    if (!coop_barrier(P.bar)) return;
    if (P.vec) {   // t was written by other SMs in this launch: read through L2
      const long long items = (long long)P.crp.rstart[ncomp] * (P.Lc.c[0].nx >> 2);
      for (long long g = tid; g < items; g += nth) restrict_seg4<T, true>(P.L, P.Lc, P.crp, P.t, P.bc, g);
      for (long long s = tid; s < P.Lc.size; s += nth) P.vc[s] = (T)0;
    } else {
      for (long long s = tid; s < P.Lc.size; s += nth) {
        restrict_at<T, LdCG>(P.L, P.Lc, P.t, P.bc, s);
        P.vc[s] = (T)0;
      }
    }
  } else {
    // v += P vc; in dataflow order the parity bit is cleared (update count 0
    // for the post-smoothing)
    if (P.vec) {
      const long long items = (long long)P.frp.rstart[ncomp] * (P.L.c[0].nx >> 3);
      for (long long g = tid; g < items; g += nth) {
        if (flow)
          prolong_seg8<T, true>(P.L, P.Lc, P.frp, P.v, P.vc, g);
        else
          prolong_seg8<T, false>(P.L, P.Lc, P.frp, P.v, P.vc, g);
      }
      if (!coop_barrier(P.bar)) return;
      sweeps(mu1, mu2);
      return;
    }
    // otherwise two sites per iteration
    auto put = [&](long long s, T val) {
      if constexpr (kFlowType) {
        if (flow) val = with_parity(val, 0u);
      }
      P.v[s] = val;
    };
    for (long long s = tid; s < P.L.size; s += 2 * nth) {
      const long long s2 = s + nth;
      const T a1 = prolong_val<T>(P.L, P.Lc, P.vc, s);
      const T a2 = s2 < P.L.size ? prolong_val<T>(P.L, P.Lc, P.vc, s2) : (T)0;
      const T v1 = P.v[s] + a1;
      const T v2 = s2 < P.L.size ? P.v[s2] + a2 : (T)0;
      put(s, v1);
      if (s2 < P.L.size) put(s2, v2);
    }
    if (!coop_barrier(P.bar)) return;
    sweeps(mu1, mu2);
  }
}

// ---------------------------------------------------------------------------
// Coarsest level: v = L^-T (L^-1 b + noise * n), FP64, one block per component.
// ---------------------------------------------------------------------------
template <typename T, bool NOISE>
__global__ void k_coarsest(LevelDev L, T* __restrict__ v, const T* __restrict__ b, Key key,
                           const unsigned long long* __restrict__ cyc) {
  extern __shared__ double sm[];
  const CompDev& c = L.c[blockIdx.x];
  const int N = c.nx * c.ny * c.nz;
  double* bb = sm;
  double* y = sm + N;
  for (int q = threadIdx.x; q < N; q += blockDim.x) bb[q] = (double)b[c.off + q];
  __syncthreads();
  for (int r = threadIdx.x; r < N; r += blockDim.x) {
    double acc = 0.0;
    for (int q = 0; q <= r; ++q) acc += c.Linv[(long long)r * N + q] * bb[q];
    if (NOISE) {
      const unsigned long long cy = *cyc;
      uint4 ctr = make_uint4((uint32_t)(r >> 2), ctr1_of(L.level, c.comp_id, 0, 0, 1), (uint32_t)cy,
                             (uint32_t)(cy >> 32));
      double n4[4];
      Normals<double>::get(philox10(ctr, key.k0, key.k1), n4);
      acc += n4[r & 3];
    }
    y[r] = acc;
  }
  __syncthreads();
  for (int col = threadIdx.x; col < N; col += blockDim.x) {
    double acc = 0.0;
    for (int r = col; r < N; ++r) acc += c.Linv[(long long)r * N + col] * y[r];
    v[c.off + col] = (T)acc;
  }
}

// ---------------------------------------------------------------------------
// Batched FAC cycle of many independent systems as one persistent launch.
//
// One cooperative launch runs a whole FAC iteration (Algorithm 1 around the
// V-cycle of Algorithm 3) for every system of a batch.  The cycle is cut into
// phases -- the FP64 outer residual, each colour pass of each sweep of each
// level, the residual and restriction of each level, the two triangular
// solves of the coarsest exact step, each prolongation, the FP64 update --
// aligned by level across the systems (a system whose hierarchy is shallower
// takes its coarsest step at its own last level and has no work in the
// deeper phases).  A phase's work items of all systems form one index range
// that every thread strides over; a grid barrier separates phases.  Each
// system's work items are those of its own per-system kernels (the same
// per-item functions, noise counters and arithmetic), with every load of data
// written earlier in the launch taken from L2.  The host builds the phase
// list and, per phase, the first item of each system.
// ---------------------------------------------------------------------------
constexpr int kBatchColours = 12;
constexpr int kBatchThreads = 256;

enum BatchPhaseType : int {
  kPhOuterRes = 0,   // r = b - A z (FP64) into the level-0 rhs, v0 = 0; squared norm (solve)
  kPhSmooth = 1,     // one colour pass (level, sweep, colour)
  kPhCoarse1 = 2,    // coarsest level: y = L^-1 b (+ n)
  kPhCoarse2 = 3,    // coarsest level: v = L^-T y
  kPhResid = 4,      // t = b - A v at a level
  kPhRestrict = 5,   // b_c = P^T t, v_c = 0
  kPhProlong = 6,    // v += P v_c
  kPhOuterUpd = 7,   // z += v0 (FP64); the solve's norm slot cleared; the chain counter advanced
};

struct BatchPhase {
  int type, level, sweep, colour;
};

struct BatchLevelDev {
  LevelDev L;
  void* v;
  void* b;
  void* t;
  ColourPass cp[kBatchColours];
  ColumnPass sp[kBatchColours];   // 8-wide segment items of colour q (v8 levels)
  ColumnPass rcp;      // residual items: 4-wide segments of z chunks (levels >= 1, nx % 4 == 0)
  int v8;              // colour passes on 8-wide segments (nx % 8 == 0, x modulus 2)
  RowPass rp;          // rows of this level's components
  int vec_down;        // restriction from this level on 4-wide coarse segments
  int vec_up;          // prolongation into this level on 8-wide fine segments
};

struct BatchSysDev {
  int levels;
  Key key;
  const unsigned long long* cyc[2];   // noise counters: [0] chain, [1] solve stages
  unsigned long long* chain_ctr;
  double* z[2];                       // FP64 iterates: [0] chain state xi, [1] velocity u
  const double* bz[2];                // right-hand sides: [0] none (0), [1] b
  double* norm2;                      // ||b - A u||^2 of the solve
  double* ywork;                      // FP64 scratch of the coarsest step
  ColumnPass fcp;                     // level-0 column items
  RowPass orp;                        // level-0 rows (outer residual on 4-wide segments)
  BatchLevelDev lev[kMaxLevels];
};

template <typename T, bool CG>
__device__ __forceinline__ double outer_residual4_item(const LevelDev& L, const RowPass& rp, const double* z,
                                                       const double* b, T* r, T* v0, long long gt) {
  const int segs = L.c[0].nx >> 2;
  const long long row_all = gt / segs;
  const int seg = (int)(gt - row_all * segs);
  int ci = 0;
  while (ci + 1 < L.ncomp && row_all >= rp.rstart[ci + 1]) ++ci;
  const CompDev& c = L.c[ci];
  const int row = (int)(row_all - rp.rstart[ci]);
  const int j = row % c.ny, k = row / c.ny;
  const int nx = c.nx;
  const long long plane = (long long)nx * c.ny;
  const long long rbase = c.off + (long long)row * nx;
  const int x0 = seg << 2;
  auto ld = [&](const double* p) { return CG ? __ldcg(p) : *p; };
  auto ld4 = [&](const double* p, double o[4]) {
    const double2 a = CG ? __ldcg(reinterpret_cast<const double2*>(p)) : *reinterpret_cast<const double2*>(p);
    const double2 d = CG ? __ldcg(reinterpret_cast<const double2*>(p + 2)) : *reinterpret_cast<const double2*>(p + 2);
    o[0] = a.x;
    o[1] = a.y;
    o[2] = d.x;
    o[3] = d.y;
  };
  double cen[4], acc[4], t4[4];
  ld4(z + rbase + x0, cen);
  const double left = ld(z + rbase + (x0 == 0 ? nx - 1 : x0 - 1));
  const double right = ld(z + rbase + (x0 + 4 == nx ? 0 : x0 + 4));
  acc[0] = left + cen[1];
  acc[1] = cen[0] + cen[2];
  acc[2] = cen[1] + cen[3];
  acc[3] = cen[2] + right;
  auto add4 = [&](long long off) {
    ld4(z + off, t4);
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[e] += t4[e];
  };
  if (c.ny > 1) {
    add4(c.off + ((long long)k * c.ny + (j == 0 ? c.ny - 1 : j - 1)) * nx + x0);
    add4(c.off + ((long long)k * c.ny + (j == c.ny - 1 ? 0 : j + 1)) * nx + x0);
  }
  if (k > 0) add4(rbase - plane + x0);
  if (k < c.nz - 1) add4(rbase + plane + x0);
  const int edges = (k == 0) + (k == c.nz - 1);
  double dz = 2.0;
  if (c.zkind == kAxisCellDir) dz += (double)edges;
  if (c.zkind == kAxisCellNeu) dz -= (double)edges;
  const double dg = (c.ny > 1 ? 4.0 : 2.0) + dz;
  const double sdg = c.s * dg;
  double rr = 0.0, bv[4] = {0.0, 0.0, 0.0, 0.0};
  if (b) ld4(b + rbase + x0, bv);
  T out[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const double res = fma(c.s, acc[e], fma(-sdg, cen[e], bv[e]));   // k_outer_residual_v4's arithmetic
    out[e] = (T)res;
    rr = fma(res, res, rr);
  }
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(r + rbase + x0) = make_float4(out[0], out[1], out[2], out[3]);
    *reinterpret_cast<float4*>(v0 + rbase + x0) = make_float4(0.f, 0.f, 0.f, 0.f);
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      r[rbase + x0 + e] = out[e];
      v0[rbase + x0 + e] = (T)0;
    }
  }
  return rr;
}

// Component and local index of item q of a level's flattened field.
__device__ __forceinline__ int comp_at(const LevelDev& L, long long q, long long* loc) {
  int ci = 0;
  while (ci + 1 < L.ncomp && q >= L.c[ci + 1].off) ++ci;
  *loc = q - L.c[ci].off;
  return ci;
}

// Loads of the persistent launch.  Data written by other blocks in an earlier
// phase are read after a grid barrier (coop_barrier: block barrier, release
// add, acquire poll, block barrier) -- the release/acquire pair orders every
// write of the phase before every read of the next one, as a grid-wide
// synchronisation does, so plain (L1-cached) loads see the phase's data.
constexpr bool kBatchL2 = false;
using BatchLd = std::conditional_t<kBatchL2, LdCG, LdPlain>;

template <typename T, bool NOISE>
__device__ __forceinline__ void batch_item(const BatchSysDev& S, const BatchPhase& P, int mode, long long g,
                                           double* nacc) {
  const int l = P.level;
  const BatchLevelDev& BL = S.lev[l];
  const LevelDev& L = BL.L;
  T* v = (T*)BL.v;
  const T* b = (const T*)BL.b;
  switch (P.type) {
    case kPhOuterRes: {
      const double rr =
          outer_residual4_item<T, kBatchL2>(L, S.orp, S.z[mode], S.bz[mode], (T*)BL.b, (T*)BL.v, g);
      if (mode == 1) *nacc += rr;
      break;
    }
    case kPhSmooth: {
      const unsigned long long cy = NOISE ? *S.cyc[mode] : 0ull;
      if (l == 0)
        fine_colour_zm_item<T, NOISE, kBatchL2>(L, S.fcp, v, b, P.colour, P.sweep, S.key, cy, g);
      else if (BL.v8 && (P.colour & 1) == 0)
        coarse_colour_v8_item<T, NOISE, 0, kBatchL2>(L, BL.cp[P.colour], BL.sp[P.colour], v, b, P.sweep, S.key, cy, g);
      else if (BL.v8)
        coarse_colour_v8_item<T, NOISE, 1, kBatchL2>(L, BL.cp[P.colour], BL.sp[P.colour], v, b, P.sweep, S.key, cy, g);
      else
        coarse_site_at<T, NOISE, BatchLd>(L, BL.cp[P.colour], v, b, P.sweep, S.key, cy, g);
      break;
    }
    case kPhCoarse1: {
      // eight consecutive items (lanes of one warp) share a row: strided
      // partial sums, then a shuffle reduction
      // (the system's items are padded to whole warps; padded lanes only
      // take part in the shuffles)
      const int sub = (int)(g & 7);
      const bool valid = (g >> 3) < L.size;
      long long r = 0;
      const int ci = valid ? comp_at(L, g >> 3, &r) : 0;
      const CompDev& c = L.c[ci];
      const long long N = (long long)c.nx * c.ny * c.nz;
      double acc = 0.0;
      if (valid)
        for (long long q = sub; q <= r; q += 8) acc += c.Linv[r * N + q] * (double)ld1<T, kBatchL2>(b + c.off + q);
      acc += __shfl_xor_sync(0xffffffffu, acc, 4);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      if (!valid || sub != 0) break;
      if (NOISE) {
        const unsigned long long cy = *S.cyc[mode];
        const uint4 ctr = make_uint4((uint32_t)(r >> 2), ctr1_of(L.level, c.comp_id, 0, 0, 1), (uint32_t)cy,
                                     (uint32_t)(cy >> 32));
        double n4[4];
        Normals<double>::get(philox10(ctr, S.key.k0, S.key.k1), n4);
        acc += n4[r & 3];
      }
      S.ywork[c.off + r] = acc;
      break;
    }
    case kPhCoarse2: {
      const int sub = (int)(g & 7);
      const bool valid = (g >> 3) < L.size;
      long long col = 0;
      const int ci = valid ? comp_at(L, g >> 3, &col) : 0;
      const CompDev& c = L.c[ci];
      const long long N = (long long)c.nx * c.ny * c.nz;
      double acc = 0.0;
      if (valid)
        for (long long r = col + sub; r < N; r += 8) acc += c.Linv[r * N + col] * ld1<double, kBatchL2>(S.ywork + c.off + r);
      acc += __shfl_xor_sync(0xffffffffu, acc, 4);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      if (valid && sub == 0) v[c.off + col] = (T)acc;
      break;
    }
    case kPhResid: {
      if (l == 0) {
        fine_residual_zm_item<T, kBatchL2>(L, S.fcp, v, b, (T*)BL.t, g);
      } else if (BL.rcp.kc > 0) {
        int ci = 0;
        while (ci + 1 < L.ncomp && g >= BL.rcp.start[ci + 1]) ++ci;
        const CompDev& c = L.c[ci];
        const int segs = c.nx >> 2;
        const long long item = g - BL.rcp.start[ci];
        const long long col = item % ((long long)c.ny * segs);
        const int chunk = (int)(item / ((long long)c.ny * segs));
        const int j = (int)(col / segs), seg = (int)(col - (long long)j * segs);
        const int k0 = chunk * BL.rcp.kc, k1 = min(k0 + BL.rcp.kc, c.nz);
        galerkin_residual_seg<T, 4, BatchLd>(c, v + c.off, b + c.off, (T*)BL.t + c.off, j, seg << 2, k0, k1);
      } else {
        int ci, i, j, k;
        site_of(L, g, &ci, &i, &j, &k);
        const CompDev& c = L.c[ci];
        ((T*)BL.t)[g] = ld1<T, kBatchL2>(b + g) - sep_apply<T, BatchLd, true>(c, v + c.off, i, j, k);
      }
      break;
    }
    case kPhRestrict: {
      const BatchLevelDev& BC = S.lev[l + 1];
      const long long nres = BL.vec_down ? (long long)BC.rp.rstart[BC.L.ncomp] * (BC.L.c[0].nx >> 2) : BC.L.size;
      if (g < nres) {
        if (BL.vec_down)
          restrict_seg4<T, kBatchL2>(L, BC.L, BC.rp, (const T*)BL.t, (T*)BC.b, g);
        else
          restrict_at<T, BatchLd>(L, BC.L, (const T*)BL.t, (T*)BC.b, g);
      } else {
        ((T*)BC.v)[g - nres] = (T)0;
      }
      break;
    }
    case kPhProlong: {
      const BatchLevelDev& BC = S.lev[l + 1];
      if (BL.vec_up)
        prolong_seg8<T, false, kBatchL2>(L, BC.L, BL.rp, v, (const T*)BC.v, g);
      else
        v[g] = ld1<T, kBatchL2>(v + g) + prolong_val<T, BatchLd>(L, BC.L, (const T*)BC.v, g);
      break;
    }
    case kPhOuterUpd: {
      double* z = S.z[mode];
      double2* z2 = reinterpret_cast<double2*>(z + 4 * g);
      double2 a = z2[0], d = z2[1];
      if constexpr (sizeof(T) == 4) {
        const float4 q = kBatchL2 ? __ldcg(reinterpret_cast<const float4*>(v + 4 * g))
                                  : *reinterpret_cast<const float4*>(v + 4 * g);
        a.x += (double)q.x;
        a.y += (double)q.y;
        d.x += (double)q.z;
        d.y += (double)q.w;
      } else {
        a.x += (double)ld1<T, kBatchL2>(v + 4 * g);
        a.y += (double)ld1<T, kBatchL2>(v + 4 * g + 1);
        d.x += (double)ld1<T, kBatchL2>(v + 4 * g + 2);
        d.y += (double)ld1<T, kBatchL2>(v + 4 * g + 3);
      }
      z2[0] = a;
      z2[1] = d;
      if (g == 0) {
        if (mode == 1) *S.norm2 = 0.0;
        if (mode == 0) *S.chain_ctr += 1ull;
      }
      break;
    }
    default:
      break;
  }
}

// start: [nphase][nsys + 1] first item of each system in each phase.
// mode 0: a stochastic cycle of every chain; 1: a deterministic cycle of every
// velocity solve.  Shared memory: nsys doubles (per-block norm partial sums).
template <typename T, bool NOISE>
__global__ void __launch_bounds__(kBatchThreads, 2) k_batch_fac(const BatchSysDev* __restrict__ sys, int nsys,
                                                             const BatchPhase* __restrict__ ph, int nphase,
                                                             const long long* __restrict__ start, unsigned* bar,
                                                             int mode, unsigned long long* tstamp) {
  // shared memory: nsys doubles (per-block norm partial sums), then the
  // phase's first-item table (nsys + 1 words)
  extern __shared__ double bnorm[];
  long long* sst = reinterpret_cast<long long*>(bnorm + nsys);
  if (tstamp && blockIdx.x == 0 && threadIdx.x == 0) tstamp[0] = global_ns();
  const long long tid = ((long long)(threadIdx.x >> 5) * gridDim.x + blockIdx.x) * 32 + (threadIdx.x & 31);
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (int p = 0; p < nphase; ++p) {
    const BatchPhase P = ph[p];
    const long long* st = start + (long long)p * (nsys + 1);
    for (int q = threadIdx.x; q <= nsys; q += blockDim.x) sst[q] = __ldg(st + q);
    const bool norm = P.type == kPhOuterRes && mode == 1;
    if (norm)
      for (int q = threadIdx.x; q < nsys; q += blockDim.x) bnorm[q] = 0.0;
    __syncthreads();
    const long long total = sst[nsys];
    int s = -1;
    double acc = 0.0;
    for (long long g = tid; g < total; g += nth) {
      if (s < 0 || g >= sst[s + 1]) {
        if (norm && s >= 0 && acc != 0.0) atomicAdd(bnorm + s, acc);
        acc = 0.0;
        // the system whose items hold g: last s with sst[s] <= g (binary search)
        int lo = s < 0 ? 0 : s + 1, hi = nsys - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (sst[mid] <= g)
            lo = mid;
          else
            hi = mid - 1;
        }
        s = lo;
      }
      batch_item<T, NOISE>(sys[s], P, mode, g - sst[s], &acc);
    }
    if (norm) {
      if (s >= 0 && acc != 0.0) atomicAdd(bnorm + s, acc);
      __syncthreads();
      for (int q = threadIdx.x; q < nsys; q += blockDim.x)
        if (bnorm[q] != 0.0) atomicAdd(sys[q].norm2, bnorm[q]);
    }
    // (the barrier's leading block barrier also guards sst for the next phase)
    if ((p + 1 < nphase || tstamp) && !coop_barrier(bar)) return;
    // phase end as block 0 sees it (profiling; after the barrier, so every
    // block finished the phase)
    if (tstamp && blockIdx.x == 0 && threadIdx.x == 0) tstamp[p + 1] = global_ns();
  }
}

// ---------------------------------------------------------------------------
// FP64 outer iteration (Algorithm 1 steps 1 and 4)
// ---------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(kBlock) k_outer_residual(LevelDev L, const double* __restrict__ z,
                                                          const double* __restrict__ b, T* __restrict__ r,
                                                          double* __restrict__ norm2) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double rr = 0.0;
  if (s < L.size) {
    int ci, i, j, k;
    site_of(L, s, &ci, &i, &j, &k);
    double off, diag;
    fine_row<double, double>(L.c[ci], z, i, j, k, &off, &diag);
    const double res = (b ? b[s] : 0.0) - (off + diag * z[s]);
    r[s] = (T)res;
    rr = res * res;
  }
  if (norm2) {
    rr = block_sum(rr);
    if (threadIdx.x == 0) atomicAdd(norm2, rr);
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_outer_update(long long n, double* __restrict__ z,
                                                        const T* __restrict__ d) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) z[s] += (double)d[s];
}

__global__ void __launch_bounds__(kBlock) k_norm2(long long n, const double* __restrict__ x,
                                                 double* __restrict__ out) {
  double acc = 0.0;
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x)
    acc += x[s] * x[s];
  acc = block_sum(acc);
  if (threadIdx.x == 0) atomicAdd(out, acc);
}

__global__ void __launch_bounds__(kBlock) k_axpby(long long n, double a, const double* __restrict__ x, double c,
                                                 const double* __restrict__ y, double* __restrict__ out) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) out[s] = a * x[s] + c * y[s];
}

__global__ void k_set_u64(unsigned long long* p, unsigned long long v) { *p = v; }
__global__ void k_inc_u64(unsigned long long* p) { *p += 1ull; }

// ---------------------------------------------------------------------------
// Peskin 4-point coupling (Section 2.1; kernel from Peskin, Acta Numerica 2002)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double peskin_phi(double r) {
  r = fabs(r);
  if (r <= 1.0) return (3.0 - 2.0 * r + sqrt(1.0 + 4.0 * r - 4.0 * r * r)) * 0.125;
  if (r <= 2.0) return (5.0 - 2.0 * r - sqrt(fmax(-7.0 + 12.0 * r - 4.0 * r * r, 0.0))) * 0.125;
  return 0.0;
}

// Node index (or -1) and weight of slot t (0..3) along one axis.
// kind: periodic (offset off in cells), vertex wall lattice, cell wall lattice.
__device__ __forceinline__ void axis_node(int kind, double x, double off, int n, int t, int* idx, double* w) {
  if (kind == kAxisTrivial) {
    *idx = t == 0 ? 0 : -1;
    *w = t == 0 ? 1.0 : 0.0;
    return;
  }
  double o = kind == kAxisVertex ? 0.0 : (kind == kAxisPeriodic ? off : 0.5);
  const int a = (int)floor(x - o) - 1 + t;
  *w = peskin_phi(x - o - (double)a);
  if (kind == kAxisPeriodic) {
    int m = a % n;
    *idx = m < 0 ? m + n : m;
  } else if (kind == kAxisVertex) {
    *idx = (a >= 1 && a <= n - 1) ? a - 1 : -1;
  } else {
    *idx = (a >= 0 && a <= n - 1) ? a : -1;
  }
}

struct CouplingGeom {
  int kind[3];
  double off[3];
  int col[3];   // particle column per axis (-1 = trivial axis)
};

__device__ __forceinline__ CouplingGeom geom_of(const CompDev& c, int dim) {
  CouplingGeom g;
  g.kind[0] = kAxisPeriodic;
  g.kind[1] = dim == 3 ? kAxisPeriodic : kAxisTrivial;
  g.kind[2] = c.zkind;
  // face-normal component: offset 0 along its own axis, 1/2 along the others
  g.off[0] = c.comp_id == 0 ? 0.0 : 0.5;
  g.off[1] = c.comp_id == 1 ? 0.0 : 0.5;
  g.off[2] = 0.0;
  g.col[0] = 0;
  g.col[1] = dim == 3 ? 1 : -1;
  g.col[2] = dim == 3 ? 2 : 1;
  return g;
}

__device__ __forceinline__ int comp_col(const CompDev& c, int dim) { return dim == 3 ? c.comp_id : (c.comp_id == 0 ? 0 : 1); }

// The 1-D kernel taps of one particle and component, shared across a warp:
// lane 4a + t (a < 3, t < 4) evaluates tap t of axis a once; node q of the
// 4^d support (q = t0 + 4 t1 + 16 t2) gathers its three taps by shuffles.
// Every lane of the warp must call both.
__device__ __forceinline__ void taps_of(const CouplingGeom& ge, const double* X, int p, int dim, int n, int lane,
                                        int* idl, double* wl) {
  *idl = -1;
  *wl = 0.0;
  if (lane < 12) {
    const int a = lane >> 2, t = lane & 3;
    const double x = ge.col[a] >= 0 ? X[(long long)p * dim + ge.col[a]] * n : 0.0;
    axis_node(ge.kind[a], x, ge.off[a], n, t, idl, wl);
  }
}

// Node q's grid index (ok == false: a tap outside the walls) and weight, the
// product taken axis by axis as the per-node evaluation does.
__device__ __forceinline__ void node_of(int q, int dim, int idl, double wl, int id[3], double* w, bool* ok) {
  const int tq[3] = {q & 3, dim == 3 ? (q >> 2) & 3 : 0, dim == 3 ? (q >> 4) & 3 : (q >> 2) & 3};
  *w = 1.0;
  *ok = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    id[a] = __shfl_sync(0xffffffffu, idl, 4 * a + tq[a]);
    const double wa = __shfl_sync(0xffffffffu, wl, 4 * a + tq[a]);
    *ok = *ok && id[a] >= 0;
    *w *= wa;
  }
}

// f(node) += F_p w(node): one warp per (particle, component), the taps
// evaluated once per axis, two nodes per lane (FP64 atomics).
__global__ void __launch_bounds__(kBlock) k_spread(LevelDev L, int n, int dim, int np, const double* __restrict__ X,
                                                  const double* __restrict__ F, double* __restrict__ b) {
  const int nodes = dim == 3 ? 64 : 16;
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= (long long)np * L.ncomp) return;   // whole warps leave together
  const int ci = (int)(wid % L.ncomp);
  const int p = (int)(wid / L.ncomp);
  const CompDev& c = L.c[ci];
  const CouplingGeom ge = geom_of(c, dim);
  int idl;
  double wl;
  taps_of(ge, X, p, dim, n, lane, &idl, &wl);
  const double f = F[(long long)p * dim + comp_col(c, dim)];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int q = lane + 32 * h;
    int id[3];
    double w;
    bool ok;
    node_of(q & 63, dim, idl, wl, id, &w, &ok);
    if (q < nodes && ok && w != 0.0)
      atomicAdd(&b[c.off + ((long long)id[2] * c.ny + id[1]) * c.nx + id[0]], f * w);
  }
}

// U_p = sum_node w(node) u(node): one warp per (particle, component), the taps
// evaluated once per axis, two nodes per lane, warp reduction.
__global__ void __launch_bounds__(kBlock) k_interp(LevelDev L, int n, int dim, int np, const double* __restrict__ X,
                                                  const double* __restrict__ u, double* __restrict__ U) {
  const int nodes = dim == 3 ? 64 : 16;
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= (long long)np * L.ncomp) return;
  const int ci = (int)(wid % L.ncomp);
  const int p = (int)(wid / L.ncomp);
  const CompDev& c = L.c[ci];
  const CouplingGeom ge = geom_of(c, dim);
  int idl;
  double wl;
  taps_of(ge, X, p, dim, n, lane, &idl, &wl);
  double acc = 0.0;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int q = lane + 32 * h;
    int id[3];
    double w;
    bool ok;
    node_of(q & 63, dim, idl, wl, id, &w, &ok);
    if (q < nodes && ok) acc += w * u[c.off + ((long long)id[2] * c.ny + id[1]) * c.nx + id[0]];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) U[(long long)p * dim + comp_col(c, dim)] = acc;
}

__global__ void __launch_bounds__(kBlock) k_em(int np, int dim, double* __restrict__ X, const double* __restrict__ V) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  for (int a = 0; a < dim; ++a) {
    double x = X[(long long)p * dim + a] + V[(long long)p * dim + a];
    if (a < dim - 1) {
      x = x - floor(x);
    } else {
      if (x < 0.0) x = -x;
      if (x > 1.0) x = 2.0 - x;
    }
    X[(long long)p * dim + a] = x;
  }
}

// ---------------------------------------------------------------------------
// MAC projection pieces (Section 4): D^ w at cells, w -= D^T phi at faces.
// ---------------------------------------------------------------------------
// div = D w on the cells, and the sum of div added to *sum: a grid-stride
// loop over a few blocks per SM, so that one FP64 atomic per block (all on
// the same word) stays off the kernel's critical path.
__global__ void __launch_bounds__(kBlock) k_divergence(LevelDev Lv, const double* __restrict__ w,
                                                      double* __restrict__ div, double* __restrict__ sum) {
  const CompDev& u = Lv.c[0];
  const CompDev& wz = Lv.c[Lv.ncomp - 1];
  const int nx = u.nx, ny = u.ny, nz = u.nz;
  const unsigned N = (unsigned)nx * (unsigned)ny * (unsigned)nz;   // < 2^31 (checked by the launcher)
  double acc = 0.0;
  for (unsigned su = blockIdx.x * blockDim.x + threadIdx.x; su < N; su += gridDim.x * blockDim.x) {
    const unsigned t = su / (unsigned)nx;
    const int i = (int)(su - t * (unsigned)nx);
    const int j = (int)(t % (unsigned)ny), k = (int)(t / (unsigned)ny);
    const long long rowc = ((long long)k * ny + j) * nx;
    double d = w[u.off + rowc + wrapi(i + 1, nx)] - w[u.off + rowc + i];
    if (Lv.ncomp == 3) {
      const CompDev& v = Lv.c[1];
      d += w[v.off + ((long long)k * ny + wrapi(j + 1, ny)) * nx + i] - w[v.off + rowc + i];
    }
    if (k < nz - 1) d += w[wz.off + rowc + i];
    if (k > 0) d -= w[wz.off + rowc - (long long)nx * ny + i];
    div[su] = d;
    acc += d;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) atomicAdd(sum, acc);
}

// x -= sum / n.  The quotient is formed once per block: an FP64 division per
// element would keep GB300's FP64 pipe busy for several times the copy.
__global__ void __launch_bounds__(kBlock) k_sub_mean(long long n, double* __restrict__ x, const double* __restrict__ sum) {
  __shared__ double mean;
  if (threadIdx.x == 0) mean = *sum / (double)n;
  __syncthreads();
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) x[s] -= mean;
}

__global__ void __launch_bounds__(kBlock) k_grad_sub(LevelDev Lv, double* __restrict__ w, const double* __restrict__ phi) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Lv.size) return;
  int ci, i, j, k;
  site_of(Lv, s, &ci, &i, &j, &k);
  const CompDev& u0 = Lv.c[0];
  const int nx = u0.nx, ny = u0.ny;
  const long long rowc = ((long long)k * ny + j) * nx;
  double g;
  const int cid = Lv.c[ci].comp_id;
  if (cid == 0) {
    g = phi[rowc + wrapi(i - 1, nx)] - phi[rowc + i];
  } else if (cid == 1) {
    g = phi[((long long)k * ny + wrapi(j - 1, ny)) * nx + i] - phi[rowc + i];
  } else {
    g = phi[rowc + i] - phi[rowc + (long long)nx * ny + i];
  }
  w[s] -= g;
}

__global__ void k_philox(const uint32_t* __restrict__ ctr, Key key, uint32_t* __restrict__ out, int n) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  uint4 c = make_uint4(ctr[4 * q], ctr[4 * q + 1], ctr[4 * q + 2], ctr[4 * q + 3]);
  uint4 r = philox10(c, key.k0, key.k1);
  out[4 * q] = r.x;
  out[4 * q + 1] = r.y;
  out[4 * q + 2] = r.z;
  out[4 * q + 3] = r.w;
}

inline unsigned grid_for(long long n, int block = kBlock) { return (unsigned)((n + block - 1) / block); }

}  // namespace

// Colour q of a Galerkin level: class origin and extents per component, and
// the first site of each component in the flattened pass (components whose
// colour count is below q + 1 contribute none).  Returns the pass's sites.
long long colour_pass_of(const LevelDev& L, int q, ColourPass* cp) {
  long long gs = 0;
  for (int ci = 0; ci < L.ncomp; ++ci) {
    const CompDev& c = L.c[ci];
    cp->gstart[ci] = gs;
    cp->nsites[ci] = 0;
    if (q < c.ncol) {
      const int cx = q % c.mx, cy = (q / c.mx) % c.my, cz = q / (c.mx * c.my);
      cp->cx[ci] = cx;
      cp->cy[ci] = cy;
      cp->cz[ci] = cz;
      cp->nxc[ci] = (c.nx - cx + c.mx - 1) / c.mx;
      cp->nyc[ci] = (c.ny - cy + c.my - 1) / c.my;
      cp->nzc[ci] = (c.nz - cz + c.mz - 1) / c.mz;
      cp->colour_id[ci] = q;
      if (cp->nxc[ci] > 0 && cp->nyc[ci] > 0 && cp->nzc[ci] > 0)
        cp->nsites[ci] = (long long)cp->nxc[ci] * cp->nyc[ci] * cp->nzc[ci];
    }
    if (cp->nxc[ci] <= 0) cp->nxc[ci] = 1;
    if (cp->nyc[ci] <= 0) cp->nyc[ci] = 1;
    auto log2_or = [](int n) {
      int l = 0;
      while ((1 << l) < n) ++l;
      return (1 << l) == n ? l : -1;
    };
    cp->lxc[ci] = log2_or(cp->nxc[ci]);
    cp->lyc[ci] = log2_or(cp->nyc[ci]);
    gs += cp->nsites[ci];
  }
  cp->gstart[L.ncomp] = gs;
  return gs;
}

// ---- batched FAC cycles as one persistent launch (host side) --------------
struct BatchPersist {
  int nsys = 0, esize = 4, mu1 = 2, mu2 = 2;
  std::vector<BatchSysDev> sys;
  BatchSysDev* dsys = nullptr;
  double* ywork = nullptr;
  double* norms = nullptr;   // [nsys] squared residual norms of the solves
  unsigned* bar = nullptr;   // grid barrier words
  // phase lists: 0 chain cycle, 1 pipelined solve cycle, 2 solve cycle from u
  std::vector<BatchPhase> ph[3];
  std::vector<long long> st[3];
  BatchPhase* dph[3] = {};
  long long* dst[3] = {};
  int kc = 16, bps = 1, blocks = 0;
};

namespace {

bool batch_vec_down(const LevelDev& Lf, const LevelDev& Lc) {
  if (Lf.c[0].nx % 8 != 0) return false;
  for (int ci = 0; ci < Lf.ncomp; ++ci)
    if (Lf.c[ci].nx != Lf.c[0].nx || Lc.c[ci].nx * 2 != Lf.c[ci].nx) return false;
  return true;
}

bool batch_vec_up(const LevelDev& Lf) {
  if (Lf.c[0].nx % 8 != 0) return false;
  for (int ci = 0; ci < Lf.ncomp; ++ci)
    if (Lf.c[ci].nx != Lf.c[0].nx) return false;
  return true;
}

RowPass rows_of(const LevelDev& L) {
  RowPass rp{};
  int rows = 0;
  for (int ci = 0; ci < L.ncomp; ++ci) {
    rp.rstart[ci] = rows;
    rows += L.c[ci].ny * L.c[ci].nz;
  }
  rp.rstart[L.ncomp] = rows;
  return rp;
}

// Work items of system S in phase P (0: the phase has no work for it).
long long batch_items(const BatchSysDev& S, const BatchPhase& P) {
  const int last = S.levels - 1, l = P.level;
  if (l > last) return 0;
  const LevelDev& L = S.lev[l].L;
  switch (P.type) {
    case kPhOuterRes:
      return (long long)S.orp.rstart[L.ncomp] * (L.c[0].nx >> 2);
    case kPhOuterUpd:
      return L.size / 4;
    case kPhSmooth:
      if (l == last) return 0;
      if (l == 0) return S.fcp.start[L.ncomp];
      return S.lev[l].v8 ? S.lev[l].sp[P.colour].start[L.ncomp] : S.lev[l].cp[P.colour].gstart[L.ncomp];
    case kPhCoarse1:
    case kPhCoarse2:   // 8 lanes per row / column, whole warps per system
      return l == last ? (8 * L.size + 31) / 32 * 32 : 0;
    case kPhResid:
      if (l == last) return 0;
      if (l == 0) return S.fcp.start[L.ncomp];
      return S.lev[l].rcp.kc > 0 ? S.lev[l].rcp.start[L.ncomp] : L.size;
    case kPhRestrict: {
      if (l == last) return 0;
      const BatchLevelDev& C = S.lev[l + 1];
      const long long nres =
          S.lev[l].vec_down ? (long long)C.rp.rstart[C.L.ncomp] * (C.L.c[0].nx >> 2) : C.L.size;
      return nres + C.L.size;
    }
    case kPhProlong:
      if (l == last) return 0;
      return S.lev[l].vec_up ? (long long)S.lev[l].rp.rstart[L.ncomp] * (L.c[0].nx >> 3) : L.size;
    default:
      return 0;
  }
}

template <typename T>
size_t batch_smem(int nsys) {
  return (size_t)nsys * sizeof(double);
}

}  // namespace

bool batch_persist_eligible(int nsys, const BatchSysHost* h) {
  for (int i = 0; i < nsys; ++i) {
    const BatchSysHost& q = h[i];
    if (q.levels < 2 || q.levels > kMaxLevels || !q.cholesky || q.esize != h[0].esize) return false;
    const LevelDev& L0 = q.lev[0];
    for (int ci = 0; ci < L0.ncomp; ++ci)
      if (L0.c[ci].nx % 8 != 0 || L0.c[ci].nx != L0.c[0].nx) return false;
    for (int l = 1; l < q.levels; ++l)
      for (int ci = 0; ci < q.lev[l].ncomp; ++ci)
        if (q.lev[l].c[ci].ncol > kBatchColours) return false;
  }
  return true;
}

cudaError_t batch_persist_configure(BatchPersist* bp, int kc, int bps) {
  if (!bp || kc < 1 || bps < 1) return cudaErrorInvalidValue;
  bp->kc = kc;
  // level-0 column items with chunks of kc rows
  for (BatchSysDev& S : bp->sys) {
    const LevelDev& L = S.lev[0].L;
    S.fcp = ColumnPass{};
    S.fcp.kc = kc;
    long long items = 0;
    for (int ci = 0; ci < L.ncomp; ++ci) {
      S.fcp.start[ci] = items;
      items += (long long)L.c[ci].ny * (L.c[ci].nx >> 3) * ((L.c[ci].nz + kc - 1) / kc);
    }
    S.fcp.start[L.ncomp] = items;
  }
  int lmax = 0;
  for (const BatchSysDev& S : bp->sys) lmax = lmax > S.levels ? lmax : S.levels;
  auto ncol_max = [&](int l) {
    if (l == 0) return 2;
    int m = 0;
    for (const BatchSysDev& S : bp->sys)
      if (l < S.levels - 1)
        for (int ci = 0; ci < S.lev[l].L.ncomp; ++ci) m = m > S.lev[l].L.c[ci].ncol ? m : S.lev[l].L.c[ci].ncol;
    return m;
  };
  auto any = [&](auto pred) {
    for (const BatchSysDev& S : bp->sys)
      if (pred(S.levels - 1)) return true;
    return false;
  };
  auto vcycle = [&](std::vector<BatchPhase>& v) {
    for (int l = 0; l < lmax; ++l) {
      if (any([&](int last) { return l < last; }))
        for (int q = 0; q < bp->mu1; ++q)
          for (int col = 0; col < ncol_max(l); ++col) v.push_back({kPhSmooth, l, q, col});
      if (any([&](int last) { return l == last; })) {
        v.push_back({kPhCoarse1, l, 0, 0});
        v.push_back({kPhCoarse2, l, 0, 0});
      }
      if (any([&](int last) { return l < last; })) {
        v.push_back({kPhResid, l, 0, 0});
        v.push_back({kPhRestrict, l, 0, 0});
      }
    }
    for (int l = lmax - 2; l >= 0; --l) {
      if (!any([&](int last) { return l < last; })) continue;
      v.push_back({kPhProlong, l, 0, 0});
      for (int q = 0; q < bp->mu2; ++q)
        for (int col = 0; col < ncol_max(l); ++col) v.push_back({kPhSmooth, l, bp->mu1 + q, col});
    }
  };
  for (int k = 0; k < 3; ++k) {
    std::vector<BatchPhase>& v = bp->ph[k];
    v.clear();
    if (k != 1) v.push_back({kPhOuterRes, 0, 0, 0});
    vcycle(v);
    v.push_back({kPhOuterUpd, 0, 0, 0});
    if (k == 1) v.push_back({kPhOuterRes, 0, 0, 0});
    std::vector<long long>& st = bp->st[k];
    st.assign(v.size() * (bp->nsys + 1), 0);
    for (size_t p = 0; p < v.size(); ++p) {
      long long acc = 0;
      for (int i = 0; i < bp->nsys; ++i) {
        st[p * (bp->nsys + 1) + i] = acc;
        acc += batch_items(bp->sys[i], v[p]);
      }
      st[p * (bp->nsys + 1) + bp->nsys] = acc;
    }
    if (bp->dph[k]) cudaFree(bp->dph[k]);
    if (bp->dst[k]) cudaFree(bp->dst[k]);
    bp->dph[k] = nullptr;
    bp->dst[k] = nullptr;
    cudaError_t e = cudaMalloc(&bp->dph[k], v.size() * sizeof(BatchPhase));
    if (e == cudaSuccess) e = cudaMalloc(&bp->dst[k], st.size() * sizeof(long long));
    if (e == cudaSuccess) e = cudaMemcpy(bp->dph[k], v.data(), v.size() * sizeof(BatchPhase), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(bp->dst[k], st.data(), st.size() * sizeof(long long), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaMemcpy(bp->dsys, bp->sys.data(), bp->sys.size() * sizeof(BatchSysDev), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  // co-resident blocks: bps per SM, if that many fit
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = (size_t)bp->nsys * sizeof(double) + (size_t)(bp->nsys + 1) * sizeof(long long);
  if (bp->esize == 4)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_fac<float, true>, kBatchThreads, smem);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_fac<double, true>, kBatchThreads, smem);
  if (e != cudaSuccess) return e;
  int occ2 = 0;
  if (bp->esize == 4)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k_batch_fac<float, false>, kBatchThreads, smem);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k_batch_fac<double, false>, kBatchThreads, smem);
  if (e != cudaSuccess) return e;
  occ = occ < occ2 ? occ : occ2;
  if (occ < 1) return cudaErrorNotSupported;
  bp->bps = bps < occ ? bps : occ;
  bp->blocks = bp->bps * sms;
  return cudaSuccess;
}

cudaError_t batch_persist_create(int nsys, const BatchSysHost* h, int mu1, int mu2, BatchPersist** out) {
  *out = nullptr;
  if (nsys < 1 || !batch_persist_eligible(nsys, h)) return cudaErrorNotSupported;
  BatchPersist* bp = new (std::nothrow) BatchPersist();
  if (!bp) return cudaErrorMemoryAllocation;
  bp->nsys = nsys;
  bp->esize = h[0].esize;
  bp->mu1 = mu1;
  bp->mu2 = mu2;
  bp->sys.resize(nsys);
  long long ywork = 0;
  for (int i = 0; i < nsys; ++i) ywork += h[i].lev[h[i].levels - 1].size;
  cudaError_t e = cudaMalloc(&bp->dsys, nsys * sizeof(BatchSysDev));
  if (e == cudaSuccess) e = cudaMalloc(&bp->ywork, (size_t)ywork * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&bp->norms, (size_t)nsys * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&bp->bar, 4 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(bp->norms, 0, (size_t)nsys * sizeof(double));
  if (e != cudaSuccess) {
    batch_persist_destroy(bp);
    return e;
  }
  long long yoff = 0;
  for (int i = 0; i < nsys; ++i) {
    const BatchSysHost& q = h[i];
    BatchSysDev& S = bp->sys[i];
    std::memset(&S, 0, sizeof(S));
    S.levels = q.levels;
    S.key = q.key;
    S.cyc[0] = q.cyc;
    S.cyc[1] = q.cyc + 1;
    S.chain_ctr = q.cyc;
    S.z[0] = q.xi;
    S.z[1] = q.u;
    S.bz[0] = nullptr;
    S.bz[1] = q.bvel;
    S.norm2 = bp->norms + i;
    S.ywork = bp->ywork + yoff;
    yoff += q.lev[q.levels - 1].size;
    for (int l = 0; l < q.levels; ++l) {
      BatchLevelDev& BL = S.lev[l];
      BL.L = q.lev[l];
      BL.v = q.v[l];
      BL.b = q.b[l];
      BL.t = q.t[l];
      BL.rp = rows_of(q.lev[l]);
      if (l >= 1) {
        const LevelDev& L = q.lev[l];
        BL.v8 = 1;
        bool four = true;
        for (int ci = 0; ci < L.ncomp; ++ci) {
          if (L.c[ci].nx % 8 != 0 || L.c[ci].mx != 2) BL.v8 = 0;
          if (L.c[ci].nx % 4 != 0) four = false;
        }
        for (int col = 0; col < kBatchColours; ++col) {
          BL.cp[col] = ColourPass{};
          colour_pass_of(L, col, &BL.cp[col]);
          ColumnPass& sp = BL.sp[col];
          sp = ColumnPass{};
          long long items = 0;
          for (int ci = 0; ci < L.ncomp; ++ci) {
            sp.start[ci] = items;
            if (BL.cp[col].nsites[ci] > 0) items += (long long)(L.c[ci].nx >> 3) * BL.cp[col].nyc[ci] * BL.cp[col].nzc[ci];
          }
          sp.start[L.ncomp] = items;
        }
        BL.rcp = ColumnPass{};
        if (four) {
          BL.rcp.kc = 8;
          long long items = 0;
          for (int ci = 0; ci < L.ncomp; ++ci) {
            BL.rcp.start[ci] = items;
            items += (long long)L.c[ci].ny * (L.c[ci].nx >> 2) * ((L.c[ci].nz + 7) / 8);
          }
          BL.rcp.start[L.ncomp] = items;
        }
      }
      BL.vec_up = l + 1 < q.levels && batch_vec_up(q.lev[l]) ? 1 : 0;
      BL.vec_down = l + 1 < q.levels && batch_vec_down(q.lev[l], q.lev[l + 1]) ? 1 : 0;
    }
    S.orp = S.lev[0].rp;
  }
  e = batch_persist_configure(bp, 16, 1);
  if (e != cudaSuccess) {
    batch_persist_destroy(bp);
    return e;
  }
  *out = bp;
  return cudaSuccess;
}

void batch_persist_destroy(BatchPersist* bp) {
  if (!bp) return;
  for (int k = 0; k < 3; ++k) {
    if (bp->dph[k]) cudaFree(bp->dph[k]);
    if (bp->dst[k]) cudaFree(bp->dst[k]);
  }
  if (bp->dsys) cudaFree(bp->dsys);
  if (bp->ywork) cudaFree(bp->ywork);
  if (bp->norms) cudaFree(bp->norms);
  if (bp->bar) cudaFree(bp->bar);
  delete bp;
}

const double* batch_persist_norms(const BatchPersist* bp) { return bp ? bp->norms : nullptr; }

int batch_persist_phases(const BatchPersist* bp, int kind, int* types, int* levels) {
  if (!bp || kind < 0 || kind > 2) return 0;
  const std::vector<BatchPhase>& v = bp->ph[kind];
  for (size_t p = 0; p < v.size(); ++p) {
    if (types) types[p] = v[p].type;
    if (levels) levels[p] = v[p].level;
  }
  return (int)v.size();
}

const unsigned* batch_persist_bar(const BatchPersist* bp) { return bp ? bp->bar : nullptr; }

void batch_persist_shape(const BatchPersist* bp, int* kc, int* bps) {
  *kc = bp ? bp->kc : 0;
  *bps = bp ? bp->bps : 0;
}

cudaError_t batch_persist_launch(BatchPersist* bp, int kind, cudaStream_t st, unsigned long long* tstamp) {
  if (!bp || kind < 0 || kind > 2) return cudaErrorInvalidValue;
  const int mode = kind == 0 ? 0 : 1;
  cudaError_t e = cudaMemsetAsync(bp->bar, 0, 4 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(bp->blocks);
  cfg.blockDim = dim3(kBatchThreads);
  cfg.dynamicSmemBytes = (size_t)bp->nsys * sizeof(double) + (size_t)(bp->nsys + 1) * sizeof(long long);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const BatchSysDev* sys = bp->dsys;
  const int nsys = bp->nsys, nph = (int)bp->ph[kind].size();
  const BatchPhase* ph = bp->dph[kind];
  const long long* stt = bp->dst[kind];
  prof::Scope ps(SELM_K_BATCH_CYCLE, st);
  if (bp->esize == 4) {
    if (mode == 0) return cudaLaunchKernelEx(&cfg, k_batch_fac<float, true>, sys, nsys, ph, nph, stt, bp->bar, mode, tstamp);
    return cudaLaunchKernelEx(&cfg, k_batch_fac<float, false>, sys, nsys, ph, nph, stt, bp->bar, mode, tstamp);
  }
  if (mode == 0) return cudaLaunchKernelEx(&cfg, k_batch_fac<double, true>, sys, nsys, ph, nph, stt, bp->bar, mode, tstamp);
  return cudaLaunchKernelEx(&cfg, k_batch_fac<double, false>, sys, nsys, ph, nph, stt, bp->bar, mode, tstamp);
}

// Blocks of a cooperative level launch on the current device: one per SM
// when a block of CoopThreads<T> threads fits, else 0 (not supported).
template <typename T>
int coop_blocks() {
  static std::atomic<int> cached[64];
  static std::atomic<bool> init[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (init[dev].load()) return cached[dev].load();
  int sms = 0, coop = 0, occ1 = 0, occ2 = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ1, k_level_coop<T, true>, CoopThreads<T>::value, 0) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, k_level_coop<T, false>, CoopThreads<T>::value, 0) !=
          cudaSuccess) {
    cudaGetLastError();
    occ1 = occ2 = 0;
  }
  const int blocks = coop && occ1 >= 1 && occ2 >= 1 ? sms : 0;
  cached[dev].store(blocks);
  init[dev].store(true);
  return blocks;
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
// Column items of the level-0 z-marching kernels (nx % 8 == 0): chunks of kc
// z rows, kc halving (down to 4) while fewer than 96K threads would run.
long long fine_column_pass(const LevelDev& L, ColumnPass* cp) {
  long long cols = 0;
  int nzmax = 0;
  for (int ci = 0; ci < L.ncomp; ++ci) {
    cols += (long long)L.c[ci].ny * (L.c[ci].nx >> 3);
    nzmax = nzmax > L.c[ci].nz ? nzmax : L.c[ci].nz;
  }
  cp->kc = 16;
  while (cp->kc > 4 && cols * ((nzmax + cp->kc - 1) / cp->kc) < 96 * 1024) cp->kc /= 2;
  long long items = 0;
  for (int ci = 0; ci < L.ncomp; ++ci) {
    cp->start[ci] = items;
    items += (long long)L.c[ci].ny * (L.c[ci].nx >> 3) * ((L.c[ci].nz + cp->kc - 1) / cp->kc);
  }
  cp->start[L.ncomp] = items;
  return items;
}

template <typename T>
cudaError_t launch_smooth(const LevelDev& L, T* v, const T* b, int sweep, bool noise, Key key,
                          const unsigned long long* cyc, cudaStream_t st) {
  if (L.level == 0 && L.c[0].nx % 8 == 0) {
    ColumnPass cp{};
    const long long items = fine_column_pass(L, &cp);
    for (int colour = 0; colour < 2; ++colour) {
      prof::Scope ps(SELM_K_FINE_SWEEP, st);
      if (noise)
        LTRY(launch_pdl(k_fine_colour_zm<T, true>, grid_for(items), kBlock, st, L, cp, v, b, colour, sweep, key, cyc));
      else
        LTRY(launch_pdl(k_fine_colour_zm<T, false>, grid_for(items), kBlock, st, L, cp, v, b, colour, sweep, key, cyc));
    }
    return cudaGetLastError();
  }
  if (L.level == 0) {
    for (int colour = 0; colour < 2; ++colour) {
      ColourPass cp{};
      long long gs = 0;
      for (int ci = 0; ci < L.ncomp; ++ci) {
        const CompDev& c = L.c[ci];
        cp.gstart[ci] = gs;
        cp.nsites[ci] = (long long)(c.nx / 2) * c.ny * c.nz;
        gs += (cp.nsites[ci] + 3) / 4;
      }
      cp.gstart[L.ncomp] = gs;
      prof::Scope ps(SELM_K_FINE_SWEEP, st);
      if (noise)
        k_fine_colour<T, true><<<grid_for(gs), kBlock, 0, st>>>(L, cp, v, b, colour, sweep, key, cyc);
      else
        k_fine_colour<T, false><<<grid_for(gs), kBlock, 0, st>>>(L, cp, v, b, colour, sweep, key, cyc);
    }
    return cudaGetLastError();
  }
  if (L.rb && L.c[0].nx % 8 == 0) {
    // banded 7-point level: march along z (chunks of 16 rows)
    ColumnPass cp{};
    cp.kc = 16;
    long long items = 0;
    for (int ci = 0; ci < L.ncomp; ++ci) {
      cp.start[ci] = items;
      items += (long long)L.c[ci].ny * (L.c[ci].nx >> 3) * ((L.c[ci].nz + cp.kc - 1) / cp.kc);
    }
    cp.start[L.ncomp] = items;
    for (int colour = 0; colour < 2; ++colour) {
      prof::Scope ps(SELM_K_COARSE_SWEEP, st);
      if (noise)
        LTRY(launch_pdl(k_band7_rb_zm<T, true>, grid_for(items), kBlock, st, L, cp, v, b, colour, sweep, key, cyc));
      else
        LTRY(launch_pdl(k_band7_rb_zm<T, false>, grid_for(items), kBlock, st, L, cp, v, b, colour, sweep, key, cyc));
    }
    return cudaGetLastError();
  }
  if (L.rb) {
    ColourPass cp{};
    long long gs = 0;
    for (int ci = 0; ci < L.ncomp; ++ci) {
      cp.gstart[ci] = gs;
      gs += (long long)(L.c[ci].nx / 2) * L.c[ci].ny * L.c[ci].nz;
    }
    cp.gstart[L.ncomp] = gs;
    for (int colour = 0; colour < 2; ++colour) {
      prof::Scope ps(SELM_K_COARSE_SWEEP, st);
      if (noise)
        k_band_rb<T, true><<<grid_for(gs), kBlock, 0, st>>>(L, cp, v, b, colour, sweep, key, cyc);
      else
        k_band_rb<T, false><<<grid_for(gs), kBlock, 0, st>>>(L, cp, v, b, colour, sweep, key, cyc);
    }
    return cudaGetLastError();
  }
  int maxcol = 0;
  for (int ci = 0; ci < L.ncomp; ++ci) maxcol = maxcol > L.c[ci].ncol ? maxcol : L.c[ci].ncol;
  bool v8 = true;   // 8-wide rows, x modulus 2: four class sites (one noise group) per thread
  for (int ci = 0; ci < L.ncomp; ++ci)
    if (L.c[ci].nx % 8 != 0 || L.c[ci].mx != 2) v8 = false;
  for (int q = 0; q < maxcol; ++q) {
    ColourPass cp{};
    const long long gs = colour_pass_of(L, q, &cp);
    if (gs == 0) continue;
    prof::Scope ps(SELM_K_COARSE_SWEEP, st);
    if (v8) {
      ColumnPass sp{};
      long long items = 0;
      for (int ci = 0; ci < L.ncomp; ++ci) {
        sp.start[ci] = items;
        if (cp.nsites[ci] > 0) items += (long long)(L.c[ci].nx >> 3) * cp.nyc[ci] * cp.nzc[ci];
      }
      sp.start[L.ncomp] = items;
      const int cx = q % 2;   // every component has x modulus 2
      if (noise && cx == 0)
        LTRY(launch_pdl(k_coarse_colour_v8<T, true, 0>, grid_for(items), kBlock, st, L, cp, sp, v, b, sweep, key, cyc));
      else if (noise)
        LTRY(launch_pdl(k_coarse_colour_v8<T, true, 1>, grid_for(items), kBlock, st, L, cp, sp, v, b, sweep, key, cyc));
      else if (cx == 0)
        LTRY(launch_pdl(k_coarse_colour_v8<T, false, 0>, grid_for(items), kBlock, st, L, cp, sp, v, b, sweep, key, cyc));
      else
        LTRY(launch_pdl(k_coarse_colour_v8<T, false, 1>, grid_for(items), kBlock, st, L, cp, sp, v, b, sweep, key, cyc));
      continue;
    }
    if (noise)
      k_coarse_site<T, true><<<grid_for(gs), kBlock, 0, st>>>(L, cp, v, b, sweep, key, cyc);
    else
      k_coarse_site<T, false><<<grid_for(gs), kBlock, 0, st>>>(L, cp, v, b, sweep, key, cyc);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_residual(const LevelDev& L, const T* v, const T* b, T* t, cudaStream_t st) {
  prof::Scope ps(SELM_K_RESIDUAL, st);
  if (L.level == 0 && L.c[0].nx % 8 == 0) {
    ColumnPass cp{};
    const long long items = fine_column_pass(L, &cp);
    LTRY(launch_pdl(k_fine_residual_zm<T>, grid_for(items), kBlock, st, L, cp, v, b, t));
    return cudaGetLastError();
  }
  if (L.rb && L.c[0].nx % 8 == 0) {
    ColumnPass cp{};
    cp.kc = 16;
    long long items = 0;
    for (int ci = 0; ci < L.ncomp; ++ci) {
      cp.start[ci] = items;
      items += (long long)L.c[ci].ny * (L.c[ci].nx >> 3) * ((L.c[ci].nz + cp.kc - 1) / cp.kc);
    }
    cp.start[L.ncomp] = items;
    LTRY(launch_pdl(k_band7_residual_zm<T>, grid_for(items), kBlock, st, L, cp, v, b, t));
    return cudaGetLastError();
  }
  bool four = L.level >= 1 && !L.rb;
  for (int ci = 0; ci < L.ncomp; ++ci)
    if (L.c[ci].nx % 4 != 0) four = false;
  if (four) {   // Galerkin level: separable form along z columns of 4-wide segments
    ColumnPass cp{};
    cp.kc = 8;
    long long items = 0;
    for (int ci = 0; ci < L.ncomp; ++ci) {
      cp.start[ci] = items;
      items += (long long)L.c[ci].ny * (L.c[ci].nx >> 2) * ((L.c[ci].nz + cp.kc - 1) / cp.kc);
    }
    cp.start[L.ncomp] = items;
    LTRY(launch_pdl(k_galerkin_residual_zm<T>, grid_for(items), kBlock, st, L, cp, v, b, t));
    return cudaGetLastError();
  }
  k_residual<T><<<grid_for(L.size), kBlock, 0, st>>>(L, v, b, t);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_restrict(const LevelDev& Lf, const LevelDev& Lc, const T* t, T* bc, cudaStream_t st) {
  prof::Scope ps(SELM_K_RESTRICT, st);
  bool v4 = Lf.c[0].nx % 8 == 0;
  for (int ci = 0; ci < Lf.ncomp; ++ci)
    if (Lf.c[ci].nx != Lf.c[0].nx || Lc.c[ci].nx * 2 != Lf.c[ci].nx) v4 = false;
  if (v4) {
    RowPass rp{};
    int rows = 0;
    for (int ci = 0; ci < Lc.ncomp; ++ci) {
      rp.rstart[ci] = rows;
      rows += Lc.c[ci].ny * Lc.c[ci].nz;
    }
    rp.rstart[Lc.ncomp] = rows;
    LTRY(launch_pdl(k_restrict_v4<T>, grid_for((long long)rows * (Lc.c[0].nx >> 2)), kBlock, st, Lf, Lc, rp, t, bc));
    return cudaGetLastError();
  }
  k_restrict<T><<<grid_for(Lc.size), kBlock, 0, st>>>(Lf, Lc, t, bc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_prolong(const LevelDev& Lf, const LevelDev& Lc, T* v, const T* vc, cudaStream_t st) {
  prof::Scope ps(SELM_K_PROLONG, st);
  if (Lf.c[0].nx % 8 == 0) {
    RowPass rp{};
    int rows = 0;
    for (int ci = 0; ci < Lf.ncomp; ++ci) {
      rp.rstart[ci] = rows;
      rows += Lf.c[ci].ny * Lf.c[ci].nz;
    }
    rp.rstart[Lf.ncomp] = rows;
    LTRY(launch_pdl(k_prolong_v8<T>, grid_for((long long)rows * (Lf.c[0].nx >> 3)), kBlock, st, Lf, Lc, rp, v, vc));
    return cudaGetLastError();
  }
  k_prolong<T><<<grid_for(Lf.size), kBlock, 0, st>>>(Lf, Lc, v, vc);
  return cudaGetLastError();
}

template <typename T>
bool level_coop_supported(const LevelDev& L) {
  if (L.level < 1) return false;
  for (int ci = 0; ci < L.ncomp; ++ci)
    if (L.c[ci].ncol > kMaxCoopColours) return false;
  return coop_blocks<T>() > 0;
}

template <typename T>
cudaError_t launch_level_coop(const LevelDev& L, const LevelDev& Lc, int phase, int mu1, int mu2, T* v, const T* b,
                              T* t, T* bc, T* vc, unsigned* bar, bool flow, bool noise, Key key,
                              const unsigned long long* cyc, cudaStream_t st) {
  const int blocks = coop_blocks<T>();
  if (blocks <= 0 || !level_coop_supported<T>(L)) return cudaErrorNotSupported;
  CoopLevel<T> P{};
  P.L = L;
  P.Lc = Lc;
  int maxcol = 0;
  for (int ci = 0; ci < L.ncomp; ++ci) maxcol = maxcol > L.c[ci].ncol ? maxcol : L.c[ci].ncol;
  P.ncolour = maxcol;
  for (int q = 0; q < maxcol; ++q) colour_pass_of(L, q, &P.cp[q]);
  // residual items: 2-wide x segments of z chunks, the shortest chunk (>= 4
  // rows) that leaves at most one item per thread
  P.rcp = ColumnPass{};
  bool even = true;
  for (int ci = 0; ci < L.ncomp; ++ci)
    if (L.c[ci].nx % 2 != 0) even = false;
  if (even) {
    const long long nth = (long long)blocks * CoopThreads<T>::value;
    for (int kc = 4; kc <= 64; kc *= 2) {
      long long items = 0;
      for (int ci = 0; ci < L.ncomp; ++ci) {
        P.rcp.start[ci] = items;
        items += (long long)L.c[ci].ny * (L.c[ci].nx >> 1) * ((L.c[ci].nz + kc - 1) / kc);
      }
      P.rcp.start[L.ncomp] = items;
      P.rcp.kc = kc;
      if (items <= nth) break;
    }
  }
  P.flow = flow && sizeof(T) == 4 && L.flow ? 1 : 0;
  P.vec = L.c[0].nx % 8 == 0 ? 1 : 0;
  for (int ci = 0; ci < L.ncomp; ++ci)
    if (L.c[ci].nx != L.c[0].nx || Lc.c[ci].nx * 2 != L.c[ci].nx) P.vec = 0;
  {
    int rows = 0, crows = 0;
    for (int ci = 0; ci < L.ncomp; ++ci) {
      P.frp.rstart[ci] = rows;
      P.crp.rstart[ci] = crows;
      rows += L.c[ci].ny * L.c[ci].nz;
      crows += Lc.c[ci].ny * Lc.c[ci].nz;
    }
    P.frp.rstart[L.ncomp] = rows;
    P.crp.rstart[L.ncomp] = crows;
  }
  if (P.flow) {
    auto mod = [](int d, int m) { return ((d % m) + m) % m; };
    for (int q = 0; q < maxcol; ++q)
      for (int ci = 0; ci < L.ncomp; ++ci) {
        const CompDev& c = L.c[ci];
        unsigned long long check = 0ull, early = 0ull;
        if (q < c.ncol) {
          const int cx = q % c.mx, cy = (q / c.mx) % c.my, cz = q / (c.mx * c.my);
          for (int dz = -2; dz <= 2; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
              for (int dx = -1; dx <= 1; ++dx) {
                const int w = (dy + 1) * 3 + dx + 1, o = (dz + 2) * 9 + w;
                if ((dz == 0 && w == 4) || (c.ny == 1 && dy != 0) || (c.w1f[w] == 0.f && c.w2f[w] == 0.f)) continue;
                check |= 1ull << o;
                const int qn = mod(cx + dx, c.mx) + c.mx * (mod(cy + dy, c.my) + c.my * mod(cz + dz, c.mz));
                if (qn < q) early |= 1ull << o;
              }
        }
        P.fcheck[q][ci] = check;
        P.fearly[q][ci] = early;
      }
  }
  P.v = v;
  P.b = b;
  P.t = t;
  P.bc = bc;
  P.vc = vc;
  P.bar = bar;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(CoopThreads<T>::value);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  prof::Scope ps(SELM_K_COARSE_SWEEP, st);
  if (noise) return cudaLaunchKernelEx(&cfg, k_level_coop<T, true>, P, phase, mu1, mu2, key, cyc);
  return cudaLaunchKernelEx(&cfg, k_level_coop<T, false>, P, phase, mu1, mu2, key, cyc);
}

template <typename T>
cudaError_t launch_coarsest(const LevelDev& L, T* v, const T* b, bool noise, Key key,
                            const unsigned long long* cyc, cudaStream_t st) {
  int nmax = 0;
  for (int ci = 0; ci < L.ncomp; ++ci) {
    const int N = L.c[ci].nx * L.c[ci].ny * L.c[ci].nz;
    nmax = N > nmax ? N : nmax;
  }
  const size_t smem = 2 * (size_t)nmax * sizeof(double);
  prof::Scope ps(SELM_K_COARSEST, st);
  if (noise)
    k_coarsest<T, true><<<L.ncomp, 256, smem, st>>>(L, v, b, key, cyc);
  else
    k_coarsest<T, false><<<L.ncomp, 256, smem, st>>>(L, v, b, key, cyc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_outer_residual(const LevelDev& L0, const double* z, const double* b, T* r, double* norm2,
                                  cudaStream_t st) {
  prof::Scope ps(SELM_K_OUTER_RESIDUAL, st);
  if (L0.c[0].nx % 4 == 0) {
    RowPass rp{};
    int rows = 0;
    for (int ci = 0; ci < L0.ncomp; ++ci) {
      rp.rstart[ci] = rows;
      rows += L0.c[ci].ny * L0.c[ci].nz;
    }
    rp.rstart[L0.ncomp] = rows;
    const long long nt = (long long)rows * (L0.c[0].nx >> 2);
    if constexpr (sizeof(T) == 4) {
      const bool aligned = ((uintptr_t)r & 15u) == 0 && L0.c[L0.ncomp - 1].off % 4 == 0 &&
                           (L0.ncomp == 1 || L0.c[1].off % 4 == 0);
      if (!aligned && norm2)
        LTRY(launch_pdl(k_outer_residual_v4<T, true>, grid_for(nt), kBlock, st, L0, rp, z, b, r, norm2));
      else if (!aligned)
        LTRY(launch_pdl(k_outer_residual_v4<T, false>, grid_for(nt), kBlock, st, L0, rp, z, b, r, norm2));
      else if (norm2)
        LTRY(launch_pdl(k_outer_residual_fx<true>, grid_for(nt), kBlock, st, L0, rp, z, b, r, norm2));
      else
        LTRY(launch_pdl(k_outer_residual_fx<false>, grid_for(nt), kBlock, st, L0, rp, z, b, r, norm2));
      return cudaGetLastError();
    }
    if (norm2)
      LTRY(launch_pdl(k_outer_residual_v4<T, true>, grid_for(nt), kBlock, st, L0, rp, z, b, r, norm2));
    else
      LTRY(launch_pdl(k_outer_residual_v4<T, false>, grid_for(nt), kBlock, st, L0, rp, z, b, r, norm2));
    return cudaGetLastError();
  }
  k_outer_residual<T><<<grid_for(L0.size), kBlock, 0, st>>>(L0, z, b, r, norm2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_outer_update(long long n, double* z, const T* d, cudaStream_t st) {
  prof::Scope ps(SELM_K_OUTER_UPDATE, st);
  if (n % 4 == 0) {
    LTRY(launch_pdl(k_outer_update_v4<T>, grid_for(n / 4), kBlock, st, n / 4, z, d));
    return cudaGetLastError();
  }
  k_outer_update<T><<<grid_for(n), kBlock, 0, st>>>(n, z, d);
  return cudaGetLastError();
}

cudaError_t launch_norm2(long long n, const double* x, double* out, cudaStream_t st) {
  long long blocks = grid_for(n);
  if (blocks > 4 * 152) blocks = 4 * 152;
  if (blocks < 1) blocks = 1;
  prof::Scope ps(SELM_K_OTHER, st);
  k_norm2<<<(unsigned)blocks, kBlock, 0, st>>>(n, x, out);
  return cudaGetLastError();
}

cudaError_t launch_axpby(long long n, double a, const double* x, double c, const double* y, double* out,
                         cudaStream_t st) {
  prof::Scope ps(SELM_K_OTHER, st);
  k_axpby<<<grid_for(n), kBlock, 0, st>>>(n, a, x, c, y, out);
  return cudaGetLastError();
}

cudaError_t launch_set_u64(unsigned long long* p, unsigned long long v, cudaStream_t st) {
  prof::Scope ps(SELM_K_OTHER, st);
  k_set_u64<<<1, 1, 0, st>>>(p, v);
  return cudaGetLastError();
}

cudaError_t launch_inc_u64(unsigned long long* p, cudaStream_t st) {
  prof::Scope ps(SELM_K_OTHER, st);
  k_inc_u64<<<1, 1, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_spread(const LevelDev& L0, int n, int dim, int np, const double* X, const double* F, double* b,
                          cudaStream_t st) {
  if (np <= 0) return cudaSuccess;
  const long long nt = (long long)np * L0.ncomp * 32;   // one warp per (particle, component)
  prof::Scope ps(SELM_K_SPREAD, st);
  k_spread<<<grid_for(nt), kBlock, 0, st>>>(L0, n, dim, np, X, F, b);
  return cudaGetLastError();
}

cudaError_t launch_interp(const LevelDev& L0, int n, int dim, int np, const double* X, const double* u, double* U,
                          cudaStream_t st) {
  if (np <= 0) return cudaSuccess;
  const long long nt = (long long)np * L0.ncomp * 32;
  prof::Scope ps(SELM_K_INTERP, st);
  k_interp<<<grid_for(nt), kBlock, 0, st>>>(L0, n, dim, np, X, u, U);
  return cudaGetLastError();
}

cudaError_t launch_em(int np, int dim, double* X, const double* V, cudaStream_t st) {
  if (np <= 0) return cudaSuccess;
  prof::Scope ps(SELM_K_OTHER, st);
  k_em<<<grid_for(np), kBlock, 0, st>>>(np, dim, X, V);
  return cudaGetLastError();
}

cudaError_t launch_divergence(const LevelDev& Lv, const double* w, double* div, double* sum, cudaStream_t st) {
  const long long N = (long long)Lv.c[0].nx * Lv.c[0].ny * Lv.c[0].nz;
  if (N >= (1ll << 31)) return cudaErrorInvalidValue;
  prof::Scope ps(SELM_K_PROJECTION, st);
  const unsigned g0 = grid_for(N), grid = g0 < 4 * 152 ? g0 : 4 * 152;
  k_divergence<<<grid, kBlock, 0, st>>>(Lv, w, div, sum);
  return cudaGetLastError();
}

cudaError_t launch_sub_mean(long long n, double* x, const double* sum, cudaStream_t st) {
  prof::Scope ps(SELM_K_PROJECTION, st);
  k_sub_mean<<<grid_for(n), kBlock, 0, st>>>(n, x, sum);
  return cudaGetLastError();
}

cudaError_t launch_grad_sub(const LevelDev& Lv, double* w, const double* phi, cudaStream_t st) {
  prof::Scope ps(SELM_K_PROJECTION, st);
  k_grad_sub<<<grid_for(Lv.size), kBlock, 0, st>>>(Lv, w, phi);
  return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, Key key, uint32_t* out, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  prof::Scope ps(SELM_K_OTHER, st);
  k_philox<<<grid_for(n), kBlock, 0, st>>>(ctr, key, out, n);
  return cudaGetLastError();
}

#define SELM_INSTANTIATE(T)                                                                                  \
  template cudaError_t launch_smooth<T>(const LevelDev&, T*, const T*, int, bool, Key,                      \
                                        const unsigned long long*, cudaStream_t);                           \
  template cudaError_t launch_residual<T>(const LevelDev&, const T*, const T*, T*, cudaStream_t);           \
  template cudaError_t launch_restrict<T>(const LevelDev&, const LevelDev&, const T*, T*, cudaStream_t);    \
  template cudaError_t launch_prolong<T>(const LevelDev&, const LevelDev&, T*, const T*, cudaStream_t);     \
  template bool level_coop_supported<T>(const LevelDev&);                                                   \
  template cudaError_t launch_level_coop<T>(const LevelDev&, const LevelDev&, int, int, int, T*, const T*, T*, T*, \
                                            T*, unsigned*, bool, bool, Key, const unsigned long long*,            \
                                            cudaStream_t);                                                        \
  template cudaError_t launch_coarsest<T>(const LevelDev&, T*, const T*, bool, Key,                         \
                                          const unsigned long long*, cudaStream_t);                         \
  template cudaError_t launch_outer_residual<T>(const LevelDev&, const double*, const double*, T*, double*, \
                                                cudaStream_t);                                              \
  template cudaError_t launch_outer_update<T>(long long, double*, const T*, cudaStream_t);

SELM_INSTANTIATE(float)
SELM_INSTANTIATE(double)

}  // namespace selm

extern "C" {

long long selm_kernel_launches(void) { return selm::prof::g_launches.load(); }

selm_status selm_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(selm::prof::g_mu);
  selm::prof::g_on = on != 0;
  return SELM_OK;
}

selm_status selm_profile_reset(void) {
  std::lock_guard<std::mutex> lk(selm::prof::g_mu);
  selm::prof::drain();
  for (int k = 0; k < SELM_K_NCLASSES; ++k) {
    selm::prof::g_ms[k] = 0.0;
    selm::prof::g_count[k] = 0;
  }
  return SELM_OK;
}

selm_status selm_profile_read(int kernel_class, double* total_ms, long long* launches) {
  if (kernel_class < 0 || kernel_class >= SELM_K_NCLASSES) return SELM_EINVAL;
  std::lock_guard<std::mutex> lk(selm::prof::g_mu);
  selm::prof::drain();
  if (total_ms) *total_ms = selm::prof::g_ms[kernel_class];
  if (launches) *launches = selm::prof::g_count[kernel_class];
  return SELM_OK;
}

}  // extern "C"
