// Spectral inner solve of the projection's pressure problem on the uniform
// channel.
//
// The projection P~ = I - G (DG)^+ D of Section 4 needs the Neumann pressure
// problem (D^ D^T) phi = D^ w.  On the uniform channel that operator is the
// Kronecker sum of the periodic second difference along x and y and the
// cell-centred Neumann second difference along z, so Fourier modes along x
// and y diagonalise it and leave, for every mode (mx, my), the tridiagonal
// system
//     (lambda(mx) + lambda(my)) phi^ + T_z phi^ = r^,
//     lambda(m) = 2 - 2 cos(2 pi m / n),  T_z = tridiag(-1, 2, -1), ends 1
// along z.  The solve used inside FP64 iterative refinement (the projection's
// FAC iteration of Algorithm 1 with this solve in place of the V-cycle) is:
//   1. forward 2-D FFT of every z plane of the FP32 residual (one CTA per
//      plane, the plane in shared memory, radix-2 decimation in frequency:
//      modes come out in bit-reversed order, which nothing needs to undo);
//   2. per mode, the z system solved by the Thomas algorithm in FP32 (the
//      all-constant mode (0, 0) is singular: its z = 0 value is pinned to 0,
//      which fixes the pressure's free constant, and its column -- the
//      worst-conditioned one -- is solved exactly in FP64 by two scans);
//   3. inverse 2-D FFT of every plane (decimation in time, bit-reversed in,
//      natural out); the real part / n^2 is the correction.
// Grids: 3-D, nx == ny == n a power of two, 4 <= n <= 128; nz >= 2.

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "../../include/selm_mg.h"
#include "selm_internal.h"
#include "selm_launch.h"
#include "selm_prof.h"

namespace selm {
namespace {

constexpr int kSpecThreads = 512;
constexpr int kThomasThreads = 128;

__device__ __forceinline__ int bitrev(int x, int logn) { return (int)(__brev((unsigned)x) >> (32 - logn)); }

// twiddles W[j] = exp(-2 pi i j / n), j < n / 2
__device__ void make_twiddles(float2* W, int n) {
  for (int j = threadIdx.x; j < (n >> 1); j += blockDim.x) {
    float s, c;
    sincospif(-2.0f * (float)j / (float)n, &s, &c);
    W[j] = make_float2(c, s);
  }
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Butterfly q of a stage over all rows (columns == false: along x) or all
// columns (along y) of an n x n plane: line and pair index, with consecutive
// threads on consecutive addresses in both cases.  n = 2^logn and
// half = 2^lh, so the index arithmetic is shifts and masks.
__device__ __forceinline__ void stage_index(int q, int logn, int lh, bool columns, int* a0, int* a1, int* j) {
  const int n = 1 << logn;
  const int line = columns ? (q & (n - 1)) : (q >> (logn - 1));
  const int p = columns ? (q >> logn) : (q & ((n >> 1) - 1));
  const int grp = p >> lh;
  *j = p & ((1 << lh) - 1);
  const int i0 = (grp << (lh + 1)) + *j, i1 = i0 + (1 << lh);
  *a0 = columns ? (i0 << logn) + line : (line << logn) + i0;
  *a1 = columns ? (i1 << logn) + line : (line << logn) + i1;
}

// Forward transform along one axis, decimation in frequency: natural order in,
// bit-reversed order out.
__device__ void fft_dif(float2* A, const float2* W, int n, int logn, bool columns) {
  for (int s = logn; s >= 1; --s) {
    const int lh = s - 1, tw_shift = logn - s;
    for (int q = threadIdx.x; q < n * (n >> 1); q += blockDim.x) {
      int a0, a1, j;
      stage_index(q, logn, lh, columns, &a0, &a1, &j);
      const float2 x0 = A[a0], x1 = A[a1];
      A[a0] = make_float2(x0.x + x1.x, x0.y + x1.y);
      A[a1] = cmul(make_float2(x0.x - x1.x, x0.y - x1.y), W[j << tw_shift]);
    }
    __syncthreads();
  }
}

// Inverse transform (unscaled) along one axis, decimation in time:
// bit-reversed order in, natural order out.
__device__ void fft_dit_inv(float2* A, const float2* W, int n, int logn, bool columns) {
  for (int s = 1; s <= logn; ++s) {
    const int lh = s - 1, tw_shift = logn - s;
    for (int q = threadIdx.x; q < n * (n >> 1); q += blockDim.x) {
      int a0, a1, j;
      stage_index(q, logn, lh, columns, &a0, &a1, &j);
      float2 w = W[j << tw_shift];
      w.y = -w.y;   // exp(+2 pi i j / (2 half))
      const float2 x0 = A[a0], t = cmul(A[a1], w);
      A[a0] = make_float2(x0.x + t.x, x0.y + t.y);
      A[a1] = make_float2(x0.x - t.x, x0.y - t.y);
    }
    __syncthreads();
  }
}

// Forward: plane k of r (FP32, [nz][n][n]) -> spectrum S[k][.][.] with both
// mode indices in bit-reversed order (the solve along z does not care; the
// inverse transform takes that order as it comes).
__global__ void __launch_bounds__(kSpecThreads) k_spec_forward(const float* __restrict__ r, float2* __restrict__ S,
                                                               int n, int logn) {
  extern __shared__ float2 sm[];
  float2* A = sm;
  float2* W = sm + n * n;
  const int k = blockIdx.x;
  const float* rp = r + (long long)k * n * n;
  make_twiddles(W, n);
  // eight loads in flight per thread before their stores (n * n is a
  // multiple of 8 * blockDim for the supported sizes, else the tail loop)
  int q = threadIdx.x;
  for (; q + 7 * (int)blockDim.x < n * n; q += 8 * blockDim.x) {
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = rp[q + e * blockDim.x];
#pragma unroll
    for (int e = 0; e < 8; ++e) A[q + e * blockDim.x] = make_float2(v[e], 0.0f);
  }
  for (; q < n * n; q += blockDim.x) A[q] = make_float2(rp[q], 0.0f);
  __syncthreads();
  fft_dif(A, W, n, logn, false);
  fft_dif(A, W, n, logn, true);
  float2* Sp = S + (long long)k * n * n;
  for (int q = threadIdx.x; q < n * n; q += blockDim.x) Sp[q] = A[q];
}

// Inverse: spectrum plane k -> delta (FP32 real part / n^2).
__global__ void __launch_bounds__(kSpecThreads) k_spec_inverse(const float2* __restrict__ S, float* __restrict__ d,
                                                               int n, int logn) {
  extern __shared__ float2 sm[];
  float2* A = sm;
  float2* W = sm + n * n;
  const int k = blockIdx.x;
  const float2* Sp = S + (long long)k * n * n;
  make_twiddles(W, n);
  int q = threadIdx.x;
  for (; q + 7 * (int)blockDim.x < n * n; q += 8 * blockDim.x) {
    float2 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = Sp[q + e * blockDim.x];
#pragma unroll
    for (int e = 0; e < 8; ++e) A[q + e * blockDim.x] = v[e];
  }
  for (; q < n * n; q += blockDim.x) A[q] = Sp[q];
  __syncthreads();
  fft_dit_inv(A, W, n, logn, false);
  fft_dit_inv(A, W, n, logn, true);
  const float inv = 1.0f / (float)(n * n);
  float* dp = d + (long long)k * n * n;
  for (int q = threadIdx.x; q < n * n; q += blockDim.x) dp[q] = A[q].x * inv;
}

// Thomas algorithm along z for the modes stored at (row py, column px)
// (mode indices bit-reversed), one thread per column, in place in S, in FP32.
// Shared memory: per thread, the forward sweep's c' and the column
// ([nz][threads] each).  The all-constant mode (0, 0) is singular; the extra
// last block solves it alone (one warp, FP64): its z = 0 value is pinned to 0,
// which fixes the pressure's free constant, and the remaining rows of the
// Neumann T_z are a flux balance, g_k = x_k - x_{k-1} = sum_{j >= k} d_j and
// x_k = sum_{i <= k} g_i -- two scans.
__global__ void __launch_bounds__(kThomasThreads) k_spec_thomas(float2* __restrict__ S, int n, int logn, int nz,
                                                                float inv_scale) {
  extern __shared__ float tsm[];
  const int t = threadIdx.x;
  const int per_row = n / (int)blockDim.x > 0 ? n / (int)blockDim.x : 1;
  const long long plane = (long long)n * n;
  if (blockIdx.x == (unsigned)(n * per_row)) {   // the (0, 0) mode, stored at column 0 of row 0
    if (t >= 32) return;
    const int rows = nz - 1;                      // unknowns x_1 .. x_{nz-1}
    const int per = (rows + 31) / 32;             // consecutive rows per lane
    double gx[8], gy[8];                          // nz <= 257
    const int k0 = 1 + t * per;
    double sx = 0.0, sy = 0.0;
    // suffix sums of d within the lane's rows, then across lanes
    for (int e = per - 1; e >= 0; --e) {
      const int k = k0 + e;
      if (k < nz) {
        const float2 f = S[k * plane];
        sx += (double)f.x * inv_scale;
        sy += (double)f.y * inv_scale;
      }
      gx[e] = sx;
      gy[e] = sy;
    }
    // exclusive suffix scan of the lane totals over higher lanes
    double tx = sx, ty = sy;
    for (int o = 1; o < 32; o <<= 1) {
      const double ux = __shfl_down_sync(0xffffffffu, tx, o), uy = __shfl_down_sync(0xffffffffu, ty, o);
      if (t + o < 32) {
        tx += ux;
        ty += uy;
      }
    }
    const double hx = tx - sx, hy = ty - sy;   // sum over higher lanes
    double px_ = 0.0, py_ = 0.0;
    for (int e = 0; e < per; ++e) {
      gx[e] += hx;
      gy[e] += hy;
      if (k0 + e < nz) {
        px_ += gx[e];
        py_ += gy[e];
      }
      gx[e] = px_;   // now the lane-local prefix of g
      gy[e] = py_;
    }
    // exclusive prefix scan of the lane totals over lower lanes
    double qx = px_, qy = py_;
    for (int o = 1; o < 32; o <<= 1) {
      const double ux = __shfl_up_sync(0xffffffffu, qx, o), uy = __shfl_up_sync(0xffffffffu, qy, o);
      if (t >= o) {
        qx += ux;
        qy += uy;
      }
    }
    const double lx = qx - px_, ly = qy - py_;
    for (int e = 0; e < per; ++e) {
      const int k = k0 + e;
      if (k < nz) S[k * plane] = make_float2((float)(gx[e] + lx), (float)(gy[e] + ly));
    }
    if (t == 0) S[0] = make_float2(0.0f, 0.0f);
    return;
  }
  const int py = blockIdx.x / per_row;
  const int px = (blockIdx.x - py * per_row) * blockDim.x + t;
  const long long col = (long long)py * n + px;
  if (px >= n) return;
  const int mx = bitrev(px, logn), my = bitrev(py, logn);
  if (mx == 0 && my == 0) return;   // solved by the last block
  float* cp = tsm;                                               // [nz][threads]
  float2* dd = reinterpret_cast<float2*>(tsm + nz * blockDim.x);  // [nz][threads]: the column
  // the whole column first (independent, coalesced loads), then the sweeps
  {
    int k = 0;
    for (; k + 8 <= nz; k += 8) {   // eight loads in flight before their stores
      float2 v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = S[(k + e) * plane + col];
#pragma unroll
      for (int e = 0; e < 8; ++e) dd[(k + e) * blockDim.x + t] = v[e];
    }
    for (; k < nz; ++k) dd[k * blockDim.x + t] = S[k * plane + col];
  }
  // lambda(m) = 2 - 2 cos(2 pi m / n) per axis
  const float lam = (2.0f - 2.0f * cospif(2.0f * (float)mx / (float)n)) +
                    (2.0f - 2.0f * cospif(2.0f * (float)my / (float)n));
  float cprev = 0.0f;
  float2 dprev = make_float2(0.0f, 0.0f);
  for (int k = 0; k < nz; ++k) {
    const float2 f = dd[k * blockDim.x + t];
    const float b = lam + ((k == 0 || k == nz - 1) ? 1.0f : 2.0f);   // Neumann ends
    const float m = b - (k == 0 ? 0.0f : -cprev);                   // a = -1
    const float r = 1.0f / m;
    const float cn = k == nz - 1 ? 0.0f : -r;
    dprev = make_float2((f.x * inv_scale + (k == 0 ? 0.0f : dprev.x)) * r,
                        (f.y * inv_scale + (k == 0 ? 0.0f : dprev.y)) * r);
    cp[k * blockDim.x + t] = cn;
    dd[k * blockDim.x + t] = dprev;
    cprev = cn;
  }
  float2 x = dprev;
  S[(nz - 1) * plane + col] = x;
  for (int k = nz - 2; k >= 0; --k) {
    const float cn = cp[k * blockDim.x + t];
    const float2 dn = dd[k * blockDim.x + t];
    x = make_float2(dn.x - cn * x.x, dn.y - cn * x.y);
    S[k * plane + col] = x;
  }
}

template <typename K>
bool set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) == cudaSuccess;
}

}  // namespace

bool spectral_pressure_supported(const LevelDev& L0) {
  if (L0.ncomp != 1) return false;
  const CompDev& c = L0.c[0];
  if (c.nx != c.ny || c.nx < 4 || c.nx > 128 || (c.nx & (c.nx - 1)) != 0 || c.nz < 2) return false;
  if (c.zkind != kAxisCellNeu) return false;
  if ((size_t)c.nz * kThomasThreads * 3 * sizeof(float) > 200 * 1024 || c.nz > 257) return false;
  return true;
}

size_t spectral_pressure_bytes(const LevelDev& L0) {
  const CompDev& c = L0.c[0];
  return (size_t)c.nx * c.ny * c.nz * sizeof(float2);
}

cudaError_t spectral_pressure_solve(const LevelDev& L0, const float* r, float* delta, void* spectrum,
                                    cudaStream_t st) {
  const CompDev& c = L0.c[0];
  const int n = c.nx, nz = c.nz;
  int logn = 0;
  while ((1 << logn) < n) ++logn;
  float2* S = (float2*)spectrum;
  const size_t fsm = (size_t)(n * n + n / 2) * sizeof(float2);
  // at least one warp per block (the (0, 0) block scans with a full warp)
  const int tthreads = n < 32 ? 32 : (n < kThomasThreads ? n : kThomasThreads);
  const int per_row = n / tthreads > 0 ? n / tthreads : 1;
  // per thread: FP32 c' and the column (float2)
  const size_t tsm = (size_t)nz * tthreads * 3 * sizeof(float);
  static std::atomic<int> ready[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !ready[dev].load()) {
    if (!set_smem(k_spec_forward, 227 * 1024) || !set_smem(k_spec_inverse, 227 * 1024) ||
        !set_smem(k_spec_thomas, 227 * 1024))
      return cudaGetLastError();
    ready[dev].store(1);
  }
  prof::Scope ps(SELM_K_PROJECTION, st);
  k_spec_forward<<<nz, kSpecThreads, fsm, st>>>(r, S, n, logn);
  k_spec_thomas<<<n * per_row + 1, tthreads, tsm, st>>>(S, n, logn, nz, (float)(1.0 / c.s));
  k_spec_inverse<<<nz, kSpecThreads, fsm, st>>>(S, delta, n, logn);
  return cudaGetLastError();
}

}  // namespace selm
