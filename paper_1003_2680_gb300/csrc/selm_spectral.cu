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
//      plane, the plane in shared memory, radix-2 decimation in time);
//   2. per mode, the z system solved by the Thomas algorithm in FP64
//      arithmetic (the all-constant mode (0, 0) is singular: its z = 0 value is
//      pinned to 0, which fixes the pressure's free constant; the gradient
//      does not see it);
//   3. inverse 2-D FFT of every plane; the real part / n^2 is the correction.
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
constexpr int kThomasThreads = 64;

__device__ __forceinline__ int bitrev(int x, int logn) { return (int)(__brev((unsigned)x) >> (32 - logn)); }

// In-place radix-2 DIT FFT of all rows (along x) or all columns (along y) of
// an n x n complex plane in shared memory whose entries sit at bit-reversed
// positions along that axis.  sign = -1 forward, +1 inverse (unscaled).
__device__ void fft_axis(float2* A, const float2* W, int n, int logn, bool columns, float sign) {
  const int half_n = n >> 1;
  for (int s = 1; s <= logn; ++s) {
    const int half = 1 << (s - 1);
    const int tw_step = n >> s;   // twiddle index stride: W[j * n / (2 half)]
    for (int q = threadIdx.x; q < n * half_n; q += blockDim.x) {
      // along columns, consecutive threads take consecutive columns (the
      // butterflies of one column are n entries apart: bank conflicts else)
      const int line = columns ? q % n : q / half_n;
      const int p = columns ? q / n : q - line * half_n;
      const int grp = p / half, j = p - grp * half;
      const int i0 = grp * 2 * half + j, i1 = i0 + half;
      float2 w = W[j * tw_step];   // exp(-2 pi i j / (2 half)); conjugated for the inverse
      w.y *= -sign;
      const int a0 = columns ? i0 * n + line : line * n + i0;
      const int a1 = columns ? i1 * n + line : line * n + i1;
      const float2 x0 = A[a0], x1 = A[a1];
      const float2 t = make_float2(w.x * x1.x - w.y * x1.y, w.x * x1.y + w.y * x1.x);
      A[a0] = make_float2(x0.x + t.x, x0.y + t.y);
      A[a1] = make_float2(x0.x - t.x, x0.y - t.y);
    }
    __syncthreads();
  }
}

// twiddles W[j] = exp(-2 pi i j / n), j < n / 2
__device__ void make_twiddles(float2* W, int n) {
  for (int j = threadIdx.x; j < (n >> 1); j += blockDim.x) {
    float s, c;
    sincospif(-2.0f * (float)j / (float)n, &s, &c);
    W[j] = make_float2(c, s);
  }
}

// Forward: plane k of r (FP32, [nz][n][n]) -> spectrum S[k][my][mx].
__global__ void __launch_bounds__(kSpecThreads) k_spec_forward(const float* __restrict__ r, float2* __restrict__ S,
                                                               int n, int logn) {
  extern __shared__ float2 sm[];
  float2* A = sm;
  float2* W = sm + n * n;
  const int k = blockIdx.x;
  const float* rp = r + (long long)k * n * n;
  make_twiddles(W, n);
  for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
    const int y = q / n, x = q - y * n;
    A[bitrev(y, logn) * n + bitrev(x, logn)] = make_float2(rp[q], 0.0f);
  }
  __syncthreads();
  fft_axis(A, W, n, logn, false, -1.0f);
  fft_axis(A, W, n, logn, true, -1.0f);
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
  for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
    const int y = q / n, x = q - y * n;
    A[bitrev(y, logn) * n + bitrev(x, logn)] = Sp[q];
  }
  __syncthreads();
  fft_axis(A, W, n, logn, false, 1.0f);
  fft_axis(A, W, n, logn, true, 1.0f);
  const float inv = 1.0f / (float)(n * n);
  float* dp = d + (long long)k * n * n;
  for (int q = threadIdx.x; q < n * n; q += blockDim.x) dp[q] = A[q].x * inv;
}

// Thomas algorithm along z for the modes (mx0 + t, my), t < blockDim.x, in
// FP64 arithmetic; S is overwritten by the solution.  Shared memory: the
// forward sweep's c' and d' per thread ([nz][threads]).
__global__ void __launch_bounds__(kThomasThreads) k_spec_thomas(float2* __restrict__ S, int n, int nz, double scale) {
  extern __shared__ double tsm[];
  const int t = threadIdx.x;
  const int per_row = n / kThomasThreads > 0 ? n / kThomasThreads : 1;
  const int my = blockIdx.x / per_row;
  const int mx = (blockIdx.x - my * per_row) * blockDim.x + t;
  if (mx >= n) return;
  double* cp = tsm;                                  // [nz][threads]
  double2* dp = (double2*)(tsm + nz * blockDim.x);   // [nz][threads]
  const long long plane = (long long)n * n;
  const long long col = (long long)my * n + mx;
  // lambda(m) = 2 - 2 cos(2 pi m / n)
  const double lam = (2.0 - 2.0 * cospi(2.0 * mx / n)) + (2.0 - 2.0 * cospi(2.0 * my / n));
  const bool zero_mode = mx == 0 && my == 0;
  double cprev = 0.0;
  double2 dprev = make_double2(0.0, 0.0);
  for (int k = 0; k < nz; ++k) {
    const float2 f = S[k * plane + col];
    double b = lam + ((k == 0 || k == nz - 1) ? 1.0 : 2.0);   // Neumann ends
    const double a = k == 0 ? 0.0 : -1.0, c = k == nz - 1 ? 0.0 : -1.0;
    double2 d = make_double2((double)f.x / scale, (double)f.y / scale);   // operator = scale (lambda + T_z)
    if (zero_mode && k == 0) {   // pinned: phi^(0, 0, z = 0) = 0
      b = 1.0;
      d = make_double2(0.0, 0.0);
    }
    const double cc = zero_mode && k == 0 ? 0.0 : c;
    const double m = b - a * cprev;
    const double cn = cc / m;
    const double2 dn = make_double2((d.x - a * dprev.x) / m, (d.y - a * dprev.y) / m);
    cp[k * blockDim.x + t] = cn;
    dp[k * blockDim.x + t] = dn;
    cprev = cn;
    dprev = dn;
  }
  double2 x = dprev;
  S[(nz - 1) * plane + col] = make_float2((float)x.x, (float)x.y);
  for (int k = nz - 2; k >= 0; --k) {
    const double cn = cp[k * blockDim.x + t];
    const double2 dn = dp[k * blockDim.x + t];
    x = make_double2(dn.x - cn * x.x, dn.y - cn * x.y);
    S[k * plane + col] = make_float2((float)x.x, (float)x.y);
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
  if ((size_t)c.nz * kThomasThreads * (sizeof(double) + 2 * sizeof(double)) > 200 * 1024) return false;
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
  const int tthreads = n < kThomasThreads ? n : kThomasThreads;
  const size_t tsm = (size_t)nz * tthreads * 3 * sizeof(double);
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
  const int per_row = n / tthreads;
  k_spec_thomas<<<n * per_row, tthreads, tsm, st>>>(S, n, nz, c.s);
  k_spec_inverse<<<nz, kSpecThreads, fsm, st>>>(S, delta, n, logn);
  return cudaGetLastError();
}

}  // namespace selm
