// Device math shared by the kernel translation units: the Philox4x32-10
// counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11), Box-Muller
// normals (Box & Muller 1958), and precision-typed square roots (so that FP32
// code never falls back to the slow FP64 path of this GPU).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace selm {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

__device__ __forceinline__ float tsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double tsqrt(double x) { return sqrt(x); }

// Normal number `lane` (0..3) of one Philox block: u = (w + 1/2) 2^-32,
// (n0, n1) = sqrt(-2 ln u0) (cos 2 pi u1, sin 2 pi u1), (n2, n3) likewise
// from (u2, u3).  Only the Box-Muller pair of `lane` is evaluated.
__device__ __forceinline__ void normal_of(uint4 w, int lane, float* out) {
  const float s = 2.3283064365386962890625e-10f;
  const uint32_t wa = lane < 2 ? w.x : w.z, wb = lane < 2 ? w.y : w.w;
  const float ua = ((float)wa + 0.5f) * s, ub = ((float)wb + 0.5f) * s;
  const float r = sqrtf(-2.0f * logf(ua));
  float sn, cs;
  sincospif(2.0f * ub, &sn, &cs);
  *out = r * ((lane & 1) ? sn : cs);
}

__device__ __forceinline__ void normal_of(uint4 w, int lane, double* out) {
  const double s = 2.3283064365386962890625e-10;
  const uint32_t wa = lane < 2 ? w.x : w.z, wb = lane < 2 ? w.y : w.w;
  const double ua = ((double)wa + 0.5) * s, ub = ((double)wb + 0.5) * s;
  const double r = sqrt(-2.0 * log(ua));
  double sn, cs;
  sincospi(2.0 * ub, &sn, &cs);
  *out = r * ((lane & 1) ? sn : cs);
}

}  // namespace selm
