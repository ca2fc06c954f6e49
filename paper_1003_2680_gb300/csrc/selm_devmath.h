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

// All four Box-Muller normals of one Philox block: u_k = (w_k + 1/2) 2^-32,
// (n0, n1) = sqrt(-2 ln u0) (cos 2 pi u1, sin 2 pi u1), (n2, n3) likewise.
template <typename T>
struct Normals;

template <>
struct Normals<double> {
  // u = (w + 1/2) 2^-32; (n0, n1) = sqrt(-2 ln u0) (cos 2 pi u1, sin 2 pi u1), etc.
  __device__ static void get(uint4 w, double n[4]) {
    const double s = 2.3283064365386962890625e-10;
    const double u0 = ((double)w.x + 0.5) * s, u1 = ((double)w.y + 0.5) * s;
    const double u2 = ((double)w.z + 0.5) * s, u3 = ((double)w.w + 0.5) * s;
    const double r0 = sqrt(-2.0 * log(u0)), r1 = sqrt(-2.0 * log(u2));
    double s1, c1, s3, c3;
    sincospi(2.0 * u1, &s1, &c1);
    sincospi(2.0 * u3, &s3, &c3);
    n[0] = r0 * c1;
    n[1] = r0 * s1;
    n[2] = r1 * c3;
    n[3] = r1 * s3;
  }
};

template <>
struct Normals<float> {
  __device__ static void get(uint4 w, float n[4]) {
    const float s = 2.3283064365386962890625e-10f;
    const float u0 = ((float)w.x + 0.5f) * s, u1 = ((float)w.y + 0.5f) * s;
    const float u2 = ((float)w.z + 0.5f) * s, u3 = ((float)w.w + 0.5f) * s;
    const float r0 = sqrtf(-2.0f * logf(u0)), r1 = sqrtf(-2.0f * logf(u2));
    float s1, c1, s3, c3;
    sincospif(2.0f * u1, &s1, &c1);
    sincospif(2.0f * u3, &s3, &c3);
    n[0] = r0 * c1;
    n[1] = r0 * s1;
    n[2] = r1 * c3;
    n[3] = r1 * s3;
  }
};

// 8-wide vector loads and stores (16-byte aligned addresses).
template <typename T>
struct Vec;
template <>
struct Vec<float> {
  __device__ static void load8(const float* p, float o[8]) {
    const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
  }
  __device__ static void store8(float* p, const float o[8]) {
    *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    *reinterpret_cast<float4*>(p + 4) = make_float4(o[4], o[5], o[6], o[7]);
  }
};
template <>
struct Vec<double> {
  __device__ static void load8(const double* p, double o[8]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double2 a = *reinterpret_cast<const double2*>(p + 2 * q);
      o[2 * q] = a.x;
      o[2 * q + 1] = a.y;
    }
  }
  __device__ static void store8(double* p, const double o[8]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) *reinterpret_cast<double2*>(p + 2 * q) = make_double2(o[2 * q], o[2 * q + 1]);
  }
};

}  // namespace selm
