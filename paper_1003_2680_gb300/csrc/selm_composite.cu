// Composite grid with one refined patch: the FAC cycle of Algorithm 1 around
// the Full-Sweep of Algorithm 2 (sm_103a).
//
// Geometry: the base channel (n cells along each periodic axis, wall-axis
// rows j = 1..n-1 with the wall centres on the walls) has its rows j = 1..K
// refined by 2 over the whole x-y extent.  The patch holds 2K layers of
// 2n x 2n (2-D: 2n) fine cells per component.  The composite operator is the
// cell-centred adaptive discretization of Section 4 (Eqs. equ_def_discr_div to
// equ_def_L) in its symmetric form A = -mu V L: the sum over faces of
// w (delta c)^2, with w = mu h^(d-2) between fine cells, mu H^(d-2) between
// base cells and at the top wall, and mu (4/3) H^(d-2) for each coarse-fine
// group (delta = coarse value - mean of its 2^(d-1) fine neighbours; the base
// wall cell below the patch is a coarse cell of value 0).
//
// One FAC iteration (reading R24 for the transfer, R25 for the patch order):
//   r   = b - A z (FP64)                  k_comp_residual
//   r_b = P^T r on the base grid          k_comp_residual (uncovered rows), k_comp_restrict (covered)
//   q_b = V-Cycle(0, r_b), base levels    the uniform library's V-cycle from level 1
//   q   = P q_b (parent copy)             k_comp_prolong
//   nu patch sweeps, 4 passes each        k_comp_patch
//   z  += q                               k_comp_update
//
// Level fields: level 0 of the internal handle is the patch (components
// concatenated, each [2K][2n][2n]); level 1 the base grid (each [n-1][n][n]).
// A composite FP64 vector is the patch field followed by the base field; the
// covered base rows (j <= K) are not unknowns (ignored on input).

#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <new>
#include <string>

#include "../../include/selm_mg.h"
#include "selm_devmath.h"
#include "selm_handle.h"
#include "selm_internal.h"
#include "selm_prof.h"

namespace selm {
namespace {

constexpr int kCBlock = 256;

struct CompGeo {
  int dim, n, K, ncomp;
  int fx, fy, fz;            // patch extents per component
  int bx, by, bz;            // base extents per component (bz = n - 1)
  long long fsize, bsize;    // per-component field sizes
  long long N0, N1;          // level-field sizes (all components)
  double sf, sb, wcf;        // face weights mu h^(d-2), mu H^(d-2), mu (4/3) H^(d-2)
  int nch;                   // fine faces per coarse-fine face: 2^(d-1)
  // the same weights as FP32 pairs (hi + lo) for the double-float chain, and
  // w2 = wcf / nch^2, w1 = wcf / nch
  float sf_h, sf_l, sb_h, sb_l, wcf_h, wcf_l, w2_h, w2_l, w1_h, w1_l;
};

inline unsigned cgrid(long long n) { return (unsigned)((n + kCBlock - 1) / kCBlock); }

__device__ __forceinline__ int cwrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Row of A at patch cell (m, q, p) of one component: off = sum_{j != i} A_ij c_j
// and diag = A_ii.  zp: the component's patch values, zb: its base values.
template <typename A, typename V>
__device__ __forceinline__ void patch_row(const CompGeo& G, const V* zp, const V* zb, int m, int q, int p, A* off,
                                          A* diag) {
  const int fx = G.fx, fy = G.fy, fz = G.fz;
  const long long plane = (long long)fx * fy;
  const long long row = (long long)m * plane + (long long)q * fx;
  A sum = (A)zp[row + cwrap(p - 1, fx)] + (A)zp[row + cwrap(p + 1, fx)];
  int nn = 2;
  if (fy > 1) {
    sum += (A)zp[(long long)m * plane + (long long)cwrap(q - 1, fy) * fx + p] +
           (A)zp[(long long)m * plane + (long long)cwrap(q + 1, fy) * fx + p];
    nn += 2;
  }
  if (m > 0) {
    sum += (A)zp[row - plane + p];
    ++nn;
  }
  if (m < fz - 1) {
    sum += (A)zp[row + plane + p];
    ++nn;
  }
  A o = -(A)G.sf * sum;
  A d = (A)G.sf * (A)nn;
  if (m == 0 || m == fz - 1) {
    // coarse-fine group: w (c_A - mean(siblings))^2 with c_A the base cell above
    // (top layer) or the wall (bottom layer)
    const int q0 = q & ~1, p0 = p & ~1;
    A sib = (A)0;
    for (int a = 0; a < (fy > 1 ? 2 : 1); ++a)
      for (int c = 0; c < 2; ++c) {
        const int qq = fy > 1 ? q0 + a : 0, pp = p0 + c;
        if (qq == q && pp == p) continue;
        sib += (A)zp[(long long)m * plane + (long long)qq * fx + pp];
      }
    const A w2 = (A)(G.wcf / ((double)G.nch * G.nch));
    o += w2 * sib;
    d += w2;
    if (m == fz - 1) {
      const A cA = (A)zb[((long long)G.K * G.by + (fy > 1 ? (q >> 1) : 0)) * G.bx + (p >> 1)];
      o -= (A)(G.wcf / G.nch) * cA;
    }
  }
  *off = o;
  *diag = d;
}

// Row of A at an uncovered base cell (r >= K, array row r = j - 1).
template <typename A, typename V>
__device__ __forceinline__ void base_row(const CompGeo& G, const V* zp, const V* zb, int r, int l, int i, A* off,
                                         A* diag) {
  const int bx = G.bx, by = G.by, bz = G.bz;
  const long long plane = (long long)bx * by;
  const long long row = (long long)r * plane + (long long)l * bx;
  A sum = (A)zb[row + cwrap(i - 1, bx)] + (A)zb[row + cwrap(i + 1, bx)];
  int nn = 2;
  if (by > 1) {
    sum += (A)zb[(long long)r * plane + (long long)cwrap(l - 1, by) * bx + i] +
           (A)zb[(long long)r * plane + (long long)cwrap(l + 1, by) * bx + i];
    nn += 2;
  }
  ++nn;                                   // face above: base row or the top wall (value 0)
  if (r + 1 < bz) sum += (A)zb[row + plane + i];
  A o = (A)0, d = (A)0;
  if (r > G.K) {
    sum += (A)zb[row - plane + i];
    ++nn;
  } else {                                // r == K: coarse-fine group with the patch's top layer
    const int m = G.fz - 1;
    const long long fplane = (long long)G.fx * G.fy;
    A mean = (A)0;
    for (int a = 0; a < (by > 1 ? 2 : 1); ++a)
      for (int c = 0; c < 2; ++c)
        mean += (A)zp[(long long)m * fplane + (long long)(by > 1 ? 2 * l + a : 0) * G.fx + 2 * i + c];
    mean *= (A)(1.0 / G.nch);
    o -= (A)G.wcf * mean;
    d += (A)G.wcf;
  }
  o -= (A)G.sb * sum;
  d += (A)G.sb * (A)nn;
  *off = o;
  *diag = d;
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// r = b - A z over the composite unknowns, in FP64; r written in T: patch
// sites into rp, uncovered base sites into rb (the restriction's identity
// part); ||r||^2 added to *norm2 when given.  b == nullptr means b = 0.
template <typename T>
__global__ void __launch_bounds__(kCBlock) k_comp_residual(CompGeo G, const double* __restrict__ z,
                                                           const double* __restrict__ b, T* __restrict__ rp,
                                                           T* __restrict__ rb, double* __restrict__ norm2) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double rr = 0.0;
  if (s < G.N0) {
    const int c = (int)(s / G.fsize);
    const long long loc = s - c * G.fsize;
    const int p = (int)(loc % G.fx);
    const long long t = loc / G.fx;
    const int q = (int)(t % G.fy), m = (int)(t / G.fy);
    double off, dg;
    patch_row<double, double>(G, z + c * G.fsize, z + G.N0 + c * G.bsize, m, q, p, &off, &dg);
    const double r = (b ? b[s] : 0.0) - (off + dg * z[s]);
    rp[s] = (T)r;
    rr = r * r;
  } else if (s < G.N0 + G.N1) {
    const long long s1 = s - G.N0;
    const int c = (int)(s1 / G.bsize);
    const long long loc = s1 - c * G.bsize;
    const int i = (int)(loc % G.bx);
    const long long t = loc / G.bx;
    const int l = (int)(t % G.by), r0 = (int)(t / G.by);
    if (r0 >= G.K) {
      double off, dg;
      base_row<double, double>(G, z + c * G.fsize, z + G.N0 + c * G.bsize, r0, l, i, &off, &dg);
      const double r = (b ? b[s] : 0.0) - (off + dg * z[s]);
      rb[s1] = (T)r;
      rr = r * r;
    }
  }
  if (norm2) {
    __shared__ double part[kCBlock / 32];
    rr = warp_sum(rr);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = rr;
    __syncthreads();
    if (threadIdx.x < 32) {
      double x = threadIdx.x < kCBlock / 32 ? part[threadIdx.x] : 0.0;
      x = warp_sum(x);
      if (threadIdx.x == 0) atomicAdd(norm2, x);
    }
  }
}

// Covered base rows of r_b = P^T r: the sum of the cell's 2^d fine children.
template <typename T>
__global__ void __launch_bounds__(kCBlock) k_comp_restrict(CompGeo G, const T* __restrict__ rp, T* __restrict__ rb) {
  const long long per = (long long)G.K * G.by * G.bx;
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= per * G.ncomp) return;
  const int c = (int)(s / per);
  const long long loc = s - c * per;
  const int i = (int)(loc % G.bx);
  const long long t = loc / G.bx;
  const int l = (int)(t % G.by), r = (int)(t / G.by);
  const T* f = rp + c * G.fsize;
  T acc = (T)0;
  for (int dm = 0; dm < 2; ++dm)
    for (int a = 0; a < (G.fy > 1 ? 2 : 1); ++a)
      for (int cc = 0; cc < 2; ++cc)
        acc += f[((long long)(2 * r + dm) * G.fy + (G.fy > 1 ? 2 * l + a : 0)) * G.fx + 2 * i + cc];
  rb[c * G.bsize + ((long long)r * G.by + l) * G.bx + i] = acc;
}

// q on the patch = P q_b: each fine cell takes its parent's value.
template <typename T>
__global__ void __launch_bounds__(kCBlock) k_comp_prolong(CompGeo G, T* __restrict__ vp, const T* __restrict__ vb) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= G.N0) return;
  const int c = (int)(s / G.fsize);
  const long long loc = s - c * G.fsize;
  const int p = (int)(loc % G.fx);
  const long long t = loc / G.fx;
  const int q = (int)(t % G.fy), m = (int)(t / G.fy);
  vp[s] = vb[c * G.bsize + ((long long)(m >> 1) * G.by + (G.fy > 1 ? (q >> 1) : 0)) * G.bx + (p >> 1)];
}

// The same copy on 8-wide segments of the patch rows (fx % 8 == 0): four
// parents, each to two consecutive fine cells.
template <typename T>
__global__ void __launch_bounds__(kCBlock) k_comp_prolong_v8(CompGeo G, T* __restrict__ vp,
                                                             const T* __restrict__ vb) {
  const int segs = G.fx >> 3;
  const long long rows = (long long)G.fz * G.fy;
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long row_all = g / segs;
  if (row_all >= rows * G.ncomp) return;
  const int seg = (int)(g - row_all * segs);
  const int c = (int)(row_all / rows);
  const long long rl = row_all - c * rows;
  const int q = (int)(rl % G.fy), m = (int)(rl / G.fy);
  const int x0 = seg << 3;
  const T* par = vb + c * G.bsize + ((long long)(m >> 1) * G.by + (G.fy > 1 ? (q >> 1) : 0)) * G.bx + (x0 >> 1);
  T out[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) out[e] = par[e >> 1];
  Vec<T>::store8(vp + c * G.fsize + ((long long)m * G.fy + q) * G.fx + x0, out);
}

// One pass of a patch sweep (reading R25): pass = 2 colour + late, colour =
// (p + q + m) mod 2, late = interface layer (m = 0 or 2K-1) and p odd.  Main
// passes (late = 0) visit all layers, late passes the two interface layers.
// One thread per candidate site of the colour; heat-bath update with the
// composite row; noise kind 2 at the site's linear patch index.
template <typename T, bool NOISE>
__global__ void __launch_bounds__(kCBlock) k_comp_patch(CompGeo G, T* __restrict__ vp, const T* __restrict__ vb,
                                                        const T* __restrict__ rp, int pass, int sweep, Key key,
                                                        const unsigned long long* __restrict__ cyc) {
  const int colour = pass >> 1, late = pass & 1;
  const int hx = G.fx >> 1;
  const int layers = late ? 2 : G.fz;
  const long long per = (long long)layers * G.fy * hx;
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= per * G.ncomp) return;
  const int c = (int)(s / per);
  const long long loc = s - c * per;
  const int hp = (int)(loc % hx);
  const long long t = loc / hx;
  const int q = (int)(t % G.fy), ml = (int)(t / G.fy);
  const int m = late ? (ml == 0 ? 0 : G.fz - 1) : ml;
  const int p = 2 * hp + ((q + m + colour) & 1);
  const bool iface = m == 0 || m == G.fz - 1;
  if (late != (int)(iface && (p & 1))) return;
  T* zp = vp + c * G.fsize;
  const long long lin = ((long long)m * G.fy + q) * G.fx + p;
  T off, dg;
  patch_row<T, T>(G, zp, vb + c * G.bsize, m, q, p, &off, &dg);
  T nv = (rp[c * G.fsize + lin] - off) / dg;
  if (NOISE) {
    const unsigned long long cy = *cyc;
    // counter word 1: level 0 | comp << 4 | pass << 8 | sweep << 12 | kind 2 << 20;
    // group = row * ceil(fx / 8) + p / 8, lane = (p mod 8) / 2
    const uint32_t c1 = ((uint32_t)c << 4) | ((uint32_t)pass << 8) | ((uint32_t)sweep << 12) | (2u << 20);
    const uint32_t grp = (uint32_t)(((long long)m * G.fy + q) * ((G.fx + 7) >> 3) + (p >> 3));
    T nn;
    normal_of(philox4x32_10(make_uint4(grp, c1, (uint32_t)cy, (uint32_t)(cy >> 32)), key.k0, key.k1), (p & 7) >> 1,
              &nn);
    nv += nn / tsqrt(dg);
  }
  zp[lin] = nv;
}

// The same pass, one thread per 8-wide segment of a patch row (fx % 8 == 0).
// The segment's four sites of the colour are all even x or all odd x, so on
// an interface layer the whole segment belongs to the main pass (even) or to
// the late pass (odd).  Siblings of a site: its x partner (x ^ 1) in the same
// row and the pair in row q ^ 1 (one of the y neighbours); the coarse cells
// above a top-layer segment are four consecutive base cells.  Noise: the
// segment's eight linear indices form two Philox groups.
template <typename T, bool NOISE>
__global__ void __launch_bounds__(kCBlock) k_comp_patch_v8(CompGeo G, T* __restrict__ vp, const T* __restrict__ vb,
                                                           const T* __restrict__ rp, int pass, int sweep, Key key,
                                                           const unsigned long long* __restrict__ cyc) {
  const int colour = pass >> 1, late = pass & 1;
  const int segs = G.fx >> 3;
  const int layers = late ? 2 : G.fz;
  const long long rows = (long long)layers * G.fy;
  const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long row_all = gt / segs;
  if (row_all >= rows * G.ncomp) return;
  const int seg = (int)(gt - row_all * segs);
  const int c = (int)(row_all / rows);
  const long long rl = row_all - c * rows;
  const int q = (int)(rl % G.fy), ml = (int)(rl / G.fy);
  const int m = late ? (ml == 0 ? 0 : G.fz - 1) : ml;
  const int par = (q + m + colour) & 1;       // the colour's sites: e = 2l + par
  const bool iface = m == 0 || m == G.fz - 1;
  if (late != (int)(iface && par)) return;
  const int fx = G.fx, fy = G.fy, fz = G.fz;
  const long long plane = (long long)fx * fy;
  T* zp = vp + c * G.fsize;
  const long long rbase = (long long)m * plane + (long long)q * fx;
  const int x0 = seg << 3;
  T cen[8], rr[8], acc[8], sq[8];
  Vec<T>::load8(zp + rbase + x0, cen);
  Vec<T>::load8(rp + c * G.fsize + rbase + x0, rr);
  const T left = zp[rbase + (x0 == 0 ? fx - 1 : x0 - 1)];
  const T right = zp[rbase + (x0 + 8 == fx ? 0 : x0 + 8)];
  int nn = 2;
#pragma unroll
  for (int e = 0; e < 8; ++e) acc[e] = (T)0;
  if (fy > 1) {
    T t[8];
    const int qm = q == 0 ? fy - 1 : q - 1, qp = q == fy - 1 ? 0 : q + 1;
    Vec<T>::load8(zp + (long long)m * plane + (long long)qm * fx + x0, t);
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[e] += t[e];
    if ((q ^ 1) == qm) {
#pragma unroll
      for (int e = 0; e < 8; ++e) sq[e] = t[e];
    }
    Vec<T>::load8(zp + (long long)m * plane + (long long)qp * fx + x0, t);
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[e] += t[e];
    if ((q ^ 1) == qp) {
#pragma unroll
      for (int e = 0; e < 8; ++e) sq[e] = t[e];
    }
    nn += 2;
  }
  if (m > 0) {
    T t[8];
    Vec<T>::load8(zp + rbase - plane + x0, t);
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[e] += t[e];
    ++nn;
  }
  if (m < fz - 1) {
    T t[8];
    Vec<T>::load8(zp + rbase + plane + x0, t);
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[e] += t[e];
    ++nn;
  }
  const T sf = (T)G.sf;
  T dg = sf * (T)nn;
  const T w2 = (T)(G.wcf / ((double)G.nch * G.nch));
  const T w1 = (T)(G.wcf / G.nch);
  T ca[4] = {(T)0, (T)0, (T)0, (T)0};
  if (iface) {
    dg += w2;
    if (m == fz - 1) {   // the four base cells above the segment
      const T* brow = vb + c * G.bsize + ((long long)G.K * G.by + (fy > 1 ? (q >> 1) : 0)) * G.bx + (x0 >> 1);
#pragma unroll
      for (int l = 0; l < 4; ++l) ca[l] = brow[l];
    }
  }
  T n4[4];
  if (NOISE) {   // one block per segment: lane l for the colour's site 2l + par
    const unsigned long long cy = *cyc;
    const uint32_t c1 = ((uint32_t)c << 4) | ((uint32_t)pass << 8) | ((uint32_t)sweep << 12) | (2u << 20);
    const uint32_t grp = (uint32_t)(((long long)m * fy + q) * segs + seg);
    Normals<T>::get(philox4x32_10(make_uint4(grp, c1, (uint32_t)cy, (uint32_t)(cy >> 32)), key.k0, key.k1), n4);
  }
  const T rsd = NOISE ? (T)1 / tsqrt(dg) : (T)0;
  const T rdg = (T)1 / dg;   // one division per row instead of one per site
#pragma unroll
  for (int l = 0; l < 4; ++l) {
#pragma unroll
    for (int pp = 0; pp < 2; ++pp) {
      if (pp != par) continue;
      const int e = 2 * l + pp;
      const T xl = e == 0 ? left : cen[e - 1];
      const T xr = e == 7 ? right : cen[e + 1];
      T off = -sf * (acc[e] + xl + xr);
      if (iface) {
        T sib = cen[e ^ 1];
        if (fy > 1) sib += sq[e] + sq[e ^ 1];
        off += w2 * sib;
        if (m == fz - 1) off -= w1 * ca[l];
      }
      T nv = (rr[e] - off) * rdg;
      if (NOISE) nv += n4[l] * rsd;
      cen[e] = nv;
    }
  }
  Vec<T>::store8(zp + rbase + x0, cen);
}

// ---------------------------------------------------------------------------
// Double-float chain state (FP32 inner cycles).  The chain value is hi + lo
// with |lo| <= ulp(hi)/2 (about 48 significant bits); sums and products use
// the error-free transformations TwoSum (Knuth) and the FMA product error
// (Dekker's splitting replaced by fma), so the chain's residual and update
// keep near-FP64 accuracy on the FP32 pipes instead of GB300's slow FP64 pipe.
// ---------------------------------------------------------------------------
struct DF {
  float h, l;
};

__device__ __forceinline__ DF df_from(float h, float l) { return {h, l}; }

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ DF df_norm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  return df_norm(s, e);
}

__device__ __forceinline__ DF df_neg(DF a) { return {-a.h, -a.l}; }

__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return df_norm(p, e);
}

__device__ __forceinline__ DF df_at(const float* hi, const float* lo, long long i) { return {hi[i], lo[i]}; }

// r = -A z for the chain (b = 0) in double-float arithmetic, written in FP32:
// patch sites into rp, uncovered base sites into rb.
__global__ void __launch_bounds__(kCBlock) k_comp_residual_df(CompGeo G, const float* __restrict__ zh,
                                                              const float* __restrict__ zl, float* __restrict__ rp,
                                                              float* __restrict__ rb) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < G.N0) {
    const int c = (int)(s / G.fsize);
    const long long loc = s - c * G.fsize;
    const int p = (int)(loc % G.fx);
    const long long t = loc / G.fx;
    const int q = (int)(t % G.fy), m = (int)(t / G.fy);
    const float* ph = zh + c * G.fsize;
    const float* pl = zl + c * G.fsize;
    const long long plane = (long long)G.fx * G.fy;
    const long long row = (long long)m * plane + (long long)q * G.fx;
    DF nb = df_add(df_at(ph, pl, row + cwrap(p - 1, G.fx)), df_at(ph, pl, row + cwrap(p + 1, G.fx)));
    int nn = 2;
    if (G.fy > 1) {
      nb = df_add(nb, df_at(ph, pl, (long long)m * plane + (long long)cwrap(q - 1, G.fy) * G.fx + p));
      nb = df_add(nb, df_at(ph, pl, (long long)m * plane + (long long)cwrap(q + 1, G.fy) * G.fx + p));
      nn += 2;
    }
    if (m > 0) {
      nb = df_add(nb, df_at(ph, pl, row - plane + p));
      ++nn;
    }
    if (m < G.fz - 1) {
      nb = df_add(nb, df_at(ph, pl, row + plane + p));
      ++nn;
    }
    const DF zc = df_at(ph, pl, row + p);
    // A z = sf (nn zc - sum of neighbours) [+ w2 (sum of the sibling group) - w1 zA]
    DF Az = df_mul(df_from(G.sf_h, G.sf_l), df_add(df_mul(df_from((float)nn, 0.f), zc), df_neg(nb)));
    if (m == 0 || m == G.fz - 1) {
      const int q0 = q & ~1, p0 = p & ~1;
      DF grp = {0.f, 0.f};
      for (int a = 0; a < (G.fy > 1 ? 2 : 1); ++a)
        for (int cc = 0; cc < 2; ++cc)
          grp = df_add(grp, df_at(ph, pl, (long long)m * plane + (long long)(G.fy > 1 ? q0 + a : 0) * G.fx + p0 + cc));
      Az = df_add(Az, df_mul(df_from(G.w2_h, G.w2_l), grp));
      if (m == G.fz - 1) {
        const long long bi = G.N0 + c * G.bsize + ((long long)G.K * G.by + (G.fy > 1 ? (q >> 1) : 0)) * G.bx + (p >> 1);
        Az = df_add(Az, df_neg(df_mul(df_from(G.w1_h, G.w1_l), df_at(zh, zl, bi))));
      }
    }
    rp[s] = -(Az.h + Az.l);
  } else if (s < G.N0 + G.N1) {
    const long long s1 = s - G.N0;
    const int c = (int)(s1 / G.bsize);
    const long long loc = s1 - c * G.bsize;
    const int i = (int)(loc % G.bx);
    const long long t = loc / G.bx;
    const int l = (int)(t % G.by), r0 = (int)(t / G.by);
    if (r0 < G.K) return;
    const float* bh = zh + G.N0 + c * G.bsize;
    const float* bl = zl + G.N0 + c * G.bsize;
    const long long plane = (long long)G.bx * G.by;
    const long long row = (long long)r0 * plane + (long long)l * G.bx;
    DF nb = df_add(df_at(bh, bl, row + cwrap(i - 1, G.bx)), df_at(bh, bl, row + cwrap(i + 1, G.bx)));
    int nn = 2;
    if (G.by > 1) {
      nb = df_add(nb, df_at(bh, bl, (long long)r0 * plane + (long long)cwrap(l - 1, G.by) * G.bx + i));
      nb = df_add(nb, df_at(bh, bl, (long long)r0 * plane + (long long)cwrap(l + 1, G.by) * G.bx + i));
      nn += 2;
    }
    ++nn;
    if (r0 + 1 < G.bz) nb = df_add(nb, df_at(bh, bl, row + plane + i));
    const DF zc = df_at(bh, bl, row + i);
    DF extra = {0.f, 0.f};
    if (r0 > G.K) {
      nb = df_add(nb, df_at(bh, bl, row - plane + i));
      ++nn;
    } else {   // wcf (zc - mean of the patch's top-layer children)
      const float* ph = zh + c * G.fsize;
      const float* pl = zl + c * G.fsize;
      const long long fplane = (long long)G.fx * G.fy;
      DF ch = {0.f, 0.f};
      for (int a = 0; a < (G.by > 1 ? 2 : 1); ++a)
        for (int cc = 0; cc < 2; ++cc)
          ch = df_add(ch, df_at(ph, pl, (long long)(G.fz - 1) * fplane + (long long)(G.by > 1 ? 2 * l + a : 0) * G.fx +
                                            2 * i + cc));
      const float inv = 1.0f / (float)G.nch;   // a power of two: exact
      extra = df_mul(df_from(G.wcf_h, G.wcf_l), df_add(zc, df_neg({ch.h * inv, ch.l * inv})));
    }
    DF Az = df_mul(df_from(G.sb_h, G.sb_l), df_add(df_mul(df_from((float)nn, 0.f), zc), df_neg(nb)));
    Az = df_add(Az, extra);
    rb[s1] = -(Az.h + Az.l);
  }
}

__device__ __forceinline__ void load8_df(const float* hi, const float* lo, long long i, DF o[8]) {
  float a[8], b[8];
  Vec<float>::load8(hi + i, a);
  Vec<float>::load8(lo + i, b);
#pragma unroll
  for (int e = 0; e < 8; ++e) o[e] = {a[e], b[e]};
}

// The chain residual r = -A z (double-float) on the patch rows, one thread
// per 8-wide segment of a patch row (fx % 8 == 0).
__global__ void __launch_bounds__(kCBlock) k_comp_residual_df_patch(CompGeo G, const float* __restrict__ zh,
                                                                    const float* __restrict__ zl,
                                                                    float* __restrict__ rp) {
  const int fx = G.fx, fy = G.fy, fz = G.fz, segs = fx >> 3;
  const long long rows = (long long)fz * fy;
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long row_all = g / segs;
  if (row_all >= rows * G.ncomp) return;
  const int seg = (int)(g - row_all * segs);
  const int c = (int)(row_all / rows);
  const long long rl = row_all - c * rows;
  const int q = (int)(rl % fy), m = (int)(rl / fy);
  const float* ph = zh + c * G.fsize;
  const float* pl = zl + c * G.fsize;
  const long long plane = (long long)fx * fy;
  const long long rbase = (long long)m * plane + (long long)q * fx;
  const int x0 = seg << 3;
  DF cur[8], nb[8], t[8], rq[8];
  load8_df(ph, pl, rbase + x0, cur);
  const DF left = df_at(ph, pl, rbase + (x0 == 0 ? fx - 1 : x0 - 1));
  const DF right = df_at(ph, pl, rbase + (x0 + 8 == fx ? 0 : x0 + 8));
#pragma unroll
  for (int e = 0; e < 8; ++e) nb[e] = df_add(e == 0 ? left : cur[e - 1], e == 7 ? right : cur[e + 1]);
  int nn = 2;
  const bool iface = m == 0 || m == fz - 1;
  if (fy > 1) {
    const int qm = q == 0 ? fy - 1 : q - 1, qp = q == fy - 1 ? 0 : q + 1;
    load8_df(ph, pl, (long long)m * plane + (long long)qm * fx + x0, t);
#pragma unroll
    for (int e = 0; e < 8; ++e) nb[e] = df_add(nb[e], t[e]);
    if ((q ^ 1) == qm) {
#pragma unroll
      for (int e = 0; e < 8; ++e) rq[e] = t[e];
    }
    load8_df(ph, pl, (long long)m * plane + (long long)qp * fx + x0, t);
#pragma unroll
    for (int e = 0; e < 8; ++e) nb[e] = df_add(nb[e], t[e]);
    if ((q ^ 1) == qp) {
#pragma unroll
      for (int e = 0; e < 8; ++e) rq[e] = t[e];
    }
    nn += 2;
  }
  if (m > 0) {
    load8_df(ph, pl, rbase - plane + x0, t);
#pragma unroll
    for (int e = 0; e < 8; ++e) nb[e] = df_add(nb[e], t[e]);
    ++nn;
  }
  if (m < fz - 1) {
    load8_df(ph, pl, rbase + plane + x0, t);
#pragma unroll
    for (int e = 0; e < 8; ++e) nb[e] = df_add(nb[e], t[e]);
    ++nn;
  }
  DF ca[4];
  if (m == fz - 1) {
    const long long bi = G.N0 + c * G.bsize + ((long long)G.K * G.by + (fy > 1 ? (q >> 1) : 0)) * G.bx + (x0 >> 1);
#pragma unroll
    for (int l = 0; l < 4; ++l) ca[l] = df_at(zh, zl, bi + l);
  }
  const DF sf = df_from(G.sf_h, G.sf_l), w2 = df_from(G.w2_h, G.w2_l), w1 = df_from(G.w1_h, G.w1_l);
  const DF fnn = df_from((float)nn, 0.f);
  float out[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    DF Az = df_mul(sf, df_add(df_mul(fnn, cur[e]), df_neg(nb[e])));
    if (iface) {
      DF grp = df_add(cur[e], cur[e ^ 1]);
      if (fy > 1) grp = df_add(grp, df_add(rq[e], rq[e ^ 1]));
      Az = df_add(Az, df_mul(w2, grp));
      if (m == fz - 1) Az = df_add(Az, df_neg(df_mul(w1, ca[e >> 1])));
    }
    out[e] = -(Az.h + Az.l);
  }
  Vec<float>::store8(rp + c * G.fsize + rbase + x0, out);
}

// The chain residual on the uncovered base rows, one thread per 8-wide
// segment of a base row (bx % 8 == 0); the interface row's coarse-fine group
// reads the sixteen patch children of the segment in each of its two rows.
__global__ void __launch_bounds__(kCBlock) k_comp_residual_df_base(CompGeo G, const float* __restrict__ zh,
                                                                   const float* __restrict__ zl,
                                                                   float* __restrict__ rb) {
  const int bx = G.bx, by = G.by, bz = G.bz, segs = bx >> 3;
  const long long rows = (long long)(bz - G.K) * by;
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long row_all = g / segs;
  if (row_all >= rows * G.ncomp) return;
  const int seg = (int)(g - row_all * segs);
  const int c = (int)(row_all / rows);
  const long long rl = row_all - c * rows;
  const int l = (int)(rl % by), r = G.K + (int)(rl / by);
  const float* bh = zh + G.N0 + c * G.bsize;
  const float* bl = zl + G.N0 + c * G.bsize;
  const long long plane = (long long)bx * by;
  const long long rbase = (long long)r * plane + (long long)l * bx;
  const int x0 = seg << 3;
  DF cur[8], nb[8], t[8];
  load8_df(bh, bl, rbase + x0, cur);
  const DF left = df_at(bh, bl, rbase + (x0 == 0 ? bx - 1 : x0 - 1));
  const DF right = df_at(bh, bl, rbase + (x0 + 8 == bx ? 0 : x0 + 8));
#pragma unroll
  for (int e = 0; e < 8; ++e) nb[e] = df_add(e == 0 ? left : cur[e - 1], e == 7 ? right : cur[e + 1]);
  int nn = 3;   // x pair + the face above (row or top wall)
  if (by > 1) {
    load8_df(bh, bl, (long long)r * plane + (long long)(l == 0 ? by - 1 : l - 1) * bx + x0, t);
#pragma unroll
    for (int e = 0; e < 8; ++e) nb[e] = df_add(nb[e], t[e]);
    load8_df(bh, bl, (long long)r * plane + (long long)(l == by - 1 ? 0 : l + 1) * bx + x0, t);
#pragma unroll
    for (int e = 0; e < 8; ++e) nb[e] = df_add(nb[e], t[e]);
    nn += 2;
  }
  if (r + 1 < bz) {
    load8_df(bh, bl, rbase + plane + x0, t);
#pragma unroll
    for (int e = 0; e < 8; ++e) nb[e] = df_add(nb[e], t[e]);
  }
  DF extra[8];
  if (r > G.K) {
    load8_df(bh, bl, rbase - plane + x0, t);
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      nb[e] = df_add(nb[e], t[e]);
      extra[e] = {0.f, 0.f};
    }
    ++nn;
  } else {
    // children of base cell x0 + e: patch layer fz-1, rows 2l (+1), cells 2(x0+e), 2(x0+e)+1
    const float* ph = zh + c * G.fsize;
    const float* pl = zl + c * G.fsize;
    const long long fplane = (long long)G.fx * G.fy;
    DF ch[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) ch[e] = {0.f, 0.f};
    for (int a = 0; a < (by > 1 ? 2 : 1); ++a) {
      const long long frow = (long long)(G.fz - 1) * fplane + (long long)(by > 1 ? 2 * l + a : 0) * G.fx + 2 * x0;
      DF u[8], w[8];
      load8_df(ph, pl, frow, u);
      load8_df(ph, pl, frow + 8, w);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        ch[e] = df_add(ch[e], df_add(u[2 * e], u[2 * e + 1]));
        ch[e + 4] = df_add(ch[e + 4], df_add(w[2 * e], w[2 * e + 1]));
      }
    }
    const float inv = 1.0f / (float)G.nch;   // a power of two: exact
    const DF wcf = df_from(G.wcf_h, G.wcf_l);
#pragma unroll
    for (int e = 0; e < 8; ++e) extra[e] = df_mul(wcf, df_add(cur[e], df_neg({ch[e].h * inv, ch[e].l * inv})));
  }
  const DF sb = df_from(G.sb_h, G.sb_l);
  const DF fnn = df_from((float)nn, 0.f);
  float out[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    DF Az = df_add(df_mul(sb, df_add(df_mul(fnn, cur[e]), df_neg(nb[e]))), extra[e]);
    out[e] = -(Az.h + Az.l);
  }
  Vec<float>::store8(rb + c * G.bsize + rbase + x0, out);
}

// z += q for the double-float chain (covered base rows untouched).
__global__ void __launch_bounds__(kCBlock) k_comp_update_df(CompGeo G, float* __restrict__ zh, float* __restrict__ zl,
                                                            const float* __restrict__ vp, const float* __restrict__ vb) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float q;
  if (s < G.N0) {
    q = vp[s];
  } else if (s < G.N0 + G.N1) {
    const long long s1 = s - G.N0;
    if ((int)((s1 % G.bsize) / ((long long)G.bx * G.by)) < G.K) return;
    q = vb[s1];
  } else {
    return;
  }
  float a, e;
  two_sum(zh[s], q, a, e);
  const DF r = df_norm(a, __fadd_rn(e, zl[s]));
  zh[s] = r.h;
  zl[s] = r.l;
}

// FP64 copy of the double-float chain (covered base rows 0).
__global__ void __launch_bounds__(kCBlock) k_comp_df_to_f64(CompGeo G, const float* __restrict__ zh,
                                                            const float* __restrict__ zl, double* __restrict__ out) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= G.N0 + G.N1) return;
  out[s] = (double)zh[s] + (double)zl[s];
}

// Main pass (late = 0) of a patch sweep marching along the patch layers: one
// thread per (component, y row, 8-wide segment, chunk of kc layers); z
// neighbours from registers, the next layer's row loaded before the current
// one is computed.  On an interface layer a segment whose colour sites have
// odd x belongs to the late pass and is left unchanged.
#ifndef SELM_PATCH_MIN_BLOCKS
#define SELM_PATCH_MIN_BLOCKS 2
#endif
template <typename T, bool NOISE>
__global__ void __launch_bounds__(kCBlock, sizeof(T) == 4 ? SELM_PATCH_MIN_BLOCKS : 1) k_comp_patch_zm(CompGeo G, T* __restrict__ vp, const T* __restrict__ vb,
                                                           const T* __restrict__ rp, int colour, int sweep, int kc,
                                                           Key key, const unsigned long long* __restrict__ cyc) {
  const int fx = G.fx, fy = G.fy, fz = G.fz, segs = fx >> 3;
  const long long chunks = (fz + kc - 1) / kc;
  const long long per = (long long)fy * segs * chunks;
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= per * G.ncomp) return;
  const int c = (int)(g / per);
  const long long item = g - c * per;
  const long long col = item % ((long long)fy * segs);
  const int chunk = (int)(item / ((long long)fy * segs));
  const int q = (int)(col / segs), seg = (int)(col - (long long)q * segs);
  const int m0 = chunk * kc, m1 = min(m0 + kc, fz);
  const long long plane = (long long)fx * fy;
  const int x0 = seg << 3;
  T* zp = vp + c * G.fsize;
  const T* rr0 = rp + c * G.fsize;
  const long long base = (long long)q * fx + x0;
  const int qm = q == 0 ? fy - 1 : q - 1, qp = q == fy - 1 ? 0 : q + 1;
  const long long ymb = (long long)qm * fx + x0, ypb = (long long)qp * fx + x0;
  const long long rowx = (long long)q * fx;
  const int xl_i = x0 == 0 ? fx - 1 : x0 - 1, xr_i = x0 + 8 == fx ? 0 : x0 + 8;
  const T sf = (T)G.sf;
  const T w2 = (T)(G.wcf / ((double)G.nch * G.nch));
  const T w1 = (T)(G.wcf / G.nch);
  const int pass = 2 * colour;
  const unsigned long long cy = NOISE ? *cyc : 0ull;
  const uint32_t c1 = ((uint32_t)c << 4) | ((uint32_t)pass << 8) | ((uint32_t)sweep << 12) | (2u << 20);
  T prev[8], cur[8], nxt[8], rr[8], ym[8], yp[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) prev[e] = (T)0;
  if (m0 > 0) Vec<T>::load8(zp + base + (long long)(m0 - 1) * plane, prev);
  Vec<T>::load8(zp + base + (long long)m0 * plane, cur);
  for (int m = m0; m < m1; ++m) {
    const long long mp = (long long)m * plane;
    if (m + 1 < fz)
      Vec<T>::load8(zp + base + mp + plane, nxt);
    else {
#pragma unroll
      for (int e = 0; e < 8; ++e) nxt[e] = (T)0;
    }
    const int par = (q + m + colour) & 1;
    const bool iface = m == 0 || m == fz - 1;
    if (!(iface && par)) {
      Vec<T>::load8(rr0 + base + mp, rr);
      int nn = 2;
      T acc[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[e] = (m > 0 ? prev[e] : (T)0) + (m + 1 < fz ? nxt[e] : (T)0);
      nn += (m > 0) + (m + 1 < fz);
      if (fy > 1) {
        Vec<T>::load8(zp + ymb + mp, ym);
        Vec<T>::load8(zp + ypb + mp, yp);
#pragma unroll
        for (int e = 0; e < 8; ++e) acc[e] += ym[e] + yp[e];
        nn += 2;
      }
      const T left = zp[rowx + mp + xl_i], right = zp[rowx + mp + xr_i];
      T dg = sf * (T)nn;
      T ca[4] = {(T)0, (T)0, (T)0, (T)0};
      if (iface) {
        dg += w2;
        if (m == fz - 1) {
          const T* brow = vb + c * G.bsize + ((long long)G.K * G.by + (fy > 1 ? (q >> 1) : 0)) * G.bx + (x0 >> 1);
#pragma unroll
          for (int l = 0; l < 4; ++l) ca[l] = brow[l];
        }
      }
      T n4[4] = {(T)0, (T)0, (T)0, (T)0};
      if (NOISE) {
        const uint32_t grp = (uint32_t)(((long long)m * fy + q) * segs + seg);
        Normals<T>::get(philox4x32_10(make_uint4(grp, c1, (uint32_t)cy, (uint32_t)(cy >> 32)), key.k0, key.k1), n4);
      }
      const T rsd = NOISE ? (T)1 / tsqrt(dg) : (T)0;
      const T rdg = (T)1 / dg;   // one division per row instead of one per site
      const bool up1 = (q ^ 1) == qp;   // which loaded y row holds the siblings' row q ^ 1
#pragma unroll
      for (int l = 0; l < 4; ++l) {
#pragma unroll
        for (int pp = 0; pp < 2; ++pp) {
          if (pp != par) continue;
          const int e = 2 * l + pp;
          const T xl = e == 0 ? left : cur[e - 1];
          const T xr = e == 7 ? right : cur[e + 1];
          T off = -sf * (acc[e] + xl + xr);
          if (iface) {
            T sib = cur[e ^ 1];
            if (fy > 1) sib += up1 ? yp[e] + yp[e ^ 1] : ym[e] + ym[e ^ 1];
            off += w2 * sib;
            if (m == fz - 1) off -= w1 * ca[l];
          }
          T nv = (rr[e] - off) * rdg;
          if (NOISE) nv += n4[l] * rsd;
          cur[e] = nv;
        }
      }
      Vec<T>::store8(zp + base + mp, cur);
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      prev[e] = cur[e];
      cur[e] = nxt[e];
    }
  }
}

// z += q on the composite unknowns (covered base rows untouched).
template <typename T>
__global__ void __launch_bounds__(kCBlock) k_comp_update(CompGeo G, double* __restrict__ z, const T* __restrict__ vp,
                                                         const T* __restrict__ vb) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < G.N0) {
    z[s] += (double)vp[s];
  } else if (s < G.N0 + G.N1) {
    const long long s1 = s - G.N0;
    const long long loc = s1 % G.bsize;
    const int r = (int)(loc / ((long long)G.bx * G.by));
    if (r >= G.K) z[s] += (double)vb[s1];
  }
}

// ||x||^2 over the composite unknowns.
__global__ void __launch_bounds__(kCBlock) k_comp_norm2(CompGeo G, const double* __restrict__ x,
                                                        double* __restrict__ out) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (s < G.N0) {
    v = x[s] * x[s];
  } else if (s < G.N0 + G.N1) {
    const long long loc = (s - G.N0) % G.bsize;
    if ((int)(loc / ((long long)G.bx * G.by)) >= G.K) v = x[s] * x[s];
  }
  __shared__ double part[kCBlock / 32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double y = threadIdx.x < kCBlock / 32 ? part[threadIdx.x] : 0.0;
    y = warp_sum(y);
    if (threadIdx.x == 0) atomicAdd(out, y);
  }
}

}  // namespace
}  // namespace selm

using namespace selm;

struct selm_comp {
  selm_comp_desc d{};
  selm_mg* mg = nullptr;     // base hierarchy (levels 1..) and level fields
  CompGeo geo{};
  int nu = 2;
  double* xi = nullptr;      // chain state, FP64 inner precision (composite vector)
  float* xh = nullptr;       // chain state, FP32 inner precision: double-float hi + lo
  float* xl = nullptr;
  double* red = nullptr;     // norm slots (in the internal handle's reduction words)
  double* host_red = nullptr;
  uint64_t cycle = 0;
  long long total_cycles = 0;
  std::string err;
  // one chain cycle (with its counter increment) as a captured CUDA graph,
  // replayed by selm_comp_sample (captured after one direct cycle)
  cudaGraphExec_t chain_graph = nullptr;
  int chain_runs = 0;
  long long graph_launches = 0, graph_vcycles = 0;
};

namespace {

#define CCK(call)                                                          \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess) {                                               \
      C->err = std::string(#call) + ": " + cudaGetErrorString(e_);         \
      return SELM_ECUDA;                                                   \
    }                                                                      \
  } while (0)

cudaStream_t CS(void* s) { return (cudaStream_t)s; }

std::string fill_comp_defaults(selm_comp_desc* d) {
  if (d->mu == 0.0) d->mu = 1.0;
  if (d->ncomp == 0) d->ncomp = 1;
  if (d->nu_pre == 0) d->nu_pre = 2;
  if (d->nu_post == 0) d->nu_post = 2;
  if (d->nu_patch == 0) d->nu_patch = 2;
  if (d->dim != 2 && d->dim != 3) return "dim must be 2 or 3";
  if (d->n < 4 || d->n % 2 != 0) return "n must be even and at least 4";
  if (d->K < 1 || d->K > d->n - 2) return "K must satisfy 1 <= K <= n-2";
  if (d->ncomp < 1 || d->ncomp > kMaxComps) return "ncomp must be 1..3";
  if (d->nu_pre < 0 || d->nu_post < 0 || d->nu_patch < 0 || d->nu_pre + d->nu_post > 64 || d->nu_patch > 64)
    return "sweep counts out of range";
  if (d->precision != SELM_FP64 && d->precision != SELM_FP32_REFINE64) return "unknown precision";
  if (d->coarse_mode != SELM_COARSE_CHOLESKY && d->coarse_mode != SELM_COARSE_SMOOTH) return "unknown coarse mode";
  if (!(d->mu > 0.0)) return "mu must be positive";
  if (d->levels == 0) d->levels = default_levels(d->n);
  if (d->levels < 1 || d->levels + 1 > kMaxLevels) return "levels out of range";
  if (d->n % (1 << (d->levels - 1)) != 0) return "n must be divisible by 2^(levels-1)";
  if ((long long)2 * d->n * 2 * d->n * 2 * d->K >= (1ll << 31)) return "patch too large";
  return "";
}

selm_mg_desc internal_desc(const selm_comp_desc& c) {
  selm_mg_desc d{};
  d.dim = c.dim;
  d.n = c.n;
  d.mu = c.mu;
  d.kT = 1.0;
  d.levels = c.levels + 1;
  d.nu_pre = c.nu_pre;
  d.nu_post = c.nu_post;
  d.precision = c.precision;
  d.projection = SELM_PROJ_NONE;
  d.coarse_mode = c.coarse_mode;
  d.tol = 1e-10;
  d.max_cycles = 1000;
  d.seed = c.seed;
  d.instance = c.instance;
  d.alloc = c.alloc;
  d.free = c.free;
  d.alloc_ctx = c.alloc_ctx;
  return d;
}

CompGeo make_geo(const selm_comp_desc& d) {
  CompGeo G{};
  G.dim = d.dim;
  G.n = d.n;
  G.K = d.K;
  G.ncomp = d.ncomp;
  G.fx = 2 * d.n;
  G.fy = d.dim == 3 ? 2 * d.n : 1;
  G.fz = 2 * d.K;
  G.bx = d.n;
  G.by = d.dim == 3 ? d.n : 1;
  G.bz = d.n - 1;
  G.fsize = (long long)G.fx * G.fy * G.fz;
  G.bsize = (long long)G.bx * G.by * G.bz;
  G.N0 = G.fsize * d.ncomp;
  G.N1 = G.bsize * d.ncomp;
  const double H = 1.0 / d.n, h = H / 2.0;
  G.sf = d.mu * std::pow(h, d.dim - 2);
  G.sb = d.mu * std::pow(H, d.dim - 2);
  G.wcf = d.mu * (4.0 / 3.0) * std::pow(H, d.dim - 2);
  G.nch = d.dim == 3 ? 4 : 2;
  auto split = [](double x, float* h, float* l) {
    *h = (float)x;
    *l = (float)(x - (double)*h);
  };
  split(G.sf, &G.sf_h, &G.sf_l);
  split(G.sb, &G.sb_h, &G.sb_l);
  split(G.wcf, &G.wcf_h, &G.wcf_l);
  split(G.wcf / ((double)G.nch * G.nch), &G.w2_h, &G.w2_l);
  split(G.wcf / G.nch, &G.w1_h, &G.w1_l);
  return G;
}

template <typename T>
selm_status residual_t(selm_comp* C, const double* z, const double* b, T* rp, T* rb, double* norm2, cudaStream_t st) {
  prof::Scope ps(SELM_K_OUTER_RESIDUAL, st);
  k_comp_residual<T><<<cgrid(C->geo.N0 + C->geo.N1), kCBlock, 0, st>>>(C->geo, z, b, rp, rb, norm2);
  CCK(cudaGetLastError());
  return SELM_OK;
}

template <typename T>
selm_status patch_sweeps_t(selm_comp* C, T* vp, const T* vb, const T* rp, int count, bool noise,
                           const unsigned long long* cyc, cudaStream_t st) {
  const CompGeo& G = C->geo;
  const Key key = C->mg->key;
  const bool v8 = G.fx % 8 == 0;
  for (int s = 0; s < count; ++s)
    for (int pass = 0; pass < 4; ++pass) {
      prof::Scope ps(SELM_K_FINE_SWEEP, st);
      const long long rows = (long long)((pass & 1) ? 2 : G.fz) * G.fy * G.ncomp;
      if (v8 && !(pass & 1)) {   // main pass: march along the layers (chunks of 16)
        const int kc = 16;
        const long long nt = (long long)G.fy * (G.fx >> 3) * ((G.fz + kc - 1) / kc) * G.ncomp;
        if (noise)
          k_comp_patch_zm<T, true><<<cgrid(nt), kCBlock, 0, st>>>(G, vp, vb, rp, pass >> 1, s, kc, key, cyc);
        else
          k_comp_patch_zm<T, false><<<cgrid(nt), kCBlock, 0, st>>>(G, vp, vb, rp, pass >> 1, s, kc, key, cyc);
      } else if (v8) {
        const long long nt = rows * (G.fx >> 3);
        if (noise)
          k_comp_patch_v8<T, true><<<cgrid(nt), kCBlock, 0, st>>>(G, vp, vb, rp, pass, s, key, cyc);
        else
          k_comp_patch_v8<T, false><<<cgrid(nt), kCBlock, 0, st>>>(G, vp, vb, rp, pass, s, key, cyc);
      } else {
        const long long nt = rows * (G.fx >> 1);
        if (noise)
          k_comp_patch<T, true><<<cgrid(nt), kCBlock, 0, st>>>(G, vp, vb, rp, pass, s, key, cyc);
        else
          k_comp_patch<T, false><<<cgrid(nt), kCBlock, 0, st>>>(G, vp, vb, rp, pass, s, key, cyc);
      }
    }
  CCK(cudaGetLastError());
  return SELM_OK;
}

// The correction half of one FAC iteration, after residual_t filled the
// level-0 and level-1 b fields from z: restrict, base V-cycle, prolong, patch
// sweeps, z += q.
template <typename T>
selm_status correct_t(selm_comp* C, double* z, bool noise, const unsigned long long* cyc, cudaStream_t st,
                      float* zh = nullptr, float* zl = nullptr) {
  const CompGeo& G = C->geo;
  Sys& s = C->mg->vel;
  T* rp = (T*)s.b[0];
  T* rb = (T*)s.b[1];
  {
    prof::Scope ps(SELM_K_RESTRICT, st);
    k_comp_restrict<T><<<cgrid((long long)G.K * G.by * G.bx * G.ncomp), kCBlock, 0, st>>>(G, rp, rb);
  }
  CCK(cudaGetLastError());
  CCK(cudaMemsetAsync(s.v[1], 0, (size_t)G.N1 * sizeof(T), st));
  selm_status r = vcycle_level(C->mg, s, 1, noise, cyc, st);
  if (r != SELM_OK) {
    C->err = C->mg->err;
    return r;
  }
  {
    prof::Scope ps(SELM_K_PROLONG, st);
    if (G.fx % 8 == 0)
      k_comp_prolong_v8<T><<<cgrid((long long)G.fz * G.fy * (G.fx >> 3) * G.ncomp), kCBlock, 0, st>>>(
          G, (T*)s.v[0], (const T*)s.v[1]);
    else
      k_comp_prolong<T><<<cgrid(G.N0), kCBlock, 0, st>>>(G, (T*)s.v[0], (const T*)s.v[1]);
  }
  CCK(cudaGetLastError());
  r = patch_sweeps_t<T>(C, (T*)s.v[0], (const T*)s.v[1], rp, C->nu, noise, cyc, st);
  if (r != SELM_OK) return r;
  {
    prof::Scope ps(SELM_K_OUTER_UPDATE, st);
    if (zh)
      k_comp_update_df<<<cgrid(G.N0 + G.N1), kCBlock, 0, st>>>(G, zh, zl, (const float*)s.v[0],
                                                               (const float*)s.v[1]);
    else
      k_comp_update<T><<<cgrid(G.N0 + G.N1), kCBlock, 0, st>>>(G, z, (const T*)s.v[0], (const T*)s.v[1]);
  }
  CCK(cudaGetLastError());
  C->total_cycles += 1;
  return SELM_OK;
}

selm_status fac_cycle(selm_comp* C, double* z, const double* b, bool noise, const unsigned long long* cyc,
                      double* norm2, cudaStream_t st) {
  Sys& s = C->mg->vel;
  selm_status r;
  if (C->mg->esize == 4) {
    r = residual_t<float>(C, z, b, (float*)s.b[0], (float*)s.b[1], norm2, st);
    if (r == SELM_OK) r = correct_t<float>(C, z, noise, cyc, st);
  } else {
    r = residual_t<double>(C, z, b, (double*)s.b[0], (double*)s.b[1], norm2, st);
    if (r == SELM_OK) r = correct_t<double>(C, z, noise, cyc, st);
  }
  return r;
}

// One stochastic FAC iteration of the handle's chain (b = 0).
selm_status chain_cycle(selm_comp* C, const unsigned long long* cyc, cudaStream_t st) {
  if (!C->xh) return fac_cycle(C, C->xi, nullptr, true, cyc, nullptr, st);
  Sys& s = C->mg->vel;
  const CompGeo& G = C->geo;
  if (G.fx % 8 == 0 && G.bx % 8 == 0) {
    {
      prof::Scope ps(SELM_K_OUTER_RESIDUAL, st);
      k_comp_residual_df_patch<<<cgrid((long long)G.fz * G.fy * (G.fx >> 3) * G.ncomp), kCBlock, 0, st>>>(
          G, C->xh, C->xl, (float*)s.b[0]);
    }
    prof::Scope ps(SELM_K_OUTER_RESIDUAL, st);
    k_comp_residual_df_base<<<cgrid((long long)(G.bz - G.K) * G.by * (G.bx >> 3) * G.ncomp), kCBlock, 0, st>>>(
        G, C->xh, C->xl, (float*)s.b[1]);
  } else {
    prof::Scope ps(SELM_K_OUTER_RESIDUAL, st);
    k_comp_residual_df<<<cgrid(G.N0 + G.N1), kCBlock, 0, st>>>(G, C->xh, C->xl, (float*)s.b[0], (float*)s.b[1]);
  }
  CCK(cudaGetLastError());
  return correct_t<float>(C, nullptr, true, cyc, st, C->xh, C->xl);
}

selm_status read_slot(selm_comp* C, int slot, double* out, cudaStream_t st) {
  CCK(cudaMemcpyAsync(C->host_red, C->red + slot, sizeof(double), cudaMemcpyDeviceToHost, st));
  CCK(cudaStreamSynchronize(st));
  *out = *C->host_red;
  return SELM_OK;
}

}  // namespace

extern "C" {

long long selm_comp_size(const selm_comp* C) { return C ? C->geo.N0 + C->geo.N1 : 0; }

size_t selm_comp_footprint(const selm_comp_desc* desc) {
  if (!desc) return 0;
  selm_comp_desc d = *desc;
  if (!fill_comp_defaults(&d).empty()) return 0;
  HostSystem hs;
  if (!build_composite_system(d.dim, d.n, d.K, d.levels, d.mu, d.ncomp, &hs).empty()) return 0;
  const CompGeo G = make_geo(d);
  return footprint_with_host(internal_desc(d), hs, (size_t)(G.N0 + G.N1) * sizeof(double));
}

selm_status selm_comp_create(const selm_comp_desc* desc, void* stream, selm_comp** out) {
  if (!desc || !out) return SELM_EINVAL;
  *out = nullptr;
  selm_comp_desc d = *desc;
  std::string e = fill_comp_defaults(&d);
  HostSystem hs;
  if (e.empty()) e = build_composite_system(d.dim, d.n, d.K, d.levels, d.mu, d.ncomp, &hs);
  if (!e.empty()) {
    std::fprintf(stderr, "selm_comp_create: %s\n", e.c_str());
    return SELM_EINVAL;
  }
  selm_comp* C = new (std::nothrow) selm_comp();
  if (!C) return SELM_ENOMEM;
  C->d = d;
  C->geo = make_geo(d);
  C->nu = d.nu_patch;
  size_t xoff = 0;
  cudaStream_t st = CS(stream);
  // level 1 (the base grid, 7-point) is smoothed red-black by its own
  // launches; the levels from 2 go to the cluster engine where their slabs fit
  // in shared memory, and the larger ones above it to cooperative launches
  selm_status r = create_with_host(internal_desc(d), hs, 2, true, 1,
                                   (size_t)(C->geo.N0 + C->geo.N1) * sizeof(double), st, &C->mg, &xoff);
  if (r != SELM_OK) {
    delete C;
    return r;
  }
  if (C->mg->esize == 4) {
    C->xh = (float*)(C->mg->ws + xoff);
    C->xl = C->xh + (C->geo.N0 + C->geo.N1);
  } else {
    C->xi = (double*)(C->mg->ws + xoff);
  }
  C->red = C->mg->red;
  C->host_red = new (std::nothrow) double[2];
  cudaError_t ce = cudaMemsetAsync(C->mg->ws + xoff, 0, (size_t)(C->geo.N0 + C->geo.N1) * sizeof(double), st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (!C->host_red || ce != cudaSuccess) {
    const selm_status why = C->host_red ? SELM_ECUDA : SELM_ENOMEM;
    selm_comp_destroy(C);
    return why;
  }
  *out = C;
  return SELM_OK;
}

selm_status selm_comp_destroy(selm_comp* C) {
  if (!C) return SELM_EINVAL;
  if (C->chain_graph) cudaGraphExecDestroy(C->chain_graph);
  if (C->mg) selm_mg_destroy(C->mg);
  delete[] C->host_red;
  delete C;
  return SELM_OK;
}

const char* selm_comp_last_error(const selm_comp* C) { return C ? C->err.c_str() : "null handle"; }

selm_status selm_comp_layout(const selm_comp* C, int part, int comp, int dims[3], long long* offset,
                             long long* size) {
  if (!C || comp < 0 || comp >= C->geo.ncomp || (part != 0 && part != 1)) return SELM_EINVAL;
  const CompGeo& G = C->geo;
  if (dims) {
    dims[0] = part == 0 ? G.fx : G.bx;
    dims[1] = part == 0 ? G.fy : G.by;
    dims[2] = part == 0 ? G.fz : G.bz;
  }
  if (offset) *offset = part == 0 ? comp * G.fsize : G.N0 + comp * G.bsize;
  if (size) *size = part == 0 ? G.fsize : G.bsize;
  return SELM_OK;
}

int selm_comp_inner_bytes(const selm_comp* C) { return C ? C->mg->esize : 0; }

selm_status selm_comp_residual(selm_comp* C, const double* z, const double* b, double* r, double* norm2,
                               void* stream) {
  if (!C || !z || !r) return SELM_EINVAL;
  cudaStream_t st = CS(stream);
  CCK(cudaMemsetAsync(r, 0, (size_t)(C->geo.N0 + C->geo.N1) * sizeof(double), st));
  if (norm2) CCK(cudaMemsetAsync(C->red + 2, 0, sizeof(double), st));
  selm_status s = residual_t<double>(C, z, b, r, r + C->geo.N0, norm2 ? C->red + 2 : nullptr, st);
  if (s != SELM_OK) return s;
  if (norm2) return read_slot(C, 2, norm2, st);
  return SELM_OK;
}

selm_status selm_comp_patch_sweeps(selm_comp* C, void* q_patch, const void* q_base, const void* r_patch, int count,
                                   uint64_t cycle, int noise, void* stream) {
  if (!C || !q_patch || !q_base || !r_patch || count < 0 || count > 64) return SELM_EINVAL;
  cudaStream_t st = CS(stream);
  if (launch_set_u64(C->mg->cyc + 1, cycle, st) != cudaSuccess) return SELM_ECUDA;
  if (C->mg->esize == 4)
    return patch_sweeps_t<float>(C, (float*)q_patch, (const float*)q_base, (const float*)r_patch, count, noise != 0,
                                 C->mg->cyc + 1, st);
  return patch_sweeps_t<double>(C, (double*)q_patch, (const double*)q_base, (const double*)r_patch, count,
                                noise != 0, C->mg->cyc + 1, st);
}

selm_status selm_comp_fac_cycle(selm_comp* C, double* z, const double* b, uint64_t cycle, int noise, void* stream) {
  if (!C || !z) return SELM_EINVAL;
  cudaStream_t st = CS(stream);
  if (launch_set_u64(C->mg->cyc + 1, cycle, st) != cudaSuccess) return SELM_ECUDA;
  return fac_cycle(C, z, b, noise != 0, C->mg->cyc + 1, nullptr, st);
}

selm_status selm_comp_solve(selm_comp* C, double* z, const double* b, double tol, int max_cycles, int* cycles,
                            double* rel_out, void* stream) {
  if (!C || !z || !b || !(tol > 0.0) || max_cycles < 0) return SELM_EINVAL;
  cudaStream_t st = CS(stream);
  const CompGeo& G = C->geo;
  CCK(cudaMemsetAsync(C->red, 0, 2 * sizeof(double), st));
  {
    prof::Scope ps(SELM_K_OTHER, st);
    k_comp_norm2<<<cgrid(G.N0 + G.N1), kCBlock, 0, st>>>(G, b, C->red);
  }
  CCK(cudaGetLastError());
  double bn2 = 0.0;
  selm_status r = read_slot(C, 0, &bn2, st);
  if (r != SELM_OK) return r;
  if (cycles) *cycles = 0;
  if (bn2 == 0.0) {
    CCK(cudaMemsetAsync(z, 0, (size_t)(G.N0 + G.N1) * sizeof(double), st));
    if (rel_out) *rel_out = 0.0;
    return SELM_OK;
  }
  const double bn = std::sqrt(bn2);
  Sys& s = C->mg->vel;
  for (int cyc = 0;; ++cyc) {
    CCK(cudaMemsetAsync(C->red + 1, 0, sizeof(double), st));
    if (C->mg->esize == 4)
      r = residual_t<float>(C, z, b, (float*)s.b[0], (float*)s.b[1], C->red + 1, st);
    else
      r = residual_t<double>(C, z, b, (double*)s.b[0], (double*)s.b[1], C->red + 1, st);
    if (r != SELM_OK) return r;
    double rn2 = 0.0;
    r = read_slot(C, 1, &rn2, st);
    if (r != SELM_OK) return r;
    const double rel = std::sqrt(rn2) / bn;
    if (rel_out) *rel_out = rel;
    if (rel <= tol) {
      if (cycles) *cycles = cyc;
      return SELM_OK;
    }
    if (cyc >= max_cycles) {
      if (cycles) *cycles = cyc;
      C->err = "composite FAC solve did not converge";
      return SELM_ENOCONV;
    }
    r = C->mg->esize == 4 ? correct_t<float>(C, z, false, C->mg->cyc + 1, st)
                          : correct_t<double>(C, z, false, C->mg->cyc + 1, st);
    if (r != SELM_OK) return r;
  }
}

// One chain cycle and its counter increment, directly or (from the second
// cycle of the handle on, with graphs on and profiling off) as a replay of
// the captured cycle: the same launches on the same buffers, the counter read
// from device memory.  Host counters moved by the capture are undone, and
// each replay credits them.
static selm_status chain_step(selm_comp* C, cudaStream_t st) {
  selm_mg* h = C->mg;
  const bool graph = h->graphs && h->cap && !prof::g_on;
  if (!graph || (!C->chain_graph && C->chain_runs++ == 0)) {
    selm_status r = chain_cycle(C, h->cyc + 0, st);
    if (r != SELM_OK) return r;
    return launch_inc_u64(h->cyc + 0, st) == cudaSuccess ? SELM_OK : SELM_ECUDA;
  }
  if (!C->chain_graph) {
    const long long l0 = prof::g_launches.load(), v0 = h->total_vcycles, c0 = C->total_cycles;
    if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      h->graphs = false;
      return chain_step(C, st);
    }
    selm_status r = chain_cycle(C, h->cyc + 0, h->cap);
    if (r == SELM_OK && launch_inc_u64(h->cyc + 0, h->cap) != cudaSuccess) r = SELM_ECUDA;
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->cap, &g);
    C->graph_launches = prof::g_launches.load() - l0;
    C->graph_vcycles = h->total_vcycles - v0;
    prof::g_launches.fetch_sub(C->graph_launches);   // recorded, not run
    h->total_vcycles = v0;
    C->total_cycles = c0;
    if (r != SELM_OK || e != cudaSuccess || !g || cudaGraphInstantiate(&C->chain_graph, g, 0) != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      C->chain_graph = nullptr;
      h->graphs = false;   // direct cycles from now on
      return chain_step(C, st);
    }
    cudaGraphDestroy(g);
  }
  CCK(cudaGraphLaunch(C->chain_graph, st));
  prof::g_launches.fetch_add(C->graph_launches);
  h->total_vcycles += C->graph_vcycles;
  C->total_cycles += 1;
  return SELM_OK;
}

selm_status selm_comp_sample(selm_comp* C, int ncycles, double* xi_out, void* stream) {
  if (!C || ncycles < 0) return SELM_EINVAL;
  cudaStream_t st = CS(stream);
  for (int q = 0; q < ncycles; ++q) {
    selm_status r = chain_step(C, st);
    if (r != SELM_OK) return r;
    C->cycle += 1;
  }
  if (xi_out) {
    if (C->xh) {
      prof::Scope ps(SELM_K_OTHER, st);
      k_comp_df_to_f64<<<cgrid(C->geo.N0 + C->geo.N1), kCBlock, 0, st>>>(C->geo, C->xh, C->xl, xi_out);
      CCK(cudaGetLastError());
    } else {
      CCK(cudaMemcpyAsync(xi_out, C->xi, (size_t)(C->geo.N0 + C->geo.N1) * sizeof(double), cudaMemcpyDeviceToDevice,
                          st));
    }
  }
  return SELM_OK;
}

selm_status selm_comp_chain(selm_comp* C, uint64_t* cycle) {
  if (!C) return SELM_EINVAL;
  if (cycle) *cycle = C->cycle;
  return SELM_OK;
}

selm_status selm_comp_set_cycle(selm_comp* C, uint64_t cycle) {
  if (!C) return SELM_EINVAL;
  if (launch_set_u64(C->mg->cyc + 0, cycle, nullptr) != cudaSuccess || cudaStreamSynchronize(nullptr) != cudaSuccess)
    return SELM_ECUDA;
  C->cycle = cycle;
  return SELM_OK;
}

selm_status selm_comp_stats(const selm_comp* C, long long* total_cycles) {
  if (!C) return SELM_EINVAL;
  if (total_cycles) *total_cycles = C->total_cycles;
  return SELM_OK;
}

}  // extern "C"
