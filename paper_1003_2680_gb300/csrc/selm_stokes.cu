// Exact discrete Stokes mobility near walls and the Ito drift of the
// particle dynamics (corrections beyond the paper's formula M = Gamma P~ A^-1
// P~ Gamma^T, which is the Stokes mobility only where P~ commutes with A).
//
// Stokes solve.  The MAC saddle point A u + D^T p = f, D u = 0 (D the
// integer divergence) is solved for its velocity u = S f by conjugate
// gradients on the pressure Schur complement
//     (D A^-1 D^T) p = D A^-1 f,     u = A^-1 f - A^-1 D^T p,
// every application of A^-1 being a FAC solve of the handle's velocity
// system (Algorithm 1) to a tolerance a hundred times tighter than the
// outer one.  The Schur complement is symmetric positive semidefinite with
// the constants as its kernel, and the right-hand side D(.) sums to zero, so
// plain CG converges on the mean-free pressures; u is accumulated from the
// A^-1 D^T d_k of the iterations, so no solve is repeated at the end.  The
// complement is close to a multiple of the identity away from the walls, so
// the iteration count hardly grows with the grid.
//
// Thermal velocities with covariance 2 kT Gamma S Gamma^T come from the
// chain xi ~ N(0, A^-1): Cov(S A xi) = S.  The Ito drift kT div_X M is the
// random finite difference (kT / delta)[M(X + delta W/2) - M(X - delta W/2)] W
// with W ~ N(0, I) from Philox (kind 3, rank = particle * dim + axis,
// counter words 2-3 = the handle's step index).

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>

#include "../../include/selm_mg.h"
#include "selm_devmath.h"
#include "selm_handle.h"
#include "selm_launch.h"
#include "selm_prof.h"

using namespace selm;

namespace {

constexpr int kT = 256;
constexpr int kRed = 304;   // reduction blocks (2 per SM)

__device__ double block_sum_s(double a) {
  __shared__ double sh[kT / 32];
  for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  __syncthreads();
  return s;
}

// part[block] = sum x . y over the block's grid-stride share (fixed order).
__global__ void __launch_bounds__(kT) k_sdot(long long n, const double* __restrict__ x, const double* __restrict__ y,
                                            double* __restrict__ part) {
  double a = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    a += x[i] * y[i];
  a = block_sum_s(a);
  if (threadIdx.x == 0) part[blockIdx.x] = a;
}

__global__ void __launch_bounds__(kT) k_sreduce(const double* __restrict__ part, int nb, double* __restrict__ out) {
  double a = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) a += part[i];
  a = block_sum_s(a);
  if (threadIdx.x == 0) *out = a;
}

// y = a x + y
__global__ void __launch_bounds__(kT) k_saxpy(long long n, double a, const double* __restrict__ x,
                                             double* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}

// y = x + b y
__global__ void __launch_bounds__(kT) k_sxpby(long long n, const double* __restrict__ x, double b,
                                             double* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = x[i] + b * y[i];
}

__global__ void __launch_bounds__(kT) k_sneg(long long n, double* __restrict__ x) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = -x[i];
}

// out = X + s W  ([n] entries)
__global__ void __launch_bounds__(kT) k_shift(long long n, const double* __restrict__ X, double s,
                                             const double* __restrict__ W, double* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = X[i] + s * W[i];
}

// W[r] = normal of rank r (Philox kind 3, counter words 2-3 = step).
__global__ void __launch_bounds__(kT) k_rfd_normals(long long n, Key key, unsigned long long step,
                                                   double* __restrict__ W) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const uint32_t c1 = 3u << 20;
  const uint4 w = philox4x32_10(make_uint4((uint32_t)(r >> 2), c1, (uint32_t)step, (uint32_t)(step >> 32)), key.k0,
                                key.k1);
  double g;
  normal_of(w, (int)(r & 3), &g);
  W[r] = g;
}

unsigned nblk(long long n) { return (unsigned)((n + kT - 1) / kT); }
unsigned rblk(long long n) {
  long long b = (n + kT - 1) / kT;
  return (unsigned)(b < 1 ? 1 : (b > kRed ? kRed : b));
}

#define SCK(call)                                                        \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) {                                             \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_);       \
      return SELM_ECUDA;                                                 \
    }                                                                    \
  } while (0)
#define SST(x)                       \
  do {                               \
    selm_status r_ = (x);            \
    if (r_ != SELM_OK) return r_;    \
  } while (0)

// Scratch: velocity fields y, w, u0; pressure fields p, r, d, q; partials
// and scalars; particle buffers (2 position sets, 2 velocity sets, W).
struct Scratch {
  double *y, *w, *u0, *p, *r, *d, *q, *part, *sc, *Xp, *Xm, *Up, *Um, *W, *f;
};

Scratch carve(selm_mg* h) {
  const long long nv = h->vel.lev[0].size;
  const long long nc = (long long)h->vel.lev[0].c[0].nx * h->vel.lev[0].c[0].ny * h->vel.lev[0].c[0].nz;
  const long long npd = (long long)h->d.max_particles * 3;
  double* b = (double*)h->stokes;
  Scratch s;
  auto take = [&](long long n) {
    double* p = b;
    b += (n + 31) / 32 * 32;
    return p;
  };
  s.y = take(nv);
  s.w = take(nv);
  s.u0 = take(nv);
  s.f = take(nv);
  s.p = take(nc);
  s.r = take(nc);
  s.d = take(nc);
  s.q = take(nc);
  s.part = take(kRed);
  s.sc = take(32);
  s.Xp = take(npd);
  s.Xm = take(npd);
  s.Up = take(npd);
  s.Um = take(npd);
  s.W = take(npd);
  return s;
}

selm_status ensure_scratch(selm_mg* h) {
  if (h->stokes) return SELM_OK;
  const long long nv = h->vel.lev[0].size;
  const long long nc = (long long)h->vel.lev[0].c[0].nx * h->vel.lev[0].c[0].ny * h->vel.lev[0].c[0].nz;
  const long long npd = (long long)h->d.max_particles * 3;
  const size_t doubles = (size_t)(4 * ((nv + 31) / 32 * 32) + 4 * ((nc + 31) / 32 * 32) + kRed + 32 +
                                  5 * ((npd + 31) / 32 * 32));
  const size_t bytes = doubles * sizeof(double);
  void* p = nullptr;
  if (h->d.alloc) {
    p = h->d.alloc(bytes, h->d.alloc_ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (!p) {
    h->err = "allocation of the Stokes scratch failed";
    return SELM_ENOMEM;
  }
  h->stokes = p;
  h->stokes_bytes = bytes;
  return SELM_OK;
}

selm_status sdot(selm_mg* h, const Scratch& s, long long n, const double* x, const double* y, int slot,
                 cudaStream_t st) {
  const unsigned nb = rblk(n);
  prof::Scope ps(SELM_K_PROJECTION, st);
  k_sdot<<<nb, kT, 0, st>>>(n, x, y, s.part);
  k_sreduce<<<1, kT, 0, st>>>(s.part, (int)nb, s.sc + slot);
  SCK(cudaGetLastError());
  return SELM_OK;
}

selm_status read_sc(selm_mg* h, const Scratch& s, double* out, int n, cudaStream_t st) {
  SCK(cudaMemcpyAsync(out, s.sc, n * sizeof(double), cudaMemcpyDeviceToHost, st));
  SCK(cudaStreamSynchronize(st));
  return SELM_OK;
}

// z = A^-1 b (FAC solve from zero).  A solve that stops short of tol only
// at the rounding floor of its right-hand side (relative residual below
// 1e-12) is accepted: the outer iteration then decides whether the Stokes
// velocity met its own tolerance.
selm_status ainv(selm_mg* h, double* z, const double* b, double tol, cudaStream_t st) {
  SCK(cudaMemsetAsync(z, 0, (size_t)h->vel.lev[0].size * sizeof(double), st));
  int cycles = 0;
  double rel = 0.0;
  const selm_status r = selm_mg_fac_solve(h, SELM_SYS_VELOCITY, z, b, tol, h->d.max_cycles > 0 ? h->d.max_cycles : 100,
                                          &cycles, &rel, st);
  if (r == SELM_ENOCONV && rel <= 1e-12) {
    h->err.clear();
    return SELM_OK;
  }
  return r;
}

// y = A^-1 D^T x (w: scratch velocity field).
selm_status ainv_dt(selm_mg* h, const Scratch& s, const double* x, double* y, double tol_in, cudaStream_t st) {
  const long long nv = h->vel.lev[0].size;
  SCK(cudaMemsetAsync(s.w, 0, (size_t)nv * sizeof(double), st));
  SCK(launch_grad_sub(h->vel.lev[0], s.w, x, st));   // w = -D^T x
  {
    prof::Scope ps(SELM_K_PROJECTION, st);
    k_sneg<<<nblk(nv), kT, 0, st>>>(nv, s.w);
    SCK(cudaGetLastError());
  }
  // A^-1 of a zero field is zero (the solve would stop at once anyway)
  return ainv(h, y, s.w, tol_in, st);
}

// u = S f; iters / resid: outer CG iterations and relative Schur residual.
selm_status stokes_solve(selm_mg* h, const double* f, double* u, double tol, int* iters, double* resid,
                         cudaStream_t st) {
  SST(ensure_scratch(h));
  const Scratch s = carve(h);
  const long long nv = h->vel.lev[0].size;
  const long long nc = (long long)h->vel.lev[0].c[0].nx * h->vel.lev[0].c[0].ny * h->vel.lev[0].c[0].nz;
  const double tol_in = tol * 1e-2 > 1e-14 ? tol * 1e-2 : 1e-14;
  // u0 = A^-1 f, r = D u0 (the Schur right-hand side), p = 0
  {
    double hs[2];
    SST(sdot(h, s, nv, f, f, 0, st));
    SST(read_sc(h, s, hs, 1, st));
    if (hs[0] == 0.0) {
      SCK(cudaMemsetAsync(u, 0, (size_t)nv * sizeof(double), st));
      if (iters) *iters = 0;
      if (resid) *resid = 0.0;
      return SELM_OK;
    }
  }
  SST(ainv(h, s.u0, f, tol_in, st));
  SCK(launch_divergence(h->vel.lev[0], s.u0, s.r, s.sc + 16, st));   // r = D u0
  SCK(cudaMemcpyAsync(u, s.u0, (size_t)nv * sizeof(double), cudaMemcpyDeviceToDevice, st));
  SCK(cudaMemcpyAsync(s.d, s.r, (size_t)nc * sizeof(double), cudaMemcpyDeviceToDevice, st));
  double hs[4];
  SST(sdot(h, s, nc, s.r, s.r, 0, st));
  SST(read_sc(h, s, hs, 1, st));
  const double r0 = std::sqrt(hs[0]);
  double rr = hs[0];
  int it = 0;
  const int max_it = 500;
  while (std::sqrt(rr) > tol * r0 && it < max_it) {
    // q = D A^-1 D^T d, y = A^-1 D^T d
    SST(ainv_dt(h, s, s.d, s.y, tol_in, st));
    SCK(launch_divergence(h->vel.lev[0], s.y, s.q, s.sc + 16, st));
    SST(sdot(h, s, nc, s.d, s.q, 1, st));
    SST(read_sc(h, s, hs, 2, st));
    if (!(hs[1] > 0.0)) break;
    const double alpha = rr / hs[1];
    {
      prof::Scope ps(SELM_K_PROJECTION, st);
      k_saxpy<<<nblk(nv), kT, 0, st>>>(nv, -alpha, s.y, u);      // u -= alpha A^-1 D^T d
      k_saxpy<<<nblk(nc), kT, 0, st>>>(nc, -alpha, s.q, s.r);    // r -= alpha q
      SCK(cudaGetLastError());
    }
    SST(sdot(h, s, nc, s.r, s.r, 0, st));
    SST(read_sc(h, s, hs, 1, st));
    const double rr_new = hs[0];
    {
      prof::Scope ps(SELM_K_PROJECTION, st);
      k_sxpby<<<nblk(nc), kT, 0, st>>>(nc, s.r, rr_new / rr, s.d);   // d = r + beta d
      SCK(cudaGetLastError());
    }
    rr = rr_new;
    ++it;
  }
  if (iters) *iters = it;
  if (resid) *resid = std::sqrt(rr) / r0;
  if (std::sqrt(rr) > tol * r0) {
    h->err = "Stokes solve did not reach tol";
    return SELM_ENOCONV;
  }
  return SELM_OK;
}

// U = Gamma S Gamma^T F at X (velocity field scratch: s.f, s.y via the solve).
selm_status stokes_mobility(selm_mg* h, const Scratch& s, int np, const double* X, const double* F, double* U,
                            double* field, cudaStream_t st) {
  SST(selm_mg_spread(h, np, X, F, s.f, st));
  SST(stokes_solve(h, s.f, field, h->d.tol, nullptr, nullptr, st));
  return selm_mg_interp(h, np, X, field, U, st);
}

selm_status rfd_drift(selm_mg* h, int np, const double* X, const double* W, double delta, double* d,
                      cudaStream_t st) {
  SST(ensure_scratch(h));
  const Scratch s = carve(h);
  const long long n = (long long)np * h->d.dim;
  {
    prof::Scope ps(SELM_K_OTHER, st);
    k_shift<<<nblk(n), kT, 0, st>>>(n, X, 0.5 * delta, W, s.Xp);
    k_shift<<<nblk(n), kT, 0, st>>>(n, X, -0.5 * delta, W, s.Xm);
    SCK(cudaGetLastError());
  }
  SST(stokes_mobility(h, s, np, s.Xp, W, s.Up, h->wcomb, st));
  SST(stokes_mobility(h, s, np, s.Xm, W, s.Um, h->wcomb, st));
  const double c = h->d.kT / delta;
  SCK(launch_axpby(n, c, s.Up, -c, s.Um, d, st));
  return SELM_OK;
}

}  // namespace

namespace selm {

void stokes_release(selm_mg* h) {
  if (!h || !h->stokes) return;
  if (h->d.free)
    h->d.free(h->stokes, h->d.alloc_ctx);
  else
    cudaFree(h->stokes);
  h->stokes = nullptr;
}

}  // namespace selm

extern "C" {

selm_status selm_mg_stokes_solve(selm_mg* h, const double* f, double* u, double tol, int* iters, double* resid,
                                 void* stream) {
  if (!h || !f || !u || tol < 0.0) return SELM_EINVAL;
  return stokes_solve(h, f, u, tol > 0.0 ? tol : h->d.tol, iters, resid, (cudaStream_t)stream);
}

selm_status selm_mg_stokes_mobility(selm_mg* h, int np, const double* X, const double* F, double* U, void* stream) {
  if (!h || np < 0 || np > h->d.max_particles || (np > 0 && (!X || !F || !U))) return SELM_EINVAL;
  if (np == 0) return SELM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  SST(ensure_scratch(h));
  const Scratch s = carve(h);
  return stokes_mobility(h, s, np, X, F, U, h->wcomb, st);
}

selm_status selm_mg_rfd_directions(selm_mg* h, int np, uint64_t step, double* W, void* stream) {
  if (!h || np < 0 || (np > 0 && !W)) return SELM_EINVAL;
  const long long n = (long long)np * h->d.dim;
  if (n == 0) return SELM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  prof::Scope ps(SELM_K_OTHER, st);
  k_rfd_normals<<<nblk(n), kT, 0, st>>>(n, h->key, step, W);
  SCK(cudaGetLastError());
  return SELM_OK;
}

selm_status selm_mg_rfd_drift(selm_mg* h, int np, const double* X, const double* W, double delta, double* d,
                              void* stream) {
  if (!h || np < 0 || np > h->d.max_particles || !(delta > 0.0) || (np > 0 && (!X || !W || !d))) return SELM_EINVAL;
  if (np == 0) return SELM_OK;
  return rfd_drift(h, np, X, W, delta, d, (cudaStream_t)stream);
}

selm_status selm_mg_stokes_step(selm_mg* h, int np, double* X, const double* F, double dt, int nsteps, int ncycles,
                                double delta, void* stream) {
  if (!h || np < 0 || np > h->d.max_particles || nsteps < 0 || ncycles < 0 || !(dt >= 0.0) || delta < 0.0 ||
      (np > 0 && (!X || !F)))
    return SELM_EINVAL;
  if (np == 0 || nsteps == 0) return SELM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  SST(ensure_scratch(h));
  const Scratch s = carve(h);
  const long long n = (long long)np * h->d.dim;
  const long long nv = h->vel.lev[0].size;
  for (int k = 0; k < nsteps; ++k) {
    // the drift at the step's start positions
    const bool drift = delta > 0.0 && h->d.kT > 0.0;
    if (drift) {
      {
        prof::Scope ps(SELM_K_OTHER, st);
        k_rfd_normals<<<nblk(n), kT, 0, st>>>(n, h->key, h->stokes_step, s.W);
        SCK(cudaGetLastError());
      }
      SST(rfd_drift(h, np, X, s.W, delta, h->V, st));     // V = d
    }
    SST(chain_advance(h, ncycles, st));
    // w = S (dt Gamma^T F + sqrt(2 kT dt) A xi)
    SST(selm_mg_spread(h, np, X, F, s.f, st));
    SCK(launch_outer_residual<double>(h->vel.lev[0], h->xi, nullptr, s.y, nullptr, st));   // y = -A xi
    SCK(launch_axpby(nv, dt, s.f, -std::sqrt(2.0 * h->d.kT * dt), s.y, s.f, st));
    SST(stokes_solve(h, s.f, h->wcomb, h->d.tol, nullptr, nullptr, st));
    SST(selm_mg_interp(h, np, X, h->wcomb, s.Up, st));
    // X += Gamma w + dt d
    if (drift) SCK(launch_axpby(n, 1.0, s.Up, dt, h->V, s.Up, st));
    SCK(launch_em(np, h->d.dim, X, s.Up, st));
    h->stokes_step += 1;
  }
  return SELM_OK;
}

}  // extern "C"
