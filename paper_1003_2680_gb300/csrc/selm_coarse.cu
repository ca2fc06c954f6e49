// Coarse-level engine: the part of the V-cycle (Algorithm 3) below the finest
// level, for one component per thread-block cluster.
//
// Why: on the Galerkin levels the 3x3x5 stencil needs 12 colour classes, so a
// V-cycle runs ~200 dependent colour passes on small grids.  As separate
// launches each pass costs a full launch plus a chain of dependent global
// loads.  Here one cluster per velocity component runs all of them:
//   * "cluster" levels are split into z-slabs, one per CTA; a CTA keeps its
//     slab plus two halo planes on each side in shared memory and, after
//     updating a site that lies in a neighbour's halo, stores the new value
//     into the neighbour's shared memory (DSMEM); cluster barriers separate
//     the colour passes;
//   * "single" levels (small grids) are held entirely by CTA 0, which runs
//     their passes with block barriers while the other CTAs wait at the next
//     cluster barrier;
//   * b, residuals and the hand-off of corrections between levels go through
//     global memory (L2), read with L1-bypassing loads.
// The visiting order (colour classes in increasing id, all sites of a class
// updated together) and the Philox streams are those of the per-pass kernels,
// so both paths produce the same chain.

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "../../include/selm_mg.h"
#include "selm_coarse.h"
#include "selm_internal.h"
#include "selm_devmath.h"
#include "selm_prof.h"

namespace cg = cooperative_groups;

namespace selm {
namespace {

// Threads per CTA: 512, which leaves up to 128 registers a thread for the
// unrolled 45-point row (at 1024 threads the 64-register cap spills it and
// the colour passes on the engine's levels run slower).
template <typename T>
struct EngThreads {
  static constexpr int value = 512;
};

__device__ __forceinline__ uint4 eng_philox10(uint4 c, uint32_t k0, uint32_t k1) { return philox4x32_10(c, k0, k1); }

__device__ __forceinline__ int ewrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

template <typename T>
__device__ __forceinline__ T ld_cg(const T* p) {
  return __ldcg(p);
}

// Position of x in a shared v row: the even x first, then the odd x, so that
// the sites of a colour class (x modulus 2) are consecutive words.
__device__ __forceinline__ int xpos(int i, int half) { return (i & 1) ? half + (i >> 1) : (i >> 1); }

// q = (kr * ny + j) * nx + i  ->  i, j, kr (shifts when nx, ny are powers of two).
template <typename T>
__device__ __forceinline__ void split_xy(const EngLevel<T>& L, int q, int* i, int* j, int* kr) {
  int r;
  if (L.lx >= 0) {
    *i = q & (L.nx - 1);
    r = q >> L.lx;
  } else {
    *i = q % L.nx;
    r = q / L.nx;
  }
  if (L.ly >= 0) {
    *j = r & (L.ny - 1);
    *kr = r >> L.ly;
  } else {
    *j = r % L.ny;
    *kr = r / L.ny;
  }
}

// Per-CTA view of one level.
template <typename T>
struct View {
  const EngLevel<T>* L;
  int z0, z1;          // owned planes [z0, z1)
  T* v;                // local v buffer: planes [z0-2, z1+2), pitches L->rp, L->pp
  int plane;           // nx * ny (sites per plane in the natural field order)
  const T* tab;        // shared: [nz][12] = z bands (10), 1/A_ii, 1/sqrt(A_ii)
  const EngColour* col;  // shared: colour classes of this level for this CTA
  __device__ __forceinline__ int loc(int i, int j, int k) const {
    return (k - z0 + 2) * L->pp + j * L->rp + xpos(i, L->half);
  }
};

template <typename T>
__device__ __forceinline__ View<T> make_view(const EngLevel<T>& L, unsigned char* smem, int rank, bool cluster) {
  View<T> w;
  w.L = &L;
  if (cluster) {
    w.z0 = min(rank * L.P, L.nz);
    w.z1 = min(w.z0 + L.P, L.nz);
  } else {
    w.z0 = 0;
    w.z1 = L.nz;
  }
  w.v = (T*)(smem + L.sv);
  w.plane = L.nx * L.ny;
  w.tab = nullptr;
  w.col = nullptr;
  return w;
}

// Row of A applied to v in the separable form: for each z offset, two 3x3
// partial sums with the level's x/y weights, combined with the row's z bands.
// centre == false excludes the diagonal term (sum_{j != i} A_ij v_j).
template <typename T, bool CENTRE>
__device__ __forceinline__ T stencil_row(const View<T>& w, int i, int j, int k) {
  const EngLevel<T>& L = *w.L;
  const int nx = L.nx, ny = L.ny, rp = L.rp;
  const int xm = xpos(i == 0 ? nx - 1 : i - 1, L.half), xp = xpos(i == nx - 1 ? 0 : i + 1, L.half);
  const int x0 = xpos(i, L.half);
  const T* zb = w.tab + k * 12;
  // Planes beyond a wall have zero band weights: their loads are clamped to
  // a valid plane (inside the slab and its halo) and multiplied by 0, so the
  // loads of all planes issue without a branch between them.
  T acc = (T)0;
#pragma unroll
  for (int dz = -2; dz <= 2; ++dz) {
    const int kk = min(max(k + dz, 0), L.nz - 1);
    const T* vp = w.v + (kk - w.z0 + 2) * L.pp;
    T p1, p2;
    if (ny == 1) {
      const T a = vp[xm], c = vp[xp];
      p1 = L.w1[3] * a + L.w1[5] * c;
      p2 = L.w2[3] * a + L.w2[5] * c;
      if (CENTRE || dz != 0) {
        const T b = vp[x0];
        p1 += L.w1[4] * b;
        p2 += L.w2[4] * b;
      }
    } else {
      const int jm = j == 0 ? ny - 1 : j - 1, jp = j == ny - 1 ? 0 : j + 1;
      const T* r0 = vp + jm * rp;
      const T* r1 = vp + j * rp;
      const T* r2 = vp + jp * rp;
      const T a0 = r0[xm], b0 = r0[x0], c0 = r0[xp];
      const T a1 = r1[xm], c1 = r1[xp];
      const T a2 = r2[xm], b2 = r2[x0], c2 = r2[xp];
      p1 = L.w1[0] * a0 + L.w1[1] * b0 + L.w1[2] * c0 + L.w1[3] * a1 + L.w1[5] * c1 + L.w1[6] * a2 +
           L.w1[7] * b2 + L.w1[8] * c2;
      p2 = L.w2[0] * a0 + L.w2[1] * b0 + L.w2[2] * c0 + L.w2[3] * a1 + L.w2[5] * c1 + L.w2[6] * a2 +
           L.w2[7] * b2 + L.w2[8] * c2;
      if (CENTRE || dz != 0) {
        const T b1 = r1[x0];
        p1 += L.w1[4] * b1;
        p2 += L.w2[4] * b1;
      }
    }
    acc += zb[dz + 2] * p1 + zb[5 + dz + 2] * p2;
  }
  return acc;
}

// q = n / d for 0 <= n < 2^24: float reciprocal estimate, then exact correction.
__device__ __forceinline__ int fdiv(int n, int d, float inv) {
  int q = (int)((float)n * inv);
  if (q * d > n) --q;
  if ((q + 1) * d <= n) ++q;
  return q;
}

struct Sync {
  bool cluster;
  __device__ __forceinline__ void operator()() const {
    if (cluster)
      cg::this_cluster().sync();
    else
      __syncthreads();
  }
};

// One colour pass of the stochastic Gauss-Seidel sweep on the owned planes:
// one thread per site; the four sites of a noise group each recompute the
// group's Philox block (cheaper than serialising their updates).  Class
// geometry, z bands, inverse diagonals and noise scales come from the
// shared-memory tables staged for the level.
template <typename T, bool NOISE>
__device__ void colour_pass(const View<T>& w, int level, int q, int sweep, const T* b, bool b_local, int boff, Key key,
                            unsigned long long cyc, int rank, int csize, bool cluster) {
  const EngLevel<T>& L = *w.L;
  const EngColour cc = w.col[q];
  if (cc.nsite <= 0) return;
  const uint32_t c1 = (uint32_t)level | ((uint32_t)L.comp_id << 4) | ((uint32_t)q << 8) | ((uint32_t)sweep << 12);
  cg::cluster_group cl = cg::this_cluster();
  for (int s = threadIdx.x; s < cc.nsite; s += blockDim.x) {
    const int rk = cc.rank_lo + s;
    int t, ii, kk, jj;
    if (cc.sx >= 0) {
      t = rk >> cc.sx;
      ii = rk & (cc.nxc - 1);
    } else {
      t = fdiv(rk, cc.nxc, cc.inv_nxc);
      ii = rk - t * cc.nxc;
    }
    if (cc.sy >= 0) {
      kk = t >> cc.sy;
      jj = t & (cc.nyc - 1);
    } else {
      kk = fdiv(t, cc.nyc, cc.inv_nyc);
      jj = t - kk * cc.nyc;
    }
    const int i = cc.cx + L.mx * ii, j = cc.cy + L.my * jj, k = cc.cz + L.mz * kk;
    const int gidx = (k * L.ny + j) * L.nx + i;
    const T bb = b_local ? b[gidx - boff] : ld_cg(b + gidx);
    const T* tr = w.tab + k * 12;
    const T off = stencil_row<T, false>(w, i, j, k);
    T nv = (bb - off) * tr[10];
    if (NOISE) {
      T nn;
      normal_of(eng_philox10(make_uint4((uint32_t)(rk >> 2), c1, (uint32_t)cyc, (uint32_t)(cyc >> 32)), key.k0,
                             key.k1),
                rk & 3, &nn);
      nv += nn * tr[11];
    }
    w.v[w.loc(i, j, k)] = nv;
    if (cluster && csize > 1) {
      // push into the halos of the CTAs owning planes within distance 2
      const int rlo = max(0, (k - 2) / L.P), rhi = min(csize - 1, (k + 2) / L.P);
      for (int r2 = rlo; r2 <= rhi; ++r2) {
        if (r2 == rank) continue;
        const int z0b = min(r2 * L.P, L.nz), z1b = min(z0b + L.P, L.nz);
        if (z0b >= z1b || k < z0b - 2 || k >= z1b + 2) continue;
        T* rem = cl.map_shared_rank(w.v, r2);
        rem[(k - z0b + 2) * L.pp + j * L.rp + xpos(i, L.half)] = nv;
      }
    }
  }
}

template <typename T>
__device__ void zero_local(const View<T>& w) {
  const int n = (w.z1 - w.z0 + 4) * w.L->pp;
  for (int q = threadIdx.x; q < n; q += blockDim.x) w.v[q] = (T)0;
}

// t = b - A v on the owned planes; t written at field index (global or local buffer).
template <typename T>
__device__ void residual(const View<T>& w, const T* b, bool b_local, int boff, T* t) {
  const EngLevel<T>& L = *w.L;
  const int n = (w.z1 - w.z0) * w.plane;
  // two sites per iteration, both computed before either is stored, so that
  // their loads overlap
  auto value = [&](int q, int* gidx) {
    int i, j, k;
    split_xy(L, q, &i, &j, &k);
    k += w.z0;
    *gidx = (k * L.ny + j) * L.nx + i;
    const T bb = b_local ? b[*gidx - boff] : ld_cg(b + *gidx);
    return bb - stencil_row<T, true>(w, i, j, k);
  };
  for (int q = threadIdx.x; q < n; q += 2 * blockDim.x) {
    const int q2 = q + blockDim.x;
    int g1 = 0, g2 = 0;
    const T r1 = value(q, &g1);
    const T r2 = q2 < n ? value(q2, &g2) : (T)0;
    t[g1] = r1;
    if (q2 < n) t[g2] = r2;
  }
}

// b_c = P^T t on the coarse planes [Z0, Z1) of level Lc (tables on the fine level Lf).
template <typename T>
__device__ void restrict_to(const EngLevel<T>& Lf, const EngLevel<T>& Lc, const T* t, bool t_local, T* bc, int Z0,
                            int Z1) {
  const int n = (Z1 - Z0) * Lc.nx * Lc.ny;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    int I, J, K;
    split_xy(Lc, q, &I, &J, &K);
    K += Z0;
    T acc = (T)0;
#pragma unroll
    for (int qz = 0; qz < 4; ++qz) {
      // an unused tap (index -1) reads row 0 with weight 0: no branch between taps
      const int kr = Lf.rz_idx[K * 4 + qz];
      const int kf = kr < 0 ? 0 : kr;
      const T wz = kr < 0 ? (T)0 : Lf.rz_w[K * 4 + qz];
      for (int qy = -1; qy <= 1; ++qy) {
        T wy;
        int jf;
        if (Lf.ny == 1) {
          if (qy != 0) continue;
          wy = (T)1;
          jf = 0;
        } else {
          wy = qy == 0 ? (T)1 : (T)0.5;
          jf = ewrap(2 * J + qy, Lf.ny);
        }
#pragma unroll
        for (int qx = -1; qx <= 1; ++qx) {
          const T wx = qx == 0 ? (T)1 : (T)0.5;
          const int idx = (kf * Lf.ny + jf) * Lf.nx + ewrap(2 * I + qx, Lf.nx);
          acc += wz * wy * wx * (t_local ? t[idx] : ld_cg(t + idx));
        }
      }
    }
    bc[(K * Lc.ny + J) * Lc.nx + I] = acc;
  }
}

// v_f += P v_c on the local planes [z0-2, z1+2) of the fine view (halo included).
template <typename T>
__device__ void prolong_into(const View<T>& w, const EngLevel<T>& Lc, const T* vc, bool vc_local, int vc_z0) {
  const EngLevel<T>& L = *w.L;
  const int p0 = max(0, w.z0 - 2), p1 = min(L.nz, w.z1 + 2);
  const int n = (p1 - p0) * w.plane;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    int i, j, k;
    split_xy(L, q, &i, &j, &k);
    k += p0;
    int xi0 = i >> 1, xi1 = xi0;
    T xw0 = (T)1, xw1 = (T)0;
    if (i & 1) {
      xi1 = ewrap(xi0 + 1, Lc.nx);
      xw0 = xw1 = (T)0.5;
    }
    int yi0 = 0, yi1 = 0;
    T yw0 = (T)1, yw1 = (T)0;
    if (L.ny > 1) {
      yi0 = yi1 = j >> 1;
      if (j & 1) {
        yi1 = ewrap(yi0 + 1, Lc.ny);
        yw0 = yw1 = (T)0.5;
      }
    }
    T acc = (T)0;
#pragma unroll
    for (int qz = 0; qz < 2; ++qz) {
      const int kr = L.pz_idx[k * 2 + qz];
      const int kc = kr < 0 ? 0 : kr;
      const T wz = kr < 0 ? (T)0 : L.pz_w[k * 2 + qz];
      const int yi[2] = {yi0, yi1}, xi[2] = {xi0, xi1};
      const T yw[2] = {yw0, yw1}, xw[2] = {xw0, xw1};
      for (int a = 0; a < 2; ++a) {
        if (yw[a] == (T)0) continue;
        for (int c = 0; c < 2; ++c) {
          if (xw[c] == (T)0) continue;
          const int idx = vc_local ? ((kc - vc_z0 + 2) * Lc.pp + yi[a] * Lc.rp + xpos(xi[c], Lc.half))
                                   : ((kc * Lc.ny + yi[a]) * Lc.nx + xi[c]);
          acc += wz * yw[a] * xw[c] * (vc_local ? vc[idx] : ld_cg(vc + idx));
        }
      }
    }
    w.v[w.loc(i, j, k)] += acc;
  }
}

template <typename T>
__device__ void store_owned(const View<T>& w, T* g) {
  const EngLevel<T>& L = *w.L;
  const int n = (w.z1 - w.z0) * w.plane;
  const int base = w.z0 * w.plane;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    int i, j, k;
    split_xy(L, q, &i, &j, &k);
    g[base + q] = w.v[w.loc(i, j, w.z0 + k)];
  }
}

// Copies b of the owned planes [z0, z1) (natural order) into shared memory.
template <typename T>
__device__ void load_owned(const View<T>& w, const T* g, T* dst) {
  const int n = (w.z1 - w.z0) * w.plane;
  const T* src = g + w.z0 * w.plane;
  for (int q = threadIdx.x; q < n; q += blockDim.x) dst[q] = ld_cg(src + q);
}

template <typename T>
__device__ void load_all(const View<T>& w, const T* g, T* dst) {
  const int n = (w.z1 - w.z0) * w.plane;
  for (int q = threadIdx.x; q < n; q += blockDim.x) dst[q] = ld_cg(g + q);
}

// Exact coarsest step in CTA 0: v = L^-T (L^-1 b + noise n), FP64.  Each
// row of L^-1 b and each column of L^-T y is a dot product split over eight
// consecutive lanes and reduced with shuffles.
template <typename T, bool NOISE>
__device__ void coarsest_step(const View<T>& w, int level, const T* b, double* y, Key key, unsigned long long cyc) {
  const EngLevel<T>& L = *w.L;
  const int N = L.nx * L.ny * L.nz;
  constexpr int G = 8;
  const int span = (N * G + 31) / 32 * 32;   // whole warps: every lane reaches the shuffles
  for (int t = threadIdx.x; t < span; t += blockDim.x) {
    const int r = t / G, g = t % G;
    double acc = 0.0;
    if (r < N)
      for (int q = g; q <= r; q += G) acc += __ldg(L.Linv + (long long)r * N + q) * (double)b[q];
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    if (r < N && g == 0) {
      if (NOISE) {
        const uint32_t c1 = (uint32_t)level | ((uint32_t)L.comp_id << 4) | (1u << 20);
        double nn;
        normal_of(eng_philox10(make_uint4((uint32_t)(r >> 2), c1, (uint32_t)cyc, (uint32_t)(cyc >> 32)), key.k0,
                               key.k1),
                  r & 3, &nn);
        acc += nn;
      }
      y[r] = acc;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < span; t += blockDim.x) {
    const int col = t / G, g = t % G;
    double acc = 0.0;
    if (col < N)
      for (int r = col + g; r < N; r += G) acc += __ldg(L.Linv + (long long)r * N + col) * y[r];
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    if (col < N && g == 0) {
      const int i = col % L.nx, rr = col / L.nx;
      w.v[w.loc(i, rr % L.ny, rr / L.ny)] = (T)acc;
    }
  }
}

template <typename T, bool NOISE>
__device__ void sweeps(const View<T>& w, int level, int first_sweep, int count, const T* b, bool b_local, int boff, Key key,
                       unsigned long long cyc, int rank, int csize, bool cluster) {
  const Sync sync{cluster};
  for (int s = 0; s < count; ++s)
    for (int q = 0; q < w.L->ncol; ++q) {
      colour_pass<T, NOISE>(w, level, q, first_sweep + s, b, b_local, boff, key, cyc, rank, csize, cluster);
      sync();
    }
}

// Fills the colour-class table of the staged level L as seen by the CTA
// owning planes [z0, z1): per class the geometry and the owned rank range.
// (No barrier: the caller syncs.)
template <typename T>
__device__ void stage_colours(const EngLevel<T>& L, int z0, int z1, EngColour* col) {
  for (int q = threadIdx.x; q < L.ncol; q += blockDim.x) {
    EngColour c;
    c.cx = q % L.mx;
    c.cy = (q / L.mx) % L.my;
    c.cz = q / (L.mx * L.my);
    c.nxc = (L.nx - c.cx + L.mx - 1) / L.mx;
    c.nyc = (L.ny - c.cy + L.my - 1) / L.my;
    const int nzc = (L.nz - c.cz + L.mz - 1) / L.mz;
    c.inv_nxc = 1.0f / (float)max(c.nxc, 1);
    c.inv_nyc = 1.0f / (float)max(c.nyc, 1);
    c.sx = (c.nxc > 0 && (c.nxc & (c.nxc - 1)) == 0) ? __ffs(c.nxc) - 1 : -1;
    c.sy = (c.nyc > 0 && (c.nyc & (c.nyc - 1)) == 0) ? __ffs(c.nyc) - 1 : -1;
    int kk_lo = z0 <= c.cz ? 0 : (z0 - c.cz + L.mz - 1) / L.mz;
    int kk_hi = z1 <= c.cz ? 0 : (z1 - c.cz + L.mz - 1) / L.mz;
    kk_hi = min(kk_hi, nzc);
    const int pr = c.nxc * c.nyc;
    c.rank_lo = kk_lo * pr;
    c.nsite = (c.nxc > 0 && c.nyc > 0 && nzc > 0 && kk_hi > kk_lo) ? (kk_hi - kk_lo) * pr : 0;
    col[q] = c;
  }
}

template <typename T, bool NOISE>
__global__ void __launch_bounds__(EngThreads<T>::value, 1) k_coarse_engine(const EngParams<T>* __restrict__ P, EngRun run) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cl = cg::this_cluster();
  const int csize = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int comp = blockIdx.x / csize;
  const EngComp<T>* E = &P->comp[comp];
  const unsigned long long cyc = *run.cyc;
  const int lt = P->l0, lc = P->L - 1;
  const int mu1 = run.mu1, mu2 = run.mu2;
  const Key key = run.key;
  EngLevel<T>* const lev0 = reinterpret_cast<EngLevel<T>*>(smem + P->lev_off);   // levels lt..lc
  EngColour* const col0 = reinterpret_cast<EngColour*>(smem + P->col_off);
  T* const stab = reinterpret_cast<T*>(smem + P->tab_off);
  auto sl_at = [&](int l) -> EngLevel<T>& { return lev0[l - lt]; };
  auto col_at = [&](int l) { return col0 + (size_t)(l - lt) * kEngMaxColours; };

  // ---- stage every level once: descriptors, then colour classes and row tables ----
  {
    constexpr int n = (int)(sizeof(EngLevel<T>) / sizeof(int));
    const int total = (lc - lt + 1) * n;
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
      const int l = lt + q / n, e = q - (q / n) * n;
      reinterpret_cast<int*>(&sl_at(l))[e] = reinterpret_cast<const int*>(&E->lev[l])[e];
    }
    __syncthreads();
    for (int l = lt; l <= lc; ++l) {
      const EngLevel<T>& L = sl_at(l);
      const View<T> w = make_view(L, smem, rank, L.cluster != 0);
      stage_colours(L, w.z0, w.z1, col_at(l));
    }
    // Row tables (per row k of each level: the z bands, 1/A_ii, 1/sqrt(A_ii))
    // and transfer tables (prolongation and restriction taps along z) of all
    // levels as one list of entries.  Each thread issues the global loads of
    // up to kStageUnroll entries before it stores any of them, so the list
    // costs about one memory latency instead of one per level and table.
    {
      // entries of level l: 12 nz row-table words, then (below the coarsest
      // level) 2 nz prolongation taps and 4 nz_c restriction taps
      auto level_entries = [&](int l) {
        const EngLevel<T>& L = sl_at(l);
        return 12 * L.nz + (l < lc ? 2 * L.nz + 4 * sl_at(l + 1).nz : 0);
      };
      int total = 0;
      for (int l = lt; l <= lc; ++l) total += level_entries(l);
      constexpr int kStageUnroll = 4;
      for (int base = threadIdx.x; base < total; base += kStageUnroll * blockDim.x) {
        T val[kStageUnroll];
        int ival[kStageUnroll], kind[kStageUnroll], lev[kStageUnroll], pos[kStageUnroll];
#pragma unroll
        for (int u = 0; u < kStageUnroll; ++u) {
          int q = base + u * (int)blockDim.x;
          kind[u] = -1;
          if (q >= total) continue;
          int l = lt;
          while (q >= level_entries(l)) {
            q -= level_entries(l);
            ++l;
          }
          const EngLevel<T>& L = sl_at(l);
          lev[u] = l;
          pos[u] = q;
          if (q < 12 * L.nz) {   // row table: band, or the diagonal (inverted below)
            const int k = q / 12, e = q - k * 12;
            kind[u] = e < 10 ? 0 : e == 10 ? 1 : 2;
            val[u] = e < 10 ? L.zb[k * 10 + e] : L.S[(long long)k * kStencil + 22];
          } else {   // transfer tap, at its slot of the level's transfer rows
            const int t = q - 12 * L.nz;
            kind[u] = 3;
            pos[u] = t;
            if (t < 2 * L.nz) {
              ival[u] = L.pz_idx[t];
              val[u] = L.pz_w[t];
            } else {
              ival[u] = L.rz_idx[t - 2 * L.nz];
              val[u] = L.rz_w[t - 2 * L.nz];
            }
          }
        }
#pragma unroll
        for (int u = 0; u < kStageUnroll; ++u) {
          if (kind[u] < 0) continue;
          const int l = lev[u];
          if (kind[u] < 3) {
            const T v = val[u];
            stab[(size_t)P->tab_row[l] * 12 + pos[u]] =
                kind[u] == 0 ? v : kind[u] == 1 ? (T)1 / v : (T)1 / tsqrt(v);
          } else {
            reinterpret_cast<int*>(smem + P->xfi_off)[P->xf_row[l] + pos[u]] = ival[u];
            reinterpret_cast<T*>(smem + P->xfw_off)[P->xf_row[l] + pos[u]] = val[u];
          }
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0)
      for (int l = lt; l < lc; ++l) {
        EngLevel<T>& L = sl_at(l);
        int* xi = reinterpret_cast<int*>(smem + P->xfi_off) + P->xf_row[l];
        T* xw = reinterpret_cast<T*>(smem + P->xfw_off) + P->xf_row[l];
        L.pz_idx = xi;
        L.pz_w = xw;
        L.rz_idx = xi + 2 * L.nz;
        L.rz_w = xw + 2 * L.nz;
      }
    __syncthreads();
  }
  auto view_of = [&](int l, bool cluster) {
    View<T> w = make_view(sl_at(l), smem, rank, cluster);
    w.tab = stab + (size_t)P->tab_row[l] * 12;
    w.col = col_at(l);
    return w;
  };

  // ---- down leg over the cluster levels ----
  int l = lt;
  for (; l < lc && sl_at(l).cluster; ++l) {
    const EngLevel<T>& L = sl_at(l);
    const EngLevel<T>& Lc = sl_at(l + 1);
    View<T> w = view_of(l, true);
    zero_local(w);
    // b of the owned planes in shared memory when the plan has room for it
    const bool bl = L.sb >= 0;
    const T* bsrc = bl ? (const T*)(smem + L.sb) : L.gb;
    const int boff = bl ? w.z0 * w.plane : 0;
    if (bl) load_owned(w, L.gb, (T*)(smem + L.sb));
    cl.sync();
    sweeps<T, NOISE>(w, l, 0, mu1, bsrc, bl, boff, key, cyc, rank, csize, true);
    residual(w, bsrc, bl, boff, L.gt);
    cl.sync();
    // the coarse planes of the restriction are split over the cluster's CTAs
    // (also when the coarse level is held by CTA 0: it reads them back)
    const int Pc = (Lc.nz + csize - 1) / csize;
    const int Z0 = min(rank * Pc, Lc.nz);
    const int Z1 = min(Z0 + Pc, Lc.nz);
    // into the first level held by CTA 0: its shared b, through distributed shared memory
    T* bdst = Lc.cluster ? Lc.gb : cl.map_shared_rank(reinterpret_cast<T*>(smem + Lc.sb), 0);
    restrict_to(L, Lc, L.gt, false, bdst, Z0, Z1);
    cl.sync();
  }
  const int lsingle = l;   // first level held by CTA 0 alone
  if (rank == 0) {
    // ---- single-CTA part: levels lsingle .. lc and back ----
    if (lsingle == lt) {   // b from global only when no cluster level restricted into it
      View<T> w = view_of(lsingle, false);
      load_all(w, sl_at(lsingle).gb, (T*)(smem + sl_at(lsingle).sb));
    }
    for (int k = lsingle; k <= lc; ++k) {
      const EngLevel<T>& L = sl_at(k);
      View<T> w = view_of(k, false);
      T* b = (T*)(smem + L.sb);
      zero_local(w);
      __syncthreads();
      if (k == lc && run.coarse_mode == SELM_COARSE_CHOLESKY) {
        coarsest_step<T, NOISE>(w, k, b, (double*)(smem + P->y_off), key, cyc);
        __syncthreads();
        break;
      }
      sweeps<T, NOISE>(w, k, 0, mu1, b, true, 0, key, cyc, 0, 1, false);
      if (k == lc) {
        sweeps<T, NOISE>(w, k, mu1, mu2, b, true, 0, key, cyc, 0, 1, false);
        break;
      }
      const EngLevel<T>& Lc = sl_at(k + 1);
      residual(w, b, true, 0, (T*)(smem + L.st));
      __syncthreads();
      restrict_to(L, Lc, (const T*)(smem + L.st), true, (T*)(smem + Lc.sb), 0, Lc.nz);
      __syncthreads();
    }
    for (int k = lc - 1; k >= lsingle; --k) {
      const EngLevel<T>& L = sl_at(k);
      const EngLevel<T>& Lc = sl_at(k + 1);
      View<T> w = view_of(k, false);
      prolong_into(w, Lc, (const T*)(smem + Lc.sv), true, 0);
      __syncthreads();
      sweeps<T, NOISE>(w, k, mu1, mu2, (const T*)(smem + L.sb), true, 0, key, cyc, 0, 1, false);
    }
    {   // the engine's result, or the hand-off to the cluster's prolongation
      View<T> w = view_of(lsingle, false);
      store_owned(w, sl_at(lsingle).gv);
    }
  }
  cl.sync();
  // ---- up leg over the cluster levels ----
  for (int k = lsingle - 1; k >= lt; --k) {
    const EngLevel<T>& L = sl_at(k);
    const EngLevel<T>& Lc = sl_at(k + 1);
    View<T> w = view_of(k, true);
    if (Lc.cluster) {
      prolong_into(w, Lc, Lc.gv, false, 0);
    } else {
      // the coarse level is held by CTA 0, which still has its v in shared
      // memory; the other CTAs first copy it (independent loads) into their own
      // unused slab of that level, then prolong from shared memory
      View<T> wc = view_of(k + 1, false);
      if (rank != 0) {
        const int nc = Lc.nx * Lc.ny * Lc.nz;
#pragma unroll 4
        for (int q = threadIdx.x; q < nc; q += blockDim.x) {
          int i, j, kk;
          split_xy(Lc, q, &i, &j, &kk);
          wc.v[wc.loc(i, j, kk)] = ld_cg(Lc.gv + q);
        }
        __syncthreads();
      }
      prolong_into(w, Lc, (const T*)wc.v, true, 0);
    }
    cl.sync();
    const bool bl = L.sb >= 0;   // staged on the way down, untouched since
    sweeps<T, NOISE>(w, k, mu1, mu2, bl ? (const T*)(smem + L.sb) : L.gb, bl, bl ? w.z0 * w.plane : 0, key, cyc, rank,
                     csize, true);
    store_owned(w, L.gv);
    cl.sync();
  }
}

template <typename T>
size_t level_bytes_cluster(const LevelDev& L, int c, int C) {
  const CompDev& d = L.c[c];
  const int P = (d.nz + C - 1) / C;
  return (size_t)(P + 4) * d.nx * d.ny * sizeof(T);
}

inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Pitches of a level's shared v slab.  A warp of a colour pass holds
// consecutive ranks of the class: x runs fastest (nx/2 sites of one parity,
// consecutive words within a row), then y in steps of 2, then z in steps of
// mz.  The row pitch rp is padded so that the rows one warp spans start on
// distinct banks (2 rp = sites per row, modulo 32 words), and the plane
// pitch pp likewise for the planes one warp spans (mz pp = sites per plane,
// modulo 32), when a warp spans more than one row or plane.
void slab_pitches(int nx, int ny, int mz, int* half, int* rp, int* pp) {
  const int h = (nx + 1) / 2;
  *half = h;
  int r = nx;
  if (ny > 1 && h < 32) {
    const int want = (((h + 1) & ~1) % 32) / 2;   // rp == want (mod 16)
    r = nx + (((want - nx) % 16) + 16) % 16;
  }
  *rp = r;
  int p = r * ny;
  const int per_plane = h * (ny > 1 ? (ny + 1) / 2 : 1);
  if (per_plane < 32 && mz > 0) {
    for (int c = p; c < p + 32; ++c)
      if ((long long)mz * c % 32 == per_plane % 32) {
        p = c;
        break;
      }
  }
  *pp = p;
}

template <typename T>
bool try_plan(const LevelDev* levs, int L, int l0, int C, bool stage_b, size_t smem_cap, EnginePlanT<T>* out) {
  // cluster levels first (largest), then single levels
  const int ncomp = levs[0].ncomp;
  size_t need_max = 0;
  EngParams<T>& p = out->params;
  p.l0 = l0;
  p.L = L;
  p.ncomp = ncomp;
  bool any_cluster = false;
  for (int c = 0; c < ncomp; ++c) {
    size_t off = 0;
    bool single_started = false;
    for (int l = l0; l < L; ++l) {
      const CompDev& d = levs[l].c[c];
      EngLevel<T>& e = p.comp[c].lev[l];
      const long long sites = (long long)d.nx * d.ny * d.nz;
      if (sites >= (1ll << 24)) return false;   // rank decode uses float reciprocals
      const bool single = single_started || l == L - 1 || sites <= kEngSingleMaxSites || C == 1;
      if (single) single_started = true;
      e.cluster = single ? 0 : 1;
      if (e.cluster) any_cluster = true;
      e.P = single ? d.nz : (d.nz + C - 1) / C;
      slab_pitches(d.nx, d.ny, d.mz, &e.half, &e.rp, &e.pp);
      const size_t vbytes = (size_t)(e.P + 4) * e.pp * sizeof(T);
      e.sv = (int)off;
      off = align16(off + vbytes);
      if (single) {
        e.sb = (int)off;
        off = align16(off + (size_t)sites * sizeof(T));
        e.st = (int)off;
        off = align16(off + (size_t)sites * sizeof(T));
      } else {
        e.sb = e.st = -1;
        if (stage_b) {   // b of the owned planes
          e.sb = (int)off;
          off = align16(off + (size_t)e.P * d.nx * d.ny * sizeof(T));
        }
      }
    }
    const CompDev& dc = levs[L - 1].c[c];
    const size_t Nc = (size_t)dc.nx * dc.ny * dc.nz;
    if (Nc > 1024) return false;
    out->y_off_comp[c] = off;
    off = align16(off + Nc * sizeof(double));
    need_max = need_max > off ? need_max : off;
  }
  // row tables of every level (components share the layout: the largest nz)
  int rows = 0;
  for (int l = l0; l < L; ++l) {
    p.tab_row[l] = rows;
    int nzl = 0;
    for (int c = 0; c < ncomp; ++c) nzl = nzl > levs[l].c[c].nz ? nzl : levs[l].c[c].nz;
    rows += nzl;
  }
  for (int c = 0; c < ncomp; ++c)
    for (int l = l0; l < L; ++l)
      if (levs[l].c[c].ncol > kEngMaxColours) return false;
  // transfer tables of the levels with a coarser level below them
  int xrows = 0;
  for (int l = l0; l < L; ++l) {
    p.xf_row[l] = xrows;
    if (l == L - 1) continue;
    int nzl = 0, nzc = 0;
    for (int c = 0; c < ncomp; ++c) {
      nzl = nzl > levs[l].c[c].nz ? nzl : levs[l].c[c].nz;
      nzc = nzc > levs[l + 1].c[c].nz ? nzc : levs[l + 1].c[c].nz;
    }
    xrows += 2 * nzl + 4 * nzc;
  }
  const size_t staged = (size_t)rows * 12 * sizeof(T) + (size_t)(L - l0) * sizeof(EngLevel<T>) +
                        (size_t)(L - l0) * kEngMaxColours * sizeof(EngColour) +
                        (size_t)xrows * (sizeof(int) + sizeof(T)) + 96;
  if (need_max + staged > smem_cap) return false;
  if (!any_cluster) C = 1;
  // every component gets the same y offset (the maximum) so that the kernel
  // can use one field
  size_t yo = 0;
  for (int c = 0; c < ncomp; ++c) yo = yo > out->y_off_comp[c] ? yo : out->y_off_comp[c];
  p.y_off = (int)yo;
  size_t ymax = 0;
  for (int c = 0; c < ncomp; ++c) {
    const CompDev& dc = levs[L - 1].c[c];
    const size_t Nc = (size_t)dc.nx * dc.ny * dc.nz;
    ymax = ymax > Nc ? ymax : Nc;
  }
  const size_t tab_off = align16(yo + ymax * sizeof(double));
  const size_t lev_off = align16(tab_off + (size_t)rows * 12 * sizeof(T));
  const size_t col_off = align16(lev_off + (size_t)(L - l0) * sizeof(EngLevel<T>));
  const size_t xfi_off = align16(col_off + (size_t)(L - l0) * kEngMaxColours * sizeof(EngColour));
  const size_t xfw_off = align16(xfi_off + (size_t)xrows * sizeof(int));
  p.tab_off = (int)tab_off;
  p.lev_off = (int)lev_off;
  p.col_off = (int)col_off;
  p.xfi_off = (int)xfi_off;
  p.xfw_off = (int)xfw_off;
  out->smem_bytes = align16(xfw_off + (size_t)xrows * sizeof(T));
  if (out->smem_bytes > smem_cap) return false;
  out->cluster = C;
  return true;
}

}  // namespace

template <typename T>
void fill_engine_tables(const LevelDev* levs, int L, void* const* gb, void* const* gv, void* const* gt,
                        EnginePlanT<T>* plan) {
  EngParams<T>& p = plan->params;
  for (int c = 0; c < p.ncomp; ++c)
    for (int l = p.l0; l < L; ++l) {
      const CompDev& d = levs[l].c[c];
      EngLevel<T>& e = p.comp[c].lev[l];
      e.nx = d.nx;
      e.ny = d.ny;
      e.nz = d.nz;
      e.mx = d.mx;
      e.my = d.my;
      e.mz = d.mz;
      e.ncol = d.ncol;
      e.comp_id = d.comp_id;
      e.S = sizeof(T) == 4 ? (const T*)d.S32 : (const T*)d.S64;
      e.zb = sizeof(T) == 4 ? (const T*)d.zb32 : (const T*)d.zb64;
      for (int q = 0; q < 9; ++q) {
        e.w1[q] = (T)d.w1[q];
        e.w2[q] = (T)d.w2[q];
      }
      auto log2_or = [](int n) {
        int l = 0;
        while ((1 << l) < n) ++l;
        return (1 << l) == n ? l : -1;
      };
      e.lx = log2_or(d.nx);
      e.ly = log2_or(d.ny);
      e.inv_nxc = 1.0f / (float)((d.nx + d.mx - 1) / d.mx);
      e.inv_nyc = 1.0f / (float)((d.ny + d.my - 1) / d.my);
      e.rz_idx = d.rz_idx;
      e.rz_w = sizeof(T) == 4 ? (const T*)d.rz_w32 : (const T*)d.rz_w64;
      e.pz_idx = d.pz_idx;
      e.pz_w = sizeof(T) == 4 ? (const T*)d.pz_w32 : (const T*)d.pz_w64;
      e.Linv = d.Linv;
      e.gb = (T*)gb[l] + d.off;
      e.gv = (T*)gv[l] + d.off;
      e.gt = (T*)gt[l] + d.off;
    }
}

namespace {
template <typename T>
bool raise_smem_limit() {
  static std::atomic<bool> done{false};
  if (done.load()) return true;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  for (auto fn : {k_coarse_engine<T, true>, k_coarse_engine<T, false>}) {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess ||
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes) !=
            cudaSuccess ||
        cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
  }
  done.store(true);
  return true;
}
}  // namespace

template <typename T>
bool plan_coarse_engine(const LevelDev* levs, int L, void* const* gb, void* const* gv, void* const* gt,
                        void* dev_params, cudaStream_t st, EnginePlanT<T>* plan, int want_cluster,
                        int min_level) {
  static_assert(sizeof(EngParams<T>) <= kEngParamBytes, "engine plan exceeds its workspace slot");
  plan->valid = false;
  if (L < 2 || !dev_params) return false;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  int cap = 0, cluster_ok = 0;
  cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&cluster_ok, cudaDevAttrClusterLaunch, dev);
  const size_t smem_cap = (size_t)cap > 2048 ? (size_t)cap - 1024 : 0;
  const int sizes[5] = {16, 8, 4, 2, 1};
  for (int l0 = min_level > 1 ? min_level : 1; l0 < L; ++l0) {
    for (int si = 0; si < 5; ++si) {
      const int C = sizes[si];
      if (C > 1 && !cluster_ok) continue;
      if (want_cluster > 0 && C > want_cluster) continue;
      EnginePlanT<T> cand{};
      // with b of the cluster levels staged in shared memory if it fits
      if (!try_plan<T>(levs, L, l0, C, true, smem_cap, &cand) &&
          !try_plan<T>(levs, L, l0, C, false, smem_cap, &cand))
        continue;
      // The dynamic shared-memory limit is a per-kernel setting shared by every
      // handle of the process: raise it once to the device maximum so that
      // plans of any size stay launchable.
      if (!raise_smem_limit<T>()) continue;
      if (cand.cluster > 1) {
        auto fn = k_coarse_engine<T, true>;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(cand.cluster * levs[0].ncomp);
        cfg.blockDim = dim3(EngThreads<T>::value);
        cfg.dynamicSmemBytes = cand.smem_bytes;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cand.cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) != cudaSuccess || nclusters < 1) {
          cudaGetLastError();
          continue;
        }
      }
      *plan = cand;
      fill_engine_tables<T>(levs, L, gb, gv, gt, plan);
      if (cudaMemcpyAsync(dev_params, &plan->params, sizeof(EngParams<T>), cudaMemcpyHostToDevice, st) !=
              cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return false;
      }
      plan->dev = (const EngParams<T>*)dev_params;
      plan->valid = true;
      return true;
    }
  }
  return false;
}

template <typename T>
cudaError_t launch_coarse_engine(const EnginePlanT<T>& plan, int mu1, int mu2, int coarse_mode, bool noise, Key key,
                                 const unsigned long long* cyc, cudaStream_t st) {
  EngRun run{mu1, mu2, coarse_mode, key, cyc};
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(plan.cluster * plan.params.ncomp);
  cfg.blockDim = dim3(EngThreads<T>::value);
  cfg.dynamicSmemBytes = plan.smem_bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = plan.cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  prof::Scope ps(SELM_K_COARSE_SWEEP, st);
  if (noise) return cudaLaunchKernelEx(&cfg, k_coarse_engine<T, true>, plan.dev, run);
  return cudaLaunchKernelEx(&cfg, k_coarse_engine<T, false>, plan.dev, run);
}

template bool plan_coarse_engine<float>(const LevelDev*, int, void* const*, void* const*, void* const*, void*,
                                        cudaStream_t, EnginePlanT<float>*, int, int);
template bool plan_coarse_engine<double>(const LevelDev*, int, void* const*, void* const*, void* const*, void*,
                                         cudaStream_t, EnginePlanT<double>*, int, int);
template cudaError_t launch_coarse_engine<float>(const EnginePlanT<float>&, int, int, int, bool, Key,
                                                 const unsigned long long*, cudaStream_t);
template cudaError_t launch_coarse_engine<double>(const EnginePlanT<double>&, int, int, int, bool, Key,
                                                  const unsigned long long*, cudaStream_t);

}  // namespace selm
