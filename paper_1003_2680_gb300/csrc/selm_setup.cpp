// Host setup of the multigrid hierarchy (FP64).
//
// Section 3.2: prolongation I_{l-1}^l is tri-linear interpolation, restriction
// is its transpose (Eq. equ_restr_prolong_variation) and the level operators
// are the variational (Galerkin) products A^(l) = I^T A I.  Because every
// operator here is a Kronecker sum of 1-D factors and the prolongation is a
// tensor product, the Galerkin product is done per axis on 1-D factors:
//   K_d <- P_d^T K_d P_d   (stiffness),   M_d <- P_d^T M_d P_d   (mass),
//   A^(l) = s * sum_d K_d (x) prod_{e != d} M_e.
// Periodic axes keep translation-invariant 3-point stencils; the wall axis
// keeps per-row bands of half-width <= 2.  The full 3x3x5 stencil of every
// row of the wall axis is tabulated for the kernels.

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "selm_internal.h"

namespace selm {
namespace {

int lattice_size(int kind, int n) {
  if (kind == kAxisTrivial) return 1;
  if (kind == kAxisVertex) return n - 1;
  return n;
}

// Top-level 1-D second difference of a wall axis as band rows [m][5].
std::vector<double> wall_stiffness(int kind, int n) {
  int m = lattice_size(kind, n);
  std::vector<double> K((size_t)m * 5, 0.0);
  for (int k = 0; k < m; ++k) {
    double* r = &K[(size_t)k * 5];
    r[2] = 2.0;
    if (k > 0) r[1] = -1.0;
    if (k < m - 1) r[3] = -1.0;
    bool edge = (k == 0) || (k == m - 1);
    if (edge && kind == kAxisCellDir) r[2] += (m == 1 ? 2.0 : 1.0);   // ghost = -u
    if (edge && kind == kAxisCellNeu) r[2] -= (m == 1 ? 2.0 : 1.0);   // ghost = +u
  }
  return K;
}

std::vector<double> wall_identity(int kind, int n) {
  int m = lattice_size(kind, n);
  std::vector<double> M((size_t)m * 5, 0.0);
  for (int k = 0; k < m; ++k) M[(size_t)k * 5 + 2] = 1.0;
  return M;
}

struct Entry {
  int fine, coarse;
  double w;
};

// Linear interpolation along a wall axis from nc cells to 2 nc cells.
// Vertex lattice: coarse node J+1 sits on fine node 2J+2; odd fine nodes take
// the mean of their neighbours, the wall nodes being 0.  Cell lattices: fine
// cells 2J and 2J+1 take 3/4 of coarse cell J and 1/4 of the neighbour on
// their side; beyond a wall that neighbour is the odd (Dirichlet) or even
// (Neumann) reflection of cell J.
std::vector<Entry> wall_prolongation(int kind, int nc) {
  std::vector<Entry> P;
  int nf = 2 * nc;
  if (kind == kAxisVertex) {
    for (int k = 0; k < nf - 1; ++k) {
      int node = k + 1;
      if (node % 2 == 0) {
        P.push_back({k, node / 2 - 1, 1.0});
      } else {
        int a = (node - 1) / 2, b = (node + 1) / 2;
        if (a >= 1 && a <= nc - 1) P.push_back({k, a - 1, 0.5});
        if (b >= 1 && b <= nc - 1) P.push_back({k, b - 1, 0.5});
      }
    }
    return P;
  }
  double ghost = (kind == kAxisCellDir) ? -1.0 : 1.0;
  for (int J = 0; J < nc; ++J) {
    for (int side = 0; side < 2; ++side) {
      int f = 2 * J + side;
      int far = side == 0 ? J - 1 : J + 1;
      double wJ = 0.75;
      if (far >= 0 && far < nc) {
        P.push_back({f, far, 0.25});
      } else {
        wJ += 0.25 * ghost;
      }
      if (wJ != 0.0) P.push_back({f, J, wJ});
    }
  }
  return P;
}

// Galerkin product of a band matrix: Bc = P^T B P (rows [mc][5]).
std::vector<double> galerkin_band(const std::vector<double>& B, int mf, const std::vector<Entry>& P,
                                  int mc, std::string* err) {
  std::vector<std::vector<Entry>> col(mc), row(mf);
  for (const auto& e : P) {
    col[e.coarse].push_back(e);
    row[e.fine].push_back(e);
  }
  std::vector<double> Bc((size_t)mc * 5, 0.0);
  for (int I = 0; I < mc; ++I) {
    for (const auto& e1 : col[I]) {
      for (int o1 = -2; o1 <= 2; ++o1) {
        int f2 = e1.fine + o1;
        if (f2 < 0 || f2 >= mf) continue;
        double kv = B[(size_t)e1.fine * 5 + o1 + 2];
        if (kv == 0.0) continue;
        for (const auto& e2 : row[f2]) {
          int o = e2.coarse - I;
          if (o < -2 || o > 2) {
            *err = "Galerkin band wider than 2";
            return Bc;
          }
          Bc[(size_t)I * 5 + o + 2] += e1.w * kv * e2.w;
        }
      }
    }
  }
  return Bc;
}

// Galerkin product of a periodic 3-point stencil with the interpolation
// stencil p = (1/2, 1, 1/2) (coarse node J on fine node 2J):
//   Sc[o] = sum_{a,b} p[a] p[b] S[2o + b - a].
void galerkin_periodic(const double S[3], double Sc[3]) {
  const double p[3] = {0.5, 1.0, 0.5};
  for (int o = -1; o <= 1; ++o) {
    double acc = 0.0;
    for (int a = -1; a <= 1; ++a)
      for (int b = -1; b <= 1; ++b) {
        int off = 2 * o + b - a;
        if (off >= -1 && off <= 1) acc += p[a + 1] * p[b + 1] * S[off + 1];
      }
    Sc[o + 1] = acc;
  }
}

int band_width(const std::vector<double>& K, const std::vector<double>& M, int m) {
  int bw = 0;
  for (int k = 0; k < m; ++k)
    for (int o = -2; o <= 2; ++o)
      if (K[(size_t)k * 5 + o + 2] != 0.0 || M[(size_t)k * 5 + o + 2] != 0.0) bw = std::max(bw, std::abs(o));
  return bw;
}

void fill_stencil(HostComp* c, double s) {
  int nz = c->dims[2];
  c->S.assign((size_t)nz * kStencil, 0.0);
  for (int k = 0; k < nz; ++k)
    for (int cz = -2; cz <= 2; ++cz)
      for (int cy = -1; cy <= 1; ++cy)
        for (int cx = -1; cx <= 1; ++cx) {
          double kz = c->Kz[(size_t)k * 5 + cz + 2], mz = c->Mz[(size_t)k * 5 + cz + 2];
          double v = c->Kx[cx + 1] * c->My[cy + 1] * mz + c->Mx[cx + 1] * c->Ky[cy + 1] * mz +
                     c->Mx[cx + 1] * c->My[cy + 1] * kz;
          c->S[(size_t)k * kStencil + ((cz + 2) * 3 + (cy + 1)) * 3 + (cx + 1)] = s * v;
        }
}

// Separable form of the same operator: per z offset cz,
//   A v = sum_cz [ s Mz[k][cz] * sum_{dy,dx} w1[dy][dx] v + s Kz[k][cz] * sum_{dy,dx} w2[dy][dx] v ]
// with w1 = Kx (x) My + Mx (x) Ky and w2 = Mx (x) My.
void fill_separable(HostComp* c, double s) {
  int nz = c->dims[2];
  c->zb.assign((size_t)nz * 10, 0.0);
  for (int k = 0; k < nz; ++k)
    for (int q = 0; q < 5; ++q) {
      c->zb[(size_t)k * 10 + q] = s * c->Mz[(size_t)k * 5 + q];
      c->zb[(size_t)k * 10 + 5 + q] = s * c->Kz[(size_t)k * 5 + q];
    }
  for (int dy = 0; dy < 3; ++dy)
    for (int dx = 0; dx < 3; ++dx) {
      c->w1[dy * 3 + dx] = c->Kx[dx] * c->My[dy] + c->Mx[dx] * c->Ky[dy];
      c->w2[dy * 3 + dx] = c->Mx[dx] * c->My[dy];
    }
}

void fill_moduli(HostComp* c) {
  c->mods[0] = c->dims[0] == 1 ? 1 : c->bw[0] + 1;
  c->mods[1] = c->dims[1] == 1 ? 1 : c->bw[1] + 1;
  c->mods[2] = c->dims[2] == 1 ? 1 : c->bw[2] + 1;
}

// Dense coarsest operator from the stencil table (periodic images summed),
// optional regularisation of the pure-Neumann null space, Cholesky A = L L^T
// and the inverse of L.
std::string coarsest_factor(HostComp* c, bool singular) {
  int nx = c->dims[0], ny = c->dims[1], nz = c->dims[2];
  int N = nx * ny * nz;
  if (N > 1024) return "coarsest level too large for the dense factor (> 1024 unknowns)";
  std::vector<double> A((size_t)N * N, 0.0);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int r = (k * ny + j) * nx + i;
        for (int cz = -2; cz <= 2; ++cz) {
          int kk = k + cz;
          if (kk < 0 || kk >= nz) continue;
          for (int cy = -1; cy <= 1; ++cy)
            for (int cx = -1; cx <= 1; ++cx) {
              double v = c->S[(size_t)k * kStencil + ((cz + 2) * 3 + (cy + 1)) * 3 + (cx + 1)];
              if (v == 0.0) continue;
              int jj = ((j + cy) % ny + ny) % ny, ii = ((i + cx) % nx + nx) % nx;
              A[(size_t)r * N + (kk * ny + jj) * nx + ii] += v;
            }
        }
      }
  if (singular) {
    double tr = 0.0;
    for (int r = 0; r < N; ++r) tr += A[(size_t)r * N + r];
    double add = (tr / N) / N;
    for (size_t q = 0; q < (size_t)N * N; ++q) A[q] += add;
  }
  std::vector<double> L((size_t)N * N, 0.0);
  for (int j = 0; j < N; ++j) {
    double d = A[(size_t)j * N + j];
    for (int p = 0; p < j; ++p) d -= L[(size_t)j * N + p] * L[(size_t)j * N + p];
    if (!(d > 0.0)) return "coarsest operator is not positive definite";
    double ljj = std::sqrt(d);
    L[(size_t)j * N + j] = ljj;
    for (int i = j + 1; i < N; ++i) {
      double v = A[(size_t)i * N + j];
      for (int p = 0; p < j; ++p) v -= L[(size_t)i * N + p] * L[(size_t)j * N + p];
      L[(size_t)i * N + j] = v / ljj;
    }
  }
  // Linv = L^-1 by forward substitution on the columns of I
  c->Linv.assign((size_t)N * N, 0.0);
  for (int col = 0; col < N; ++col) {
    for (int i = col; i < N; ++i) {
      double v = (i == col) ? 1.0 : 0.0;
      for (int p = col; p < i; ++p) v -= L[(size_t)i * N + p] * c->Linv[(size_t)p * N + col];
      c->Linv[(size_t)i * N + col] = v / L[(size_t)i * N + i];
    }
  }
  return "";
}

// Kz0 / Mz0 (optional, rows [m][5]) replace the wall kind's second difference
// and unit mass on the top level (the composite base grid's Galerkin factors).
std::string build_system(int dim, int n, int levels, double scale, const std::vector<int>& zkinds,
                         const std::vector<int>& ids, bool singular, HostSystem* out,
                         const std::vector<double>* Kz0 = nullptr, const std::vector<double>* Mz0 = nullptr) {
  if (dim != 2 && dim != 3) return "dim must be 2 or 3";
  if (n < 2) return "n must be at least 2";
  if (levels < 1 || levels > kMaxLevels) return "levels out of range";
  if (n % (1 << (levels - 1)) != 0) return "n must be divisible by 2^(levels-1)";
  out->dim = dim;
  out->n = n;
  out->levels = levels;
  out->ncomp = (int)zkinds.size();
  out->scale = scale;
  out->singular = singular;
  for (int l = 0; l < kMaxLevels; ++l) out->lev[l].clear();
  for (int ci = 0; ci < out->ncomp; ++ci) {
    HostComp c{};
    c.kind[0] = kAxisPeriodic;
    c.kind[1] = dim == 3 ? kAxisPeriodic : kAxisTrivial;
    c.kind[2] = zkinds[ci];
    c.comp_id = ids[ci];
    int ncell = n;
    // level 0 factors
    const double Kp[3] = {-1.0, 2.0, -1.0}, Mp[3] = {0.0, 1.0, 0.0}, Z3[3] = {0.0, 0.0, 0.0};
    std::memcpy(c.Kx, Kp, sizeof Kp);
    std::memcpy(c.Mx, Mp, sizeof Mp);
    if (dim == 3) {
      std::memcpy(c.Ky, Kp, sizeof Kp);
    } else {
      std::memcpy(c.Ky, Z3, sizeof Z3);
    }
    std::memcpy(c.My, Mp, sizeof Mp);
    c.Kz = Kz0 ? *Kz0 : wall_stiffness(c.kind[2], ncell);
    c.Mz = Mz0 ? *Mz0 : wall_identity(c.kind[2], ncell);
    if ((int)c.Kz.size() != lattice_size(c.kind[2], ncell) * 5 || (int)c.Mz.size() != lattice_size(c.kind[2], ncell) * 5)
      return "top-level z bands have the wrong size";
    for (int l = 0; l < levels; ++l) {
      c.dims[0] = ncell;
      c.dims[1] = dim == 3 ? ncell : 1;
      c.dims[2] = lattice_size(c.kind[2], ncell);
      if (c.dims[2] < 1) return "wall axis has no unknowns at some level";
      c.bw[0] = (c.dims[0] > 1 && (c.Kx[0] != 0.0 || c.Mx[0] != 0.0)) ? 1 : 0;
      c.bw[1] = (c.dims[1] > 1 && (c.Ky[0] != 0.0 || c.My[0] != 0.0)) ? 1 : 0;
      c.bw[2] = band_width(c.Kz, c.Mz, c.dims[2]);
      fill_moduli(&c);
      fill_stencil(&c, scale);
      fill_separable(&c, scale);
      c.rz_idx.clear();
      c.rz_w.clear();
      c.pz_idx.clear();
      c.pz_w.clear();
      c.Linv.clear();
      HostComp cur = c;
      if (l < levels - 1) {
        int nc = ncell / 2;
        int mf = c.dims[2], mc = lattice_size(c.kind[2], nc);
        if (mc < 1) return "too many levels for the wall axis";
        std::vector<Entry> P = wall_prolongation(c.kind[2], nc);
        // transfer tables
        cur.rz_idx.assign((size_t)mc * 4, -1);
        cur.rz_w.assign((size_t)mc * 4, 0.0);
        cur.pz_idx.assign((size_t)mf * 2, -1);
        cur.pz_w.assign((size_t)mf * 2, 0.0);
        std::vector<int> ccount(mc, 0), fcount(mf, 0);
        for (const auto& e : P) {
          if (ccount[e.coarse] >= 4 || fcount[e.fine] >= 2) return "transfer table overflow";
          cur.rz_idx[(size_t)e.coarse * 4 + ccount[e.coarse]] = e.fine;
          cur.rz_w[(size_t)e.coarse * 4 + ccount[e.coarse]++] = e.w;
          cur.pz_idx[(size_t)e.fine * 2 + fcount[e.fine]] = e.coarse;
          cur.pz_w[(size_t)e.fine * 2 + fcount[e.fine]++] = e.w;
        }
        // Galerkin factors of the next level
        std::string err;
        std::vector<double> Kz = galerkin_band(c.Kz, mf, P, mc, &err);
        std::vector<double> Mz = galerkin_band(c.Mz, mf, P, mc, &err);
        if (!err.empty()) return err;
        double t[3];
        galerkin_periodic(c.Kx, t);
        std::memcpy(c.Kx, t, sizeof t);
        galerkin_periodic(c.Mx, t);
        std::memcpy(c.Mx, t, sizeof t);
        if (dim == 3) {
          galerkin_periodic(c.Ky, t);
          std::memcpy(c.Ky, t, sizeof t);
          galerkin_periodic(c.My, t);
          std::memcpy(c.My, t, sizeof t);
        }
        c.Kz = Kz;
        c.Mz = Mz;
        ncell = nc;
      } else {
        std::string err = coarsest_factor(&cur, singular);
        if (!err.empty()) return err;
      }
      out->lev[l].push_back(cur);
    }
  }
  // colourings must be valid on every smoothed periodic axis
  for (int l = 0; l < levels; ++l)
    for (const auto& c : out->lev[l]) {
      if (l == 0 && c.dims[0] % 2 != 0) return "x extent must be even for red-black ordering";
      for (int a = 0; a < 2; ++a)
        if (c.dims[a] > 1 && c.dims[a] % c.mods[a] != 0 && l < levels - 1)
          return "periodic extent not a multiple of the colour modulus";
    }
  return "";
}

}  // namespace

// The dataflow order of the cooperative passes waits on a neighbour only when
// its update can be ordered against the site's: the neighbours a pass tests
// (window planes with a band entry of the row, x-y positions with a weight,
// in FP32, the centre excluded) must be coupled to the site (non-zero stencil
// entry), of another colour class, inside the walls, and must test the site
// in turn.  Any exception leaves the level to the barrier form.
bool coop_flow_ok(const HostComp& c) {
  const int nz = c.dims[2];
  if (c.S.size() != (size_t)nz * kStencil || c.zb.size() != (size_t)nz * 10) return false;
  if (c.dims[0] % 2 != 0) return false;   // periodic x colouring needs an even extent
  for (int a = 0; a < 3; ++a)
    if (c.mods[a] < 1 || (a < 2 && c.dims[a] > 1 && c.dims[a] % c.mods[a] != 0)) return false;
  auto plane = [&](int k, int dz) {
    return (float)c.zb[(size_t)k * 10 + dz + 2] != 0.f || (float)c.zb[(size_t)k * 10 + 5 + dz + 2] != 0.f;
  };
  auto xy = [&](int q) { return (float)c.w1[q] != 0.f || (float)c.w2[q] != 0.f; };
  auto mod = [](int d, int m) { return ((d % m) + m) % m; };
  for (int k = 0; k < nz; ++k)
    for (int dz = -2; dz <= 2; ++dz) {
      if (!plane(k, dz)) continue;
      if (k + dz < 0 || k + dz >= nz) return false;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int q = (dy + 1) * 3 + dx + 1;
          if ((dz == 0 && q == 4) || (c.dims[1] == 1 && dy != 0) || !xy(q)) continue;
          if (c.S[(size_t)k * kStencil + (dz + 2) * 9 + q] == 0.0) return false;
          if (mod(dx, c.mods[0]) == 0 && mod(dy, c.mods[1]) == 0 && mod(dz, c.mods[2]) == 0) return false;
          if (!plane(k + dz, -dz) || !xy(8 - q)) return false;
        }
    }
  return true;
}

int default_levels(int n) {
  int levels = 1, m = n;
  while (m % 2 == 0 && m / 2 >= 4) {
    m /= 2;
    ++levels;
  }
  return levels;
}

std::string build_velocity_system(int dim, int n, int levels, double mu, HostSystem* out) {
  double h = 1.0 / n;
  double scale = mu * std::pow(h, dim - 2);
  if (dim == 3)
    return build_system(dim, n, levels, scale, {kAxisCellDir, kAxisCellDir, kAxisVertex}, {0, 1, 2},
                        false, out);
  return build_system(dim, n, levels, scale, {kAxisCellDir, kAxisVertex}, {0, 2}, false, out);
}

std::string build_pressure_system(int dim, int n, int levels, HostSystem* out) {
  return build_system(dim, n, levels, 1.0, {kAxisCellNeu}, {3}, true, out);
}

// Composite grid (Section 4, Algorithms 1-2): base channel with wall centres
// on the walls (vertex-type z, n-1 unknown rows) and its rows j = 1..K refined
// by 2 over the whole x-y extent.  With the parent-copy prolongation, the
// Galerkin base operator P^T A P is the 7-point operator with z-dependent
// weights (unit mu H^(d-2)): z faces 4/3 at the bottom wall and across the
// interface, 2 between covered rows, 1 elsewhere; x-y mass 2 on covered rows.
// Level 0 of the result describes the patch (no tables), levels 1.. are the
// base grid and its Galerkin coarsenings.
std::string build_composite_system(int dim, int n, int K, int levels_base, double mu, int ncomp, HostSystem* out) {
  if (dim != 2 && dim != 3) return "dim must be 2 or 3";
  if (n < 4 || n % 2 != 0) return "n must be even and at least 4";
  if (K < 1 || K > n - 2) return "patch rows K must satisfy 1 <= K <= n-2";
  if (ncomp < 1 || ncomp > kMaxComps) return "ncomp out of range";
  if (levels_base < 1 || levels_base + 1 > kMaxLevels) return "levels out of range";
  const double H = 1.0 / n;
  const double scale = mu * std::pow(H, dim - 2);
  std::vector<double> wz(n, 1.0);   // face f between wall-axis node f and f+1
  wz[0] = 4.0 / 3.0;
  for (int f = 1; f < K; ++f) wz[f] = 2.0;
  wz[K] = 4.0 / 3.0;
  const int m = n - 1;
  std::vector<double> Kz((size_t)m * 5, 0.0), Mz((size_t)m * 5, 0.0);
  for (int r = 0; r < m; ++r) {
    double* k = &Kz[(size_t)r * 5];
    k[2] = wz[r] + wz[r + 1];
    if (r > 0) k[1] = -wz[r];
    if (r < m - 1) k[3] = -wz[r + 1];
    Mz[(size_t)r * 5 + 2] = r < K ? 2.0 : 1.0;
  }
  HostSystem base;
  std::vector<int> kinds(ncomp, kAxisVertex), ids(ncomp);
  for (int c = 0; c < ncomp; ++c) ids[c] = c;
  std::string err = build_system(dim, n, levels_base, scale, kinds, ids, false, &base, &Kz, &Mz);
  if (!err.empty()) return err;
  out->dim = dim;
  out->n = n;
  out->levels = levels_base + 1;
  out->ncomp = ncomp;
  out->scale = scale;
  out->singular = false;
  for (int l = 0; l < kMaxLevels; ++l) out->lev[l].clear();
  for (int c = 0; c < ncomp; ++c) {
    HostComp p{};
    p.kind[0] = kAxisPeriodic;
    p.kind[1] = dim == 3 ? kAxisPeriodic : kAxisTrivial;
    p.kind[2] = kAxisVertex;
    p.dims[0] = 2 * n;
    p.dims[1] = dim == 3 ? 2 * n : 1;
    p.dims[2] = 2 * K;
    p.comp_id = c;
    p.mods[0] = p.mods[1] = p.mods[2] = 2;
    p.S.assign((size_t)p.dims[2] * kStencil, 0.0);
    p.zb.assign((size_t)p.dims[2] * 10, 0.0);
    out->lev[0].push_back(p);
  }
  for (int l = 0; l < levels_base; ++l) out->lev[l + 1] = base.lev[l];
  return "";
}

}  // namespace selm
