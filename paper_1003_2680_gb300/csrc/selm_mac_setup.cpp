// Host setup of the staggered composite grid (FP64): face numbering, the
// composite velocity operator, divergence, gradient, pressure operator, FAC
// base hierarchy with Galerkin operators and colour classes, the coarsest
// factor, and the extension to the uniform fine lattice for the particles.
//
// Face numbering (the composite vector's order):
//   1. for each fine cell (m, q, p) in (z, y, x) order: its low x face, then
//      (3-D) its low y face;
//   2. the same for the base cells of rows K..n-1;
//   3. z faces between fine layers, m = 1..2K-1, (m, q, p) order;
//   4. (0 < K < n) the interface faces, one per base cell of row K;
//   5. z faces between base rows, j = K+1..n-1.
// Cells: the fine cells (m, q, p), then the base cells (j - K, l, i).

#include <algorithm>
#include <cmath>
#include <cstring>
#include <utility>

#include "selm_internal.h"
#include "selm_mac.h"

namespace selm {
namespace mac {
namespace {

enum Lev : int { kFine = 0, kBase = 1, kIface = 2 };

struct FaceKey {
  int axis, lev, k, j, i;
};

struct Trip {
  int r, c;
  double v;
};

int wrap(int a, int m) { return ((a % m) + m) % m; }

// CSR from triplets: duplicates summed, columns ascending, exact zeros kept
// out.
Csr from_triplets(int nr, int nc, std::vector<Trip>& t) {
  Csr out;
  out.nr = nr;
  out.nc = nc;
  std::vector<long long> cnt(nr + 1, 0);
  for (const Trip& e : t) ++cnt[e.r + 1];
  for (int r = 0; r < nr; ++r) cnt[r + 1] += cnt[r];
  std::vector<std::pair<int, double>> tmp(t.size());
  std::vector<long long> pos(cnt.begin(), cnt.end() - 1);
  for (const Trip& e : t) tmp[pos[e.r]++] = {e.c, e.v};
  out.ptr.assign(nr + 1, 0);
  for (int r = 0; r < nr; ++r) {
    auto b = tmp.begin() + cnt[r], e = tmp.begin() + cnt[r + 1];
    std::sort(b, e, [](const std::pair<int, double>& x, const std::pair<int, double>& y) { return x.first < y.first; });
    for (auto it = b; it != e;) {
      int c = it->first;
      double s = 0.0;
      for (; it != e && it->first == c; ++it) s += it->second;
      if (s != 0.0) {
        out.col.push_back(c);
        out.val.push_back(s);
      }
    }
    out.ptr[r + 1] = (long long)out.col.size();
  }
  return out;
}

Csr transpose(const Csr& a) {
  Csr t;
  t.nr = a.nc;
  t.nc = a.nr;
  t.ptr.assign(a.nc + 1, 0);
  for (int c : a.col) ++t.ptr[c + 1];
  for (int r = 0; r < a.nc; ++r) t.ptr[r + 1] += t.ptr[r];
  t.col.resize(a.col.size());
  t.val.resize(a.val.size());
  std::vector<long long> pos(t.ptr.begin(), t.ptr.end() - 1);
  for (int r = 0; r < a.nr; ++r)
    for (long long q = a.ptr[r]; q < a.ptr[r + 1]; ++q) {
      long long p = pos[a.col[q]]++;
      t.col[p] = r;
      t.val[p] = a.val[q];
    }
  return t;
}

// C = A B, row by row with a dense accumulator over B's columns.
Csr multiply(const Csr& a, const Csr& b) {
  Csr c;
  c.nr = a.nr;
  c.nc = b.nc;
  c.ptr.assign(a.nr + 1, 0);
  std::vector<double> acc(b.nc, 0.0);
  std::vector<char> seen(b.nc, 0);
  std::vector<int> touched;
  for (int r = 0; r < a.nr; ++r) {
    touched.clear();
    for (long long q = a.ptr[r]; q < a.ptr[r + 1]; ++q) {
      const int k = a.col[q];
      const double av = a.val[q];
      for (long long s = b.ptr[k]; s < b.ptr[k + 1]; ++s) {
        const int j = b.col[s];
        if (!seen[j]) {
          seen[j] = 1;
          touched.push_back(j);
        }
        acc[j] += av * b.val[s];
      }
    }
    std::sort(touched.begin(), touched.end());
    for (int j : touched) {
      if (acc[j] != 0.0) {
        c.col.push_back(j);
        c.val.push_back(acc[j]);
      }
      acc[j] = 0.0;
      seen[j] = 0;
    }
    c.ptr[r + 1] = (long long)c.col.size();
  }
  return c;
}

double diag_of(const Csr& a, int r) {
  for (long long q = a.ptr[r]; q < a.ptr[r + 1]; ++q)
    if (a.col[q] == r) return a.val[q];
  return 0.0;
}

// First-fit colouring in index order of the rows `rows` of `a` (the graph of
// the principal submatrix on those rows): a row takes the smallest class not
// used by an earlier row it couples to.  Returns the classes as row lists
// (ascending).
std::vector<std::vector<int>> first_fit(const Csr& a, const std::vector<int>& rows) {
  std::vector<int> colour(a.nr, -2);            // -2: not in the set
  for (int r : rows) colour[r] = -1;
  std::vector<std::vector<int>> classes;
  std::vector<char> used;
  for (int r : rows) {
    const double dr = std::fabs(diag_of(a, r));
    used.assign(classes.size() + 1, 0);
    for (long long q = a.ptr[r]; q < a.ptr[r + 1]; ++q) {
      const int c = a.col[q];
      if (c == r || colour[c] < 0) continue;
      if (std::fabs(a.val[q]) <= kGraphRtol * dr) continue;
      used[colour[c]] = 1;
    }
    int k = 0;
    while (used[k]) ++k;
    colour[r] = k;
    if (k == (int)classes.size()) classes.emplace_back();
    classes[k].push_back(r);
  }
  return classes;
}

// ---- 1-D lattices of the MAC grid and their linear interpolation ----------
enum Kind1 : int { kP = 0, kV = 1, kC = 2, kO = 3 };

int size1(int kind, int cells) { return kind == kO ? 1 : (kind == kV ? cells - 1 : cells); }

// Interpolation from a lattice of nc cells to one of 2 nc cells: rows of the
// fine lattice, each a list of (coarse unknown, weight).  Periodic: coarse
// node J on fine node 2J, odd fine nodes the mean of their neighbours.
// Wall-normal (vertex) lattice: the same on the interior nodes, wall nodes 0.
// Cell lattice between no-slip walls: fine cells 2J, 2J+1 take 3/4 of coarse
// cell J and 1/4 of the neighbour on their side, the neighbour beyond a wall
// being minus cell J.
std::vector<std::vector<std::pair<int, double>>> interp1(int kind, int nc) {
  std::vector<std::vector<std::pair<int, double>>> rows;
  if (kind == kO) {
    rows.push_back({{0, 1.0}});
    return rows;
  }
  const int mf = size1(kind, 2 * nc);
  rows.resize(mf);
  if (kind == kP) {
    for (int J = 0; J < nc; ++J) {
      rows[2 * J].push_back({J, 1.0});
      rows[2 * J + 1].push_back({J, 0.5});
      rows[2 * J + 1].push_back({(J + 1) % nc, 0.5});
    }
  } else if (kind == kV) {
    for (int k = 0; k < mf; ++k) {
      const int node = k + 1;                  // fine node index (walls at 0 and 2 nc)
      if (node % 2 == 0) {
        rows[k].push_back({node / 2 - 1, 1.0});
      } else {
        for (int cn : {(node - 1) / 2, (node + 1) / 2})
          if (cn >= 1 && cn <= nc - 1) rows[k].push_back({cn - 1, 0.5});
      }
    }
  } else {
    for (int J = 0; J < nc; ++J) {
      for (int side = 0; side < 2; ++side) {
        const int f = 2 * J + side, far = side ? J + 1 : J - 1;
        if (far >= 0 && far < nc) {
          rows[f].push_back({J, 0.75});
          rows[f].push_back({far, 0.25});
        } else {
          rows[f].push_back({J, 0.5});
        }
      }
    }
  }
  for (auto& r : rows) std::sort(r.begin(), r.end());
  return rows;
}

// Component layout of the uniform MAC velocity lattice of `cells` cells per
// axis: kinds (x, y, z) and dims.
struct CompLat {
  int kind[3];
  int dims[3];     // nx, ny, nz
};

std::vector<CompLat> velocity_lattice(int dim, int cells) {
  std::vector<CompLat> out;
  const int yk = dim == 3 ? kP : kO;
  const int ncomp = dim == 3 ? 3 : 2;
  for (int c = 0; c < ncomp; ++c) {
    const bool normal = c == ncomp - 1;
    CompLat L;
    L.kind[0] = kP;
    L.kind[1] = yk;
    L.kind[2] = normal ? kV : kC;
    for (int a = 0; a < 3; ++a) L.dims[a] = size1(L.kind[a], a == 1 && dim == 2 ? 1 : cells);
    out.push_back(L);
  }
  return out;
}

std::vector<long long> lattice_offsets(const std::vector<CompLat>& lat) {
  std::vector<long long> off(lat.size() + 1, 0);
  for (size_t c = 0; c < lat.size(); ++c)
    off[c + 1] = off[c] + (long long)lat[c].dims[0] * lat[c].dims[1] * lat[c].dims[2];
  return off;
}

// Tensor-product interpolation of every component from `cells` to 2 `cells`
// per axis (rows: the fine lattice, block diagonal by component).
Csr lattice_interp(int dim, int cells) {
  const auto fl = velocity_lattice(dim, 2 * cells), cl = velocity_lattice(dim, cells);
  const auto fo = lattice_offsets(fl), co = lattice_offsets(cl);
  std::vector<Trip> t;
  for (size_t c = 0; c < fl.size(); ++c) {
    std::vector<std::vector<std::pair<int, double>>> p1[3];
    for (int a = 0; a < 3; ++a) p1[a] = interp1(fl[c].kind[a], a == 1 && dim == 2 ? 1 : cells);
    const int fx = fl[c].dims[0], fy = fl[c].dims[1], fz = fl[c].dims[2];
    const int cx = cl[c].dims[0], cy = cl[c].dims[1];
    for (int k = 0; k < fz; ++k)
      for (int j = 0; j < fy; ++j)
        for (int i = 0; i < fx; ++i) {
          const long long row = fo[c] + ((long long)k * fy + j) * fx + i;
          for (auto& ez : p1[2][k])
            for (auto& ey : p1[1][j])
              for (auto& ex : p1[0][i])
                t.push_back({(int)row, (int)(co[c] + ((long long)ez.first * cy + ey.first) * cx + ex.first),
                             ez.second * ey.second * ex.second});
        }
  }
  return from_triplets((int)fo.back(), (int)co.back(), t);
}

// ---- face numbering -------------------------------------------------------
struct Numbering {
  int d, n, K;
  int fnz, fny, fnx, bnz, bny, bnx, nper;
  long long o_xyb, o_zf, o_zi, o_zb, total;
  int n_fine_cells, n_cells;

  Numbering(int d_, int n_, int K_) : d(d_), n(n_), K(K_) {
    fnz = 2 * K;
    fny = d == 3 ? 2 * n : 1;
    fnx = 2 * n;
    bnz = n - K;
    bny = d == 3 ? n : 1;
    bnx = n;
    nper = d == 3 ? 2 : 1;
    n_fine_cells = fnz * fny * fnx;
    n_cells = n_fine_cells + bnz * bny * bnx;
    o_xyb = (long long)n_fine_cells * nper;
    o_zf = o_xyb + (long long)bnz * bny * bnx * nper;
    o_zi = o_zf + (long long)std::max(fnz - 1, 0) * fny * fnx;
    o_zb = o_zi + ((K > 0 && K < n) ? (long long)bny * bnx : 0);
    total = o_zb + (long long)std::max(n - K - 1, 0) * bny * bnx;
  }
  int fine_cell(int m, int q, int p) const { return (m * fny + wrap(q, fny)) * fnx + wrap(p, fnx); }
  int base_cell(int j, int l, int i) const {
    return n_fine_cells + ((j - K) * bny + wrap(l, bny)) * bnx + wrap(i, bnx);
  }
  // face of a key; -1 if the key names no unknown
  int face(int axis, int lev, int k, int j, int i) const {
    if (axis < 2) {
      if (lev == kFine) return (int)(((long long)(k * fny + wrap(j, fny)) * fnx + wrap(i, fnx)) * nper + axis);
      return (int)(o_xyb + ((long long)((k - K) * bny + wrap(j, bny)) * bnx + wrap(i, bnx)) * nper + axis);
    }
    if (lev == kFine) return (int)(o_zf + ((long long)(k - 1) * fny + wrap(j, fny)) * fnx + wrap(i, fnx));
    if (lev == kIface) return (int)(o_zi + (long long)wrap(j, bny) * bnx + wrap(i, bnx));
    return (int)(o_zb + ((long long)(k - K - 1) * bny + wrap(j, bny)) * bnx + wrap(i, bnx));
  }
  std::vector<FaceKey> keys() const {
    std::vector<FaceKey> out;
    out.reserve(total);
    for (int m = 0; m < fnz; ++m)
      for (int q = 0; q < fny; ++q)
        for (int p = 0; p < fnx; ++p)
          for (int a = 0; a < nper; ++a) out.push_back({a, kFine, m, q, p});
    for (int j = K; j < n; ++j)
      for (int l = 0; l < bny; ++l)
        for (int i = 0; i < bnx; ++i)
          for (int a = 0; a < nper; ++a) out.push_back({a, kBase, j, l, i});
    for (int m = 1; m < fnz; ++m)
      for (int q = 0; q < fny; ++q)
        for (int p = 0; p < fnx; ++p) out.push_back({2, kFine, m, q, p});
    if (K > 0 && K < n)
      for (int l = 0; l < bny; ++l)
        for (int i = 0; i < bnx; ++i) out.push_back({2, kIface, K, l, i});
    for (int j = K + 1; j < n; ++j)
      for (int l = 0; l < bny; ++l)
        for (int i = 0; i < bnx; ++i) out.push_back({2, kBase, j, l, i});
    return out;
  }
};

// Velocity component of a face axis (2-D: x -> 0, z -> 1).
int comp_of_axis(int d, int axis) { return d == 3 ? axis : (axis == 0 ? 0 : 1); }

}  // namespace

std::string build_plan(int dim, int n, int K, int levels, double mu, Plan* out) {
  if (dim != 2 && dim != 3) return "dim must be 2 or 3";
  if (n < 4 || n % 2) return "n must be even and >= 4";
  if (K < 0 || K > n) return "K must lie in [0, n]";
  if (levels <= 0) levels = default_levels(n);
  for (int l = 1, m = n; l < levels; ++l) {
    if (m % 2 || m / 2 < 2) return "n must be divisible by 2^(levels-1) with >= 2 cells on the coarsest level";
    m /= 2;
  }
  const Numbering N(dim, n, K);
  if (N.total > (1ll << 30) || (long long)N.n_cells > (1ll << 30)) return "grid too large";
  Plan& P = *out;
  P.dim = dim;
  P.n = n;
  P.K = K;
  P.levels = levels;
  P.mu = mu;
  P.n_faces = (int)N.total;
  P.n_cells = N.n_cells;
  P.n_fine_cells = N.n_fine_cells;
  const double H = 1.0 / n, h = 0.5 * H;
  const int d = dim;
  const auto keys = N.keys();
  if ((long long)keys.size() != N.total) return "face numbering mismatch";

  // ---- cells, faces: divergence, gradient (Eq. equ_def_discr_div, the
  // coarse-face gradient rule; reading R21) --------------------------------
  P.vol.assign(N.n_cells, std::pow(H, d));
  std::fill(P.vol.begin(), P.vol.begin() + N.n_fine_cells, std::pow(h, d));
  P.weight.assign(N.total, 0.0);
  {
    std::vector<Trip> td, tg;
    const int kids = d == 3 ? 4 : 2;
    for (int f = 0; f < (int)N.total; ++f) {
      const FaceKey& e = keys[f];
      int plus;
      std::vector<std::pair<int, double>> minus;
      double area, dist;
      if (e.lev == kFine) {
        area = std::pow(h, d - 1);
        dist = h;
        plus = N.fine_cell(e.k, e.j, e.i);
        if (e.axis == 0) minus.push_back({N.fine_cell(e.k, e.j, e.i - 1), 1.0});
        else if (e.axis == 1) minus.push_back({N.fine_cell(e.k, e.j - 1, e.i), 1.0});
        else minus.push_back({N.fine_cell(e.k - 1, e.j, e.i), 1.0});
      } else if (e.lev == kBase) {
        area = std::pow(H, d - 1);
        dist = H;
        plus = N.base_cell(e.k, e.j, e.i);
        if (e.axis == 0) minus.push_back({N.base_cell(e.k, e.j, e.i - 1), 1.0});
        else if (e.axis == 1) minus.push_back({N.base_cell(e.k, e.j - 1, e.i), 1.0});
        else minus.push_back({N.base_cell(e.k - 1, e.j, e.i), 1.0});
      } else {
        area = std::pow(H, d - 1);
        dist = 0.75 * H;
        plus = N.base_cell(K, e.j, e.i);
        for (int a = 0; a < (d == 3 ? 2 : 1); ++a)
          for (int c = 0; c < 2; ++c)
            minus.push_back({N.fine_cell(N.fnz - 1, d == 3 ? 2 * e.j + a : 0, 2 * e.i + c), 1.0 / kids});
      }
      P.weight[f] = area * dist;
      td.push_back({plus, f, -area / P.vol[plus]});
      tg.push_back({f, plus, 1.0 / dist});
      for (auto& m : minus) {
        td.push_back({m.first, f, m.second * area / P.vol[m.first]});
        tg.push_back({f, m.first, -m.second / dist});
      }
    }
    P.D = from_triplets(N.n_cells, (int)N.total, td);
    P.G = from_triplets((int)N.total, N.n_cells, tg);
    Csr DG = multiply(P.D, P.G);
    for (int r = 0; r < DG.nr; ++r)
      for (long long q = DG.ptr[r]; q < DG.ptr[r + 1]; ++q) DG.val[q] *= P.vol[r];
    P.S = DG;
  }

  // ---- velocity operator A = -mu V L (energy form; reading R22) -----------
  {
    std::vector<Trip> t;
    auto term = [&](double w, const std::vector<std::pair<int, double>>& cs) {
      for (auto& a : cs)
        for (auto& b : cs) t.push_back({a.first, b.first, mu * w * a.second * b.second});
    };
    auto pair = [&](double w, int a, int b) { term(w, {{a, 1.0}, {b, -1.0}}); };
    const double Ha = std::pow(H, d - 1);
    // tangential components: cell lattice across the walls
    for (int a = 0; a < (d == 3 ? 2 : 1); ++a) {
      for (int lev = kFine; lev <= kBase; ++lev) {
        const double s = lev == kFine ? h : H, area = std::pow(s, d - 1);
        const int k0 = lev == kFine ? 0 : K, k1 = lev == kFine ? N.fnz : n;
        const int ny = lev == kFine ? N.fny : N.bny, nx = lev == kFine ? N.fnx : N.bnx;
        for (int k = k0; k < k1; ++k)
          for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
              const int me = N.face(a, lev, k, j, i);
              // neighbour along the component's own axis, then the other periodic axis
              pair(area / s, me, a == 0 ? N.face(a, lev, k, j, i + 1) : N.face(a, lev, k, j + 1, i));
              if (d == 3) pair(area / s, me, a == 0 ? N.face(a, lev, k, j + 1, i) : N.face(a, lev, k, j, i + 1));
              if (k < k1 - 1) pair(area / s, me, N.face(a, lev, k + 1, j, i));
              if (k == 0) term(area / (0.5 * s), {{me, 1.0}});                       // wall z = 0
              if ((lev == kBase && k == n - 1) || (lev == kFine && k == N.fnz - 1 && K == n))
                term(area / (0.5 * s), {{me, 1.0}});                                 // wall z = 1
            }
      }
      if (K > 0 && K < n) {
        // coarse-fine group: the base node of row K against the fine nodes of
        // the top slab layer under its box face, (1/4, 1/2, 1/4) along the
        // component's axis times 1/2 across (3-D), distance (3/4) H
        for (int j = 0; j < N.bny; ++j)
          for (int i = 0; i < N.bnx; ++i) {
            std::vector<std::pair<int, double>> cs{{N.face(a, kBase, K, j, i), 1.0}};
            const double wt[3] = {0.25, 0.5, 0.25};
            for (int dt = -1; dt <= 1; ++dt)
              for (int e = 0; e < (d == 3 ? 2 : 1); ++e) {
                const double we = d == 3 ? 0.5 : 1.0;
                const int f = a == 0 ? N.face(0, kFine, N.fnz - 1, d == 3 ? 2 * j + e : 0, 2 * i + dt)
                                     : N.face(1, kFine, N.fnz - 1, 2 * j + dt, 2 * i + e);
                cs.push_back({f, -wt[dt + 1] * we});
              }
            term(Ha / (0.75 * H), cs);
          }
      }
    }
    // wall-normal component: vertex lattice across the walls
    struct ZNode {
      int lev, k, j, i;
      double s, height;
    };
    std::vector<ZNode> zn;
    for (int m = 1; m < N.fnz; ++m)
      for (int q = 0; q < N.fny; ++q)
        for (int p = 0; p < N.fnx; ++p) zn.push_back({kFine, m, q, p, h, h});
    if (K > 0 && K < n)
      for (int l = 0; l < N.bny; ++l)
        for (int i = 0; i < N.bnx; ++i) zn.push_back({kIface, K, l, i, H, 0.75 * H});
    for (int j = K + 1; j < n; ++j)
      for (int l = 0; l < N.bny; ++l)
        for (int i = 0; i < N.bnx; ++i) zn.push_back({kBase, j, l, i, H, H});
    for (const ZNode& z : zn) {
      const int me = N.face(2, z.lev, z.k, z.j, z.i);
      const double side = std::pow(z.s, d - 2) * z.height;   // box face normal to x or y
      pair(side / z.s, me, N.face(2, z.lev, z.k, z.j, z.i + 1));
      if (d == 3) pair(side / z.s, me, N.face(2, z.lev, z.k, z.j + 1, z.i));
      const double area = std::pow(z.s, d - 1);              // box face normal to z
      if (z.lev == kFine) {
        if (z.k + 1 < N.fnz) pair(area / h, me, N.face(2, kFine, z.k + 1, z.j, z.i));
        else if (K == n) term(area / h, {{me, 1.0}});
        if (z.k == 1) term(area / h, {{me, 1.0}});
      } else {
        const int up = z.lev == kIface ? K + 1 : z.k + 1;
        if (up <= n - 1) pair(area / H, me, N.face(2, kBase, up, z.j, z.i));
        else term(area / H, {{me, 1.0}});
        if (z.lev == kBase && z.k == 1) term(area / H, {{me, 1.0}});
      }
    }
    if (K > 0 && K < n) {
      // the interface node against the fine z nodes of the top slab layer:
      // 1/2^(d-1) each, distance h
      for (int l = 0; l < N.bny; ++l)
        for (int i = 0; i < N.bnx; ++i) {
          std::vector<std::pair<int, double>> cs{{N.face(2, kIface, K, l, i), 1.0}};
          for (int e = 0; e < (d == 3 ? 2 : 1); ++e)
            for (int tt = 0; tt < 2; ++tt)
              cs.push_back({N.face(2, kFine, N.fnz - 1, d == 3 ? 2 * l + e : 0, 2 * i + tt), -0.5 * (d == 3 ? 0.5 : 1.0)});
          term(Ha / h, cs);
        }
    }
    P.A = from_triplets((int)N.total, (int)N.total, t);
  }

  // ---- FAC base hierarchy (reading R23) --------------------------------------
  {
    const auto bl = velocity_lattice(d, n);
    const auto bo = lattice_offsets(bl);
    const auto fl = velocity_lattice(d, 2 * n);
    std::vector<Trip> t;
    std::vector<std::vector<std::pair<int, double>>> p1[3][3];   // [comp][axis]
    for (size_t c = 0; c < bl.size(); ++c)
      for (int a = 0; a < 3; ++a) p1[c][a] = interp1(bl[c].kind[a], a == 1 && d == 2 ? 1 : n);
    for (int f = 0; f < (int)N.total; ++f) {
      const FaceKey& e = keys[f];
      const int c = comp_of_axis(d, e.axis);
      const int kk = e.axis == 2 ? e.k - 1 : e.k;
      const int jj = d == 3 ? e.j : 0;
      if (e.lev != kFine) {
        t.push_back({f, (int)(bo[c] + ((long long)kk * bl[c].dims[1] + jj) * bl[c].dims[0] + e.i), 1.0});
        continue;
      }
      for (auto& ez : p1[c][2][kk])
        for (auto& ey : p1[c][1][jj])
          for (auto& ex : p1[c][0][e.i])
            t.push_back({f, (int)(bo[c] + ((long long)ez.first * bl[c].dims[1] + ey.first) * bl[c].dims[0] + ex.first),
                         ez.second * ey.second * ex.second});
    }
    (void)fl;
    P.P = from_triplets((int)N.total, (int)bo.back(), t);
    P.ops.push_back(multiply(transpose(P.P), multiply(P.A, P.P)));
    int cells = n;
    for (int l = 0; l + 1 < levels; ++l) {
      cells /= 2;
      P.Pl.push_back(lattice_interp(d, cells));
      const Csr& pl = P.Pl.back();
      P.ops.push_back(multiply(transpose(pl), multiply(P.ops.back(), pl)));
    }
    for (int l = 0; l + 1 < levels; ++l) {
      std::vector<int> rows(P.ops[l].nr);
      for (int r = 0; r < P.ops[l].nr; ++r) rows[r] = r;
      P.colours.push_back(first_fit(P.ops[l], rows));
    }
    std::vector<int> slab;
    for (int f = 0; f < (int)N.total; ++f)
      if (keys[f].lev == kFine) slab.push_back(f);
    P.patch_colours = first_fit(P.A, slab);
    // exact draw on the coarsest level: A = L L^T, Linv = L^-1
    const Csr& Ac = P.ops.back();
    const int m = Ac.nr;
    if (m > 8192) return "coarsest level too large for the dense factor";
    std::vector<double> L((size_t)m * m, 0.0);
    for (int r = 0; r < m; ++r)
      for (long long q = Ac.ptr[r]; q < Ac.ptr[r + 1]; ++q) L[(size_t)r * m + Ac.col[q]] = Ac.val[q];
    for (int j = 0; j < m; ++j) {
      double s = L[(size_t)j * m + j];
      for (int k = 0; k < j; ++k) s -= L[(size_t)j * m + k] * L[(size_t)j * m + k];
      if (!(s > 0.0)) return "coarsest operator is not positive definite";
      const double ljj = std::sqrt(s);
      L[(size_t)j * m + j] = ljj;
      for (int i = j + 1; i < m; ++i) {
        double v = L[(size_t)i * m + j];
        for (int k = 0; k < j; ++k) v -= L[(size_t)i * m + k] * L[(size_t)j * m + k];
        L[(size_t)i * m + j] = v / ljj;
      }
      for (int i = 0; i < j; ++i) L[(size_t)i * m + j] = 0.0;
    }
    P.Linv.assign((size_t)m * m, 0.0);
    for (int c = 0; c < m; ++c) {              // column c of L^-1 by forward substitution
      for (int i = c; i < m; ++i) {
        double v = i == c ? 1.0 : 0.0;
        for (int k = c; k < i; ++k) v -= L[(size_t)i * m + k] * P.Linv[(size_t)k * m + c];
        P.Linv[(size_t)i * m + c] = v / L[(size_t)i * m + i];
      }
    }
  }

  // ---- particles: extension to the uniform fine lattice (reading R24) -----
  {
    const auto bl = velocity_lattice(d, n);
    const auto bo = lattice_offsets(bl);
    const auto fl = velocity_lattice(d, 2 * n);
    const auto fo = lattice_offsets(fl);
    // R: base lattice <- composite (the unknown where a base node is one, the
    // mean of the coinciding fine faces on covered base nodes)
    std::vector<Trip> tr;
    for (size_t c = 0; c < bl.size(); ++c) {
      const int axis = (d == 3) ? (int)c : (c == 0 ? 0 : 2);
      for (int k = 0; k < bl[c].dims[2]; ++k)
        for (int j = 0; j < bl[c].dims[1]; ++j)
          for (int i = 0; i < bl[c].dims[0]; ++i) {
            const int row = (int)(bo[c] + ((long long)k * bl[c].dims[1] + j) * bl[c].dims[0] + i);
            const int kz = axis == 2 ? k + 1 : k;
            if (kz >= K) {
              const int lev = (axis == 2 && kz == K && K > 0 && K < n) ? kIface : kBase;
              tr.push_back({row, N.face(axis, lev, kz, j, i), 1.0});
              continue;
            }
            std::vector<int> kids;
            for (int e = 0; e < (d == 3 ? 2 : 1); ++e)
              for (int tt = 0; tt < 2; ++tt) {
                if (axis == 0) kids.push_back(N.face(0, kFine, 2 * kz + tt, d == 3 ? 2 * j + e : 0, 2 * i));
                else if (axis == 1) kids.push_back(N.face(1, kFine, 2 * kz + tt, 2 * j, 2 * i + e));
                else kids.push_back(N.face(2, kFine, 2 * kz, d == 3 ? 2 * j + e : 0, 2 * i + tt));
              }
            for (int f : kids) tr.push_back({row, f, 1.0 / kids.size()});
          }
    }
    const Csr R = from_triplets((int)bo.back(), (int)N.total, tr);
    // E: slab nodes are the composite unknowns, the others the tri-linear
    // interpolation of R u
    const Csr Pn = lattice_interp(d, n);       // fine lattice <- base lattice
    const Csr PnR = multiply(Pn, R);
    std::vector<Trip> te;
    for (size_t c = 0; c < fl.size(); ++c) {
      const int axis = (d == 3) ? (int)c : (c == 0 ? 0 : 2);
      for (int k = 0; k < fl[c].dims[2]; ++k)
        for (int j = 0; j < fl[c].dims[1]; ++j)
          for (int i = 0; i < fl[c].dims[0]; ++i) {
            const int row = (int)(fo[c] + ((long long)k * fl[c].dims[1] + j) * fl[c].dims[0] + i);
            const int kz = axis == 2 ? k + 1 : k;
            if (kz < 2 * K) {
              te.push_back({row, N.face(axis, kFine, kz, j, i), 1.0});
            } else {
              for (long long q = PnR.ptr[row]; q < PnR.ptr[row + 1]; ++q) te.push_back({row, PnR.col[q], PnR.val[q]});
            }
          }
    }
    P.E = from_triplets((int)fo.back(), (int)N.total, te);
    P.fine_ncomp = (int)fl.size();
    for (size_t c = 0; c < fl.size(); ++c) {
      for (int a = 0; a < 3; ++a) P.fine_dims[c][a] = fl[c].dims[a];
      P.fine_off[c] = fo[c];
    }
    P.fine_size = fo.back();
  }
  return "";
}

}  // namespace mac
}  // namespace selm
