// Library-internal structures shared by the host setup, the kernels and the
// C-ABI layer.  Nothing here is part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

namespace selm {

constexpr int kMaxLevels = 16;
constexpr int kMaxComps = 3;
constexpr int kStencil = 45;  // 5 (z) x 3 (y) x 3 (x) Galerkin stencil, offsets z -2..2, y/x -1..1

// 1-D lattice kinds of the MAC discretization of Section 4: periodic axes,
// the wall-normal lattice with its nodes on the walls, and cell lattices
// half a cell from the walls (odd ghost for no-slip velocity, even ghost for
// the Neumann pressure).
enum AxisKind : int {
  kAxisPeriodic = 0,   // periodic, n nodes
  kAxisVertex = 1,     // wall-normal lattice, n-1 interior nodes, Dirichlet wall nodes
  kAxisCellDir = 2,    // cell lattice, odd-reflection ghost (no-slip tangential)
  kAxisCellNeu = 3,    // cell lattice, even-reflection ghost (Neumann pressure)
  kAxisTrivial = 4     // the absent y axis of a 2-D problem
};

// Device view of one scalar component at one multigrid level.  Passed to
// kernels by value inside LevelDev.
struct CompDev {
  int nx, ny, nz;          // unknowns per axis
  long long off;           // element offset of the component in the level field
  int comp_id;             // component id used in the Philox counter
  int zkind;               // AxisKind of the wall axis
  int mx, my, mz, ncol;    // colour moduli and colour count (levels >= 1)
  double s;                // operator scale (level-0 7/5-point stencil)
  const double* S64;       // [nz][45] Galerkin stencil coefficients (levels >= 1)
  const float* S32;
  const int* rz_idx;       // restriction to the next level: [nz_coarse][4] fine z index, -1 = none
  const double* rz_w64;    // [nz_coarse][4] weights
  const float* rz_w32;
  const int* pz_idx;       // prolongation from the next level: [nz][2] coarse z index, -1 = none
  const double* pz_w64;
  const float* pz_w32;
  const double* Linv;      // coarsest level: [N][N] inverse of the Cholesky factor (row-major, lower)
  const double* zb64;      // [nz][10]: s*Mz band row then s*Kz band row (offsets -2..2)
  const float* zb32;
  double w1[9], w2[9];     // periodic x/y weights: Kx(x)My + Mx(x)Ky and Mx(x)My, index (dy+1)*3+dx+1
  float w1f[9], w2f[9];    // the same in FP32 (no per-site conversion in FP32 kernels)
};

struct LevelDev {
  int level;
  int ncomp;
  int rb;                  // 1: a banded (Galerkin-form) level smoothed in red-black order
  int flow;                // 1: FP32 cooperative colour passes may run in dataflow order
  long long size;          // elements of the whole level field
  CompDev c[kMaxComps];
};

// Host-side plan of one component at one level.
struct HostComp {
  int kind[3];             // AxisKind per axis x, y, z
  int dims[3];             // unknowns nx, ny, nz
  int comp_id;
  double Kx[3], Mx[3], Ky[3], My[3];   // periodic / trivial stencils, offsets -1..1
  std::vector<double> Kz, Mz;          // [nz][5] band rows, offsets -2..2
  int bw[3];               // bandwidths per axis
  std::vector<double> S;   // [nz][45] full stencil (scaled)
  std::vector<double> zb;  // [nz][10] scaled z bands (Mz then Kz)
  double w1[9], w2[9];     // x/y weights of the separable form
  // transfer tables to the next coarser level
  std::vector<int> rz_idx;
  std::vector<double> rz_w;
  std::vector<int> pz_idx;
  std::vector<double> pz_w;
  // coarsest level
  std::vector<double> Linv;
  int mods[3];
  long long size() const { return (long long)dims[0] * dims[1] * dims[2]; }
};

struct HostSystem {
  int dim = 3;
  int n = 0;
  int levels = 0;
  int ncomp = 0;
  double scale = 1.0;
  bool singular = false;   // pure-Neumann (pressure): regularised coarsest factor
  std::vector<HostComp> lev[kMaxLevels];
  long long level_size(int l) const {
    long long s = 0;
    for (const auto& c : lev[l]) s += c.size();
    return s;
  }
};

// Builds the Galerkin hierarchy (host, FP64).  Returns an empty string on
// success, otherwise the reason.
std::string build_velocity_system(int dim, int n, int levels, double mu, HostSystem* out);
std::string build_pressure_system(int dim, int n, int levels, HostSystem* out);
std::string build_composite_system(int dim, int n, int K, int levels_base, double mu, int ncomp, HostSystem* out);
int default_levels(int n);
// Whether the FP32 cooperative passes of a Galerkin level may run in dataflow
// order (every neighbour the passes test is coupled to the site, both ways).
bool coop_flow_ok(const HostComp& c);

// Philox stream layout shared by the kernels (see include/selm_mg.h).
inline uint32_t pack_ctr1(int level, int comp, int colour, int sweep, int kind) {
  return (uint32_t)level | ((uint32_t)comp << 4) | ((uint32_t)colour << 8) |
         ((uint32_t)sweep << 12) | ((uint32_t)kind << 20);
}

}  // namespace selm
