// Staggered (MAC) composite grid with a refined slab: host-side plan.
// Library-internal; nothing here is part of the public ABI.
//
// Geometry (Section 4 with the refined-slab composite of Section 3.2): the
// unit box, periodic in x (and y in 3-D), no-slip walls at z = 0 and z = 1;
// base cells of width H = 1/n, the bottom K base rows refined by 2 over the
// whole periodic extent.  Unknowns are the normal velocities of the faces of
// the fine and base cells (velocity) and the cell-centre pressures.  Every
// operator of this grid is held as an explicit sparse matrix built once on
// the host: the composite velocity operator, divergence, gradient, pressure
// operator, the transfers of the FAC base hierarchy with its Galerkin
// operators, and the extension of composite fields to the uniform fine
// lattice that carries the particle kernels.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace selm {
namespace mac {

// Compressed sparse rows, FP64 values, columns ascending within a row.
struct Csr {
  int nr = 0, nc = 0;
  std::vector<long long> ptr{0};
  std::vector<int> col;
  std::vector<double> val;
  long long nnz() const { return (long long)col.size(); }
};

struct Plan {
  int dim = 3, n = 0, K = 0, levels = 0;
  double mu = 1.0;
  int n_faces = 0, n_cells = 0, n_fine_cells = 0;
  // velocity (faces) and pressure (cells)
  Csr A;                         // A = -mu V L on the faces (energy form)
  Csr D, G;                      // divergence (cells x faces), gradient (faces x cells)
  Csr S;                         // diag(vol) D G: symmetric, kernel = constants
  std::vector<double> vol;       // cell volumes
  std::vector<double> weight;    // face weights area x distance
  // FAC base hierarchy
  Csr P;                         // composite faces <- base level 0
  std::vector<Csr> Pl;           // base level l <- base level l + 1
  std::vector<Csr> ops;          // Galerkin operators of the base levels
  std::vector<std::vector<std::vector<int>>> colours;   // [level][class] rows, ascending
  std::vector<std::vector<int>> patch_colours;          // classes of the slab faces (composite indices)
  std::vector<double> Linv;      // coarsest level: inverse Cholesky factor, row-major lower
  // particles: the uniform fine MAC lattice (2n cells per axis)
  Csr E;                         // fine lattice nodes <- composite faces
  int fine_ncomp = 0;
  int fine_dims[3][3] = {};      // [comp] {nx, ny, nz}
  long long fine_off[3] = {};
  long long fine_size = 0;
};

// Off-diagonal entries at or below this fraction of their row's diagonal are
// rounding residues of exact cancellations in the Galerkin products and are
// not couplings of the colouring graph.
constexpr double kGraphRtol = 1e-12;

// Builds the plan; returns an empty string on success, else the reason.
std::string build_plan(int dim, int n, int K, int levels, double mu, Plan* out);

}  // namespace mac
}  // namespace selm
