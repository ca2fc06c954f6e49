/*
 * selm_mac.h - C ABI of the staggered (MAC) composite grid: the velocity and
 * pressure unknowns of Section 4 on a grid whose bottom K base rows are
 * refined by 2 over the whole periodic extent, with the composite
 * divergence, gradient and projection, the stochastic FAC iteration of
 * Algorithms 1-3 on the composite velocity operator, and particles coupled
 * through the fine level's kernel (Algorithm 4).
 *
 * Conventions are those of selm_mg.h (device pointers owned by the caller,
 * every call enqueued on `stream`, status codes of selm_status).  The paper
 * writes its composite rules for cell-centred unknowns; the staggered rules
 * this library uses are:
 *
 * - Unknowns.  Base cells have width H = 1/n, fine cells h = H/2; fine cells
 *   cover 0 <= z <= K H.  Pressures sit at the cell centres, normal
 *   velocities on the cell faces; the wall faces carry no unknown; the
 *   interface z = K H carries one velocity per base cell of row K (the
 *   coarse face owns the interface flux).
 * - Face order of a composite velocity vector (selm_mac_faces() entries):
 *   (1) per fine cell (m, q, p) in (z, y, x) order its low x face, then (3-D)
 *   its low y face; (2) the same for the base cells of rows K..n-1; (3) the
 *   z faces between fine layers m = 1..2K-1; (4) the interface faces (when
 *   0 < K < n); (5) the z faces between base rows K+1..n-1.  Cell order of a
 *   pressure vector: the fine cells (m, q, p), then the base cells.
 * - Divergence (Eq. equ_def_discr_div): the flux sum over a cell's faces
 *   over its volume, a fine cell below the interface taking its 1/2^(d-1)
 *   share of the base face.  Gradient: the difference of the two cell values
 *   over their distance, across the interface (base value - mean of the
 *   fine cells below) / (3/4 H) (Eqs. equ_def_discr_grad to
 *   equ_def_discr_grad_last).  L = D G is symmetric in the cell-volume inner
 *   product and P~ = I - G L^+ D is the projection onto discretely
 *   divergence-free fields, orthogonal in the face-weight (area x distance)
 *   inner product W.
 * - Velocity operator A = -mu V L, per component, from the energy form
 *   mu sum (area/dist)(u_a - u_b)^2 over the box faces shared by two nodes of
 *   one level, the walls, and one term (area/dist)(u_c - sum w_f u_f)^2 per
 *   coarse-fine group, w_f the share of the base node's box face that the
 *   fine node covers; dist = 3/4 H for the tangential components and h for
 *   the wall-normal one.
 * - FAC (Algorithm 1 around Algorithm 2): r = b - A z; q_b = V-cycle on the
 *   base MAC grid of P^T r (Algorithm 3 with tri-linear transfers, Galerkin
 *   operators, an exact draw on the coarsest level); q = P q_b (identity on
 *   the base faces that stay unknowns, tri-linear on the slab); nu heat-bath
 *   sweeps of A q = r over the slab faces; z += q.  Every sparse level is
 *   visited in the colour classes of a first-fit colouring of its graph in
 *   index order.
 * - Noise: Philox4x32-10 as in selm_mg.h; base level l sweeps take the
 *   class rank, level l + 1, component 0, kind 0; the coarsest draw kind 1;
 *   the slab sweeps kind 2 addressed by the face index; colour classes from
 *   16 continue in counter word 1's top byte (colour >> 4) << 24.
 * - Particles (reading of Algorithm 4 on this grid): every particle uses the
 *   fine level's 4-point kernel on the uniform fine MAC lattice (2n cells per
 *   axis); a lattice node takes the composite value on the slab and above it
 *   the tri-linear interpolation of the base field (the composite value on
 *   base faces, the mean of the coinciding fine faces on covered ones).
 *   M = Gamma P~ A^-1 P~^T Gamma^T, g = sqrt(2 kT) Gamma P~ xi with
 *   P~^T = W P~ W^-1.
 */
#ifndef SELM_MAC_H
#define SELM_MAC_H

#include <stddef.h>
#include <stdint.h>

#include "selm_mg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct selm_mac selm_mac;  /* opaque handle, owned by the library */

typedef struct {
  int dim;             /* 2 or 3 */
  int n;               /* base cells per axis; even, divisible by 2^(levels-1) */
  int K;               /* refined base rows, 0 <= K <= n (0: uniform base grid, n: uniform fine grid) */
  int levels;          /* base multigrid levels; 0 = coarsen while the edge stays even and >= 4 */
  double mu;           /* viscosity; 0 -> 1 */
  double kT;           /* thermal energy of the particle dynamics; 0 -> none */
  int nu_pre, nu_post; /* (mu1, mu2) sweeps of the base V-cycle; 0 -> 2 */
  int nu_patch;        /* sweeps over the slab per FAC cycle; 0 -> 2 */
  int precision;       /* SELM_FP64, or SELM_FP32_REFINE64 (FP32 V-cycle and slab sweeps, FP64 residual and update) */
  int projection;      /* SELM_PROJ_NONE (P~ = I) or SELM_PROJ_MAC */
  double tol;          /* FAC stop ||b - A z|| <= tol ||b||; 0 -> 1e-10 */
  int max_cycles;      /* 0 -> 100 */
  double proj_tol;     /* relative residual of the pressure solve of P~; 0 -> 1e-13 */
  uint64_t seed, instance;   /* Philox key material of the chain */
} selm_mac_desc;

/* Validate `desc`, build every operator on the host (FP64), upload on
   `stream`.  The host build is O(unknowns); the coarsest base level must
   hold at most 8192 unknowns. */
selm_status selm_mac_create(const selm_mac_desc* desc, void* stream, selm_mac** out);
selm_status selm_mac_destroy(selm_mac* h);
const char* selm_mac_last_error(const selm_mac* h);

/* Sizes: composite velocity unknowns, pressure cells, base levels, colour
   classes of base level `level` (level = -1: the slab faces). */
long long selm_mac_faces(const selm_mac* h);
long long selm_mac_cells(const selm_mac* h);
int selm_mac_levels(const selm_mac* h);
int selm_mac_colours(const selm_mac* h, int level);
/* Element size (4 or 8) of the inner cycle's fields. */
int selm_mac_inner_bytes(const selm_mac* h);

/* ---- operators -------------------------------------------------------- */
/* Au = A u (velocity operator), FP64. */
selm_status selm_mac_apply(selm_mac* h, const double* u, double* Au, void* stream);
/* div = D u (cells), grad = G p (faces), FP64. */
selm_status selm_mac_divergence(selm_mac* h, const double* u, double* div, void* stream);
selm_status selm_mac_gradient(selm_mac* h, const double* p, double* grad, void* stream);
/* out = P~ u (adjoint = 0) or P~^T u = W P~ W^-1 u (adjoint = 1); out may
   equal u.  The pressure L phi = D u (phi of zero volume mean) is solved by
   conjugate gradients on diag(vol) L (Jacobi preconditioned, FP64) to
   proj_tol; iters / resid (optional HOST pointers) receive the iteration
   count and relative residual (synchronises the stream). */
selm_status selm_mac_project(selm_mac* h, const double* u, double* out, int adjoint, int* iters, double* resid,
                             void* stream);

/* ---- FAC (Algorithms 1-3) --------------------------------------------- */
/* One FAC cycle z <- z + q for A z = b with noise amplitude sigma (0: the
   deterministic cycle; 1 keeps N(A^-1 b, A^-1) invariant) and Philox
   counter `cycle` (counter words 2-3). */
selm_status selm_mac_fac_cycle(selm_mac* h, double* z, const double* b, double sigma, uint64_t cycle,
                               void* stream);
/* FAC cycles from the given z until ||b - A z|| <= tol ||b|| (tol = 0: the
   descriptor's).  cycles / rel: optional HOST pointers.  Synchronises. */
selm_status selm_mac_solve(selm_mac* h, double* z, const double* b, double tol, int max_cycles, int* cycles,
                           double* rel, void* stream);
/* Advance the persistent chain xi (starts at 0, counter 0) by `ncycles`
   stochastic cycles with b = 0 and sigma = 1 (xi -> N(0, A^-1)); xi_out
   (optional, device, selm_mac_faces() doubles) receives a copy. */
selm_status selm_mac_sample(selm_mac* h, int ncycles, double* xi_out, void* stream);
/* Device pointer of xi and the counter of the next chain cycle. */
selm_status selm_mac_chain(selm_mac* h, double** xi, uint64_t* cycle);
selm_status selm_mac_set_chain(selm_mac* h, uint64_t cycle, void* stream);   /* xi = 0, counter = cycle */

/* ---- particles (Algorithm 4) ------------------------------------------ */
/* U = Gamma u at X (interpolation through the fine lattice). */
selm_status selm_mac_interp(selm_mac* h, int np, const double* X, const double* u, double* U, void* stream);
/* f = Gamma^T F (spreading, the adjoint of selm_mac_interp). */
selm_status selm_mac_spread(selm_mac* h, int np, const double* X, const double* F, double* f, void* stream);
/* U = M F = Gamma P~ A^-1 P~^T Gamma^T F (FAC solve to tol).  cycles:
   optional HOST pointer (synchronises). */
selm_status selm_mac_mobility(selm_mac* h, int np, const double* X, const double* F, double* U, int* cycles,
                              void* stream);
/* Advance the chain by `ncycles` and return g = sqrt(2 kT) Gamma P~ xi at X. */
selm_status selm_mac_thermal(selm_mac* h, int np, const double* X, int ncycles, double* g, void* stream);
/* `nsteps` Euler-Maruyama steps with fixed forces F (Algorithm 4):
   u = A^-1 P~^T Gamma^T F, the chain advanced by ncycles,
   X <- X + Gamma P~ (dt u + sqrt(2 kT dt) xi), then periodic wrap and
   reflection at the walls.  X: [np][dim], updated in place. */
selm_status selm_mac_step(selm_mac* h, int np, double* X, const double* F, double dt, int nsteps, int ncycles,
                          void* stream);

/* Cycles run so far by the handle (deterministic and stochastic). */
long long selm_mac_total_cycles(const selm_mac* h);

/* ---- host-side inspection of the plan (no GPU needed) -------------------
   Build the plan of `desc` on the host and return one of its sparse matrices
   in compressed sparse rows (0-based, columns ascending): *ptr has nr + 1
   entries, *col / *val nnz; the three arrays are HOST memory allocated by
   the library, released with selm_mac_host_free.  `level` selects the base
   level of SELM_MAC_MAT_OPS (Galerkin operator) and SELM_MAC_MAT_PL
   (interpolation from level + 1).  SELM_EINVAL for an invalid descriptor or
   selector. */
enum {
  SELM_MAC_MAT_A = 0,    /* composite velocity operator (faces x faces) */
  SELM_MAC_MAT_D = 1,    /* divergence (cells x faces) */
  SELM_MAC_MAT_G = 2,    /* gradient (faces x cells) */
  SELM_MAC_MAT_S = 3,    /* diag(cell volume) D G */
  SELM_MAC_MAT_P = 4,    /* composite faces <- base level 0 */
  SELM_MAC_MAT_E = 5,    /* fine lattice nodes <- composite faces */
  SELM_MAC_MAT_OPS = 6,  /* Galerkin operator of base level `level` */
  SELM_MAC_MAT_PL = 7    /* base level `level` <- level + 1 */
};
selm_status selm_mac_host_matrix(const selm_mac_desc* desc, int which, int level, int* nr, int* nc, long long* nnz,
                                 long long** ptr, int** col, double** val);
/* Colour class of every row of base level `level` (level = -1: every
   composite face, -1 for the faces outside the slab), HOST array of *n ints
   released with selm_mac_host_free. */
selm_status selm_mac_host_colours(const selm_mac_desc* desc, int level, int* n, int** colour);
void selm_mac_host_free(void* p);

#ifdef __cplusplus
}
#endif

#endif /* SELM_MAC_H */
