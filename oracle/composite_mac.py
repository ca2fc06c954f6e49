"""Composite MAC grid: divergence, gradient and projection across a refined slab.

TEST INFRASTRUCTURE ONLY (see the package header).  First piece of the
staggered composite grid with the projection: the pressure side.

Geometry (the refined-slab reading of the composite benchmark, with the MAC
staggering of Section 4): the unit box, periodic in x (and y in 3-D), walls
at z = 0 and z = 1.  Base cells have width H = 1/n; the bottom K base rows
(0 <= z <= K H) are refined by 2 over the whole periodic extent into fine
cells of width h = H/2.  K = 0 leaves the uniform base grid and K = n the
uniform fine grid.

* Cells (pressure unknowns): fine cells (m, q, p), m < 2K, centred at
  ((p+1/2) h, (q+1/2) h, (m+1/2) h); base cells (j, l, i), j >= K, centred at
  ((i+1/2) H, (l+1/2) H, (j+1/2) H).
* Faces (normal-velocity unknowns): x- and y-faces of every cell at its own
  level; z-faces between two fine layers and between two base rows; the wall
  faces carry no unknown (no penetration).  The interface z = K H is cut into
  2^(d-1) fine faces below each base cell; its normal velocity lives on the
  base face, one unknown per base cell of row K (reading: the coarse face
  owns the interface velocity, so that the paper's coarse-face gradient is
  the exact adjoint of the flux-sum divergence).
* Divergence (Eq. equ_def_discr_div): (D u)_c = (1/|c|) sum over the faces
  of c of area x outward normal velocity.  A fine cell below the interface
  sees its 1/2^(d-1) share of the base face.
* Gradient: across a face between two cells of one level, the difference of
  the two cell values over their distance (Eq. equ_def_discr_grad0); across
  the interface, (base value - mean of the 2^(d-1) fine values below) over
  (3/4) H (Eqs. equ_def_discr_grad to equ_def_discr_grad_last: the
  coarse-fine face takes the mean of the fine cells, the denominator is the
  distance between the two levels' centres).
* With face weights w_f = area x distance, sum_c |c| p_c (D u)_c =
  - sum_f w_f u_f (G p)_f, so L = D G is V-symmetric (V = diag |c|) and
  P~ = I - G L^+ D is the W-orthogonal projection onto discretely
  divergence-free fields (Section 2.1 requires P~ = P~^T in that inner
  product; Section 4 gives L = D G).
"""

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


class CompositeMAC:
    """Cells, faces, D, G and the projection of one composite MAC grid."""

    def __init__(self, n, K, dim):
        assert dim in (2, 3) and 0 <= K <= n
        self.n, self.K, self.dim = n, K, dim
        self.H = 1.0 / n
        self.h = self.H / 2.0
        ny = (lambda m: m) if dim == 3 else (lambda m: 1)
        self.fine_shape = (2 * K, ny(2 * n), 2 * n)
        self.base_shape = (n - K, ny(n), n)
        self.n_fine = int(np.prod(self.fine_shape))
        self.n_cells = self.n_fine + int(np.prod(self.base_shape))
        self.vol = np.concatenate([np.full(self.n_fine, self.h ** dim),
                                   np.full(self.n_cells - self.n_fine, self.H ** dim)])
        self.faces = []          # (axis, plus cell, [(minus cell, share)], area, dist, position)
        self._build_faces()
        self.n_faces = len(self.faces)
        self.area = np.array([f[3] for f in self.faces])
        self.dist = np.array([f[4] for f in self.faces])
        self.weight = self.area * self.dist
        self.D = self._divergence()
        self.G = self._gradient()
        self._lu = None

    # -- cells -------------------------------------------------------------
    def fine_cell(self, m, q, p):
        nz, ny, nx = self.fine_shape
        return (m * ny + (q % ny)) * nx + (p % nx)

    def base_cell(self, j, l, i):
        _, ny, nx = self.base_shape
        return self.n_fine + ((j - self.K) * ny + (l % ny)) * nx + (i % nx)

    def cell_centres(self):
        """(x, y, z) of every cell (y = 0 in 2-D)."""
        out = np.zeros((self.n_cells, 3))
        nz, ny, nx = self.fine_shape
        for m in range(nz):
            for q in range(ny):
                for p in range(nx):
                    out[self.fine_cell(m, q, p)] = ((p + .5) * self.h, (q + .5) * self.h if self.dim == 3 else 0.0,
                                                    (m + .5) * self.h)
        bz, by, bx = self.base_shape
        for j in range(self.K, self.n):
            for l in range(by):
                for i in range(bx):
                    out[self.base_cell(j, l, i)] = ((i + .5) * self.H, (l + .5) * self.H if self.dim == 3 else 0.0,
                                                    (j + .5) * self.H)
        return out

    # -- faces -------------------------------------------------------------
    def _build_faces(self):
        d, h, H, K, n = self.dim, self.h, self.H, self.K, self.n
        fa, Ha = h ** (d - 1), H ** (d - 1)
        nz, ny, nx = self.fine_shape
        bz, by, bx = self.base_shape
        # periodic axes: the face at the low side of each cell, between its
        # left neighbour (minus) and the cell (plus)
        for m in range(nz):
            for q in range(ny):
                for p in range(nx):
                    c = self.fine_cell(m, q, p)
                    self.faces.append((0, c, [(self.fine_cell(m, q, p - 1), 1.0)], fa, h, (p * h, q, m)))
                    if d == 3:
                        self.faces.append((1, c, [(self.fine_cell(m, q - 1, p), 1.0)], fa, h, (p, q * h, m)))
        for j in range(K, n):
            for l in range(by):
                for i in range(bx):
                    c = self.base_cell(j, l, i)
                    self.faces.append((0, c, [(self.base_cell(j, l, i - 1), 1.0)], Ha, H, (i * H, l, j)))
                    if d == 3:
                        self.faces.append((1, c, [(self.base_cell(j, l - 1, i), 1.0)], Ha, H, (i, l * H, j)))
        # wall-normal axis: interior faces of the slab, the interface, the base
        for m in range(1, nz):
            for q in range(ny):
                for p in range(nx):
                    self.faces.append((2, self.fine_cell(m, q, p), [(self.fine_cell(m - 1, q, p), 1.0)], fa, h,
                                       (p, q, m * h)))
        if 0 < K < n:
            kids = 2 ** (d - 1)
            for l in range(by):
                for i in range(bx):
                    below = [(self.fine_cell(nz - 1, 2 * l + a if d == 3 else 0, 2 * i + c), 1.0 / kids)
                             for a in range(2 if d == 3 else 1) for c in range(2)]
                    self.faces.append((2, self.base_cell(K, l, i), below, Ha, 0.75 * H, (i, l, K * H)))
        for j in range(K + 1, n):
            for l in range(by):
                for i in range(bx):
                    self.faces.append((2, self.base_cell(j, l, i), [(self.base_cell(j - 1, l, i), 1.0)], Ha, H,
                                       (i, l, j * H)))

    def _divergence(self):
        rows, cols, vals = [], [], []
        for f, (axis, plus, minus, area, dist, _) in enumerate(self.faces):
            rows.append(plus)
            cols.append(f)
            vals.append(-area / self.vol[plus])              # inflow through the plus cell's low face
            for c, share in minus:
                rows.append(c)
                cols.append(f)
                vals.append(share * area / self.vol[c])      # outflow through the minus cells' high faces
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.n_cells, self.n_faces))

    def _gradient(self):
        rows, cols, vals = [], [], []
        for f, (axis, plus, minus, area, dist, _) in enumerate(self.faces):
            rows.append(f)
            cols.append(plus)
            vals.append(1.0 / dist)
            for c, share in minus:
                rows.append(f)
                cols.append(c)
                vals.append(-share / dist)
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.n_faces, self.n_cells))

    # -- pressure operator and projection ----------------------------------
    def laplacian(self):
        """L = D G (Eq. equ_def_L) on the composite cells, no flux through the walls."""
        return (self.D @ self.G).tocsr()

    def _solver(self):
        if self._lu is None:
            S = (sp.diags(self.vol) @ self.laplacian()).tocsc()     # V L: symmetric, kernel = constants
            self._lu = spla.splu(S[1:, 1:].tocsc())                  # cell 0 pinned: nonsingular
        return self._lu

    def pressure_solve(self, rhs):
        """phi with L phi = rhs and sum |c| phi_c = 0, for a rhs with sum |c| rhs_c = 0
        (a consistent right-hand side: the walls carry no flux)."""
        b = self.vol * rhs
        phi = np.zeros(self.n_cells)
        phi[1:] = self._solver().solve(b[1:])
        return phi - (self.vol @ phi) / self.vol.sum()

    def project(self, u):
        """P~ u = u - G phi, L phi = D u."""
        return u - self.G @ self.pressure_solve(self.D @ u)
