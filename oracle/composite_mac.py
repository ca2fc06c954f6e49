"""Composite MAC grid: divergence, gradient and projection across a refined slab.

TEST INFRASTRUCTURE ONLY (see the package header).  The staggered composite
grid with the projection: divergence, gradient, the projection (reading
R21), the velocity operators of the three components (reading R22), the
stochastic FAC cycle on them (reading R23) and particles on the grid
(reading R24).

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

from . import coupling, grid


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
        self.faces = []          # (axis, plus cell, [(minus cell, share)], area, dist, key)
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
    def _add_face(self, key, plus, minus, area, dist):
        self.face_of[key] = len(self.faces)
        self.faces.append((key[0], plus, minus, area, dist, key))

    def _build_faces(self):
        """Faces keyed (axis, level, k, j, i): level 'f' fine, 'c' base, 'i' the
        interface; (k, j, i) are the plus cell's indices at that level (for
        the interface, k = K)."""
        d, h, H, K, n = self.dim, self.h, self.H, self.K, self.n
        fa, Ha = h ** (d - 1), H ** (d - 1)
        nz, ny, nx = self.fine_shape
        bz, by, bx = self.base_shape
        self.face_of = {}
        # periodic axes: the face at the low side of each cell, between its
        # left neighbour (minus) and the cell (plus)
        for m in range(nz):
            for q in range(ny):
                for p in range(nx):
                    c = self.fine_cell(m, q, p)
                    self._add_face((0, "f", m, q, p), c, [(self.fine_cell(m, q, p - 1), 1.0)], fa, h)
                    if d == 3:
                        self._add_face((1, "f", m, q, p), c, [(self.fine_cell(m, q - 1, p), 1.0)], fa, h)
        for j in range(K, n):
            for l in range(by):
                for i in range(bx):
                    c = self.base_cell(j, l, i)
                    self._add_face((0, "c", j, l, i), c, [(self.base_cell(j, l, i - 1), 1.0)], Ha, H)
                    if d == 3:
                        self._add_face((1, "c", j, l, i), c, [(self.base_cell(j, l - 1, i), 1.0)], Ha, H)
        # wall-normal axis: interior faces of the slab, the interface, the base
        for m in range(1, nz):
            for q in range(ny):
                for p in range(nx):
                    self._add_face((2, "f", m, q, p), self.fine_cell(m, q, p), [(self.fine_cell(m - 1, q, p), 1.0)],
                                   fa, h)
        if 0 < K < n:
            kids = 2 ** (d - 1)
            for l in range(by):
                for i in range(bx):
                    below = [(self.fine_cell(nz - 1, 2 * l + a if d == 3 else 0, 2 * i + c), 1.0 / kids)
                             for a in range(2 if d == 3 else 1) for c in range(2)]
                    self._add_face((2, "i", K, l, i), self.base_cell(K, l, i), below, Ha, 0.75 * H)
        for j in range(K + 1, n):
            for l in range(by):
                for i in range(bx):
                    self._add_face((2, "c", j, l, i), self.base_cell(j, l, i), [(self.base_cell(j - 1, l, i), 1.0)],
                                   Ha, H)

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

    def face_positions(self):
        """(x, y, z) of every velocity node (the centre of its face; y = 0 in 2-D)."""
        out = np.zeros((self.n_faces, 3))
        for f, (axis, plus, minus, area, dist, key) in enumerate(self.faces):
            _, lev, k, j, i = key
            s = self.h if lev == "f" else self.H
            pos = [(i + 0.5) * s, (j + 0.5) * s, (k + 0.5) * s]
            pos[axis] -= 0.5 * s                  # the plus cell's low face
            if lev == "i":
                pos[2] = self.K * self.H
            if self.dim == 2:
                pos[1] = 0.0
            out[f] = pos
        return out

    # -- velocity operator ---------------------------------------------------
    def interface_groups(self, a):
        """Coarse-fine groups of component a across the interface: (base node,
        [(fine node, omega)], distance between the two rows of nodes).  omega is
        the part of the base node's box face covered by the fine node's box
        face: (1/4, 1/2, 1/4) along the component's own periodic axis (its
        nodes are faces, the base face spans two fine cells), 1/2 across a cell
        axis, and 1/2^(d-1) for the wall-normal component (cell-type along x
        and y)."""
        d, h, H, K, n = self.dim, self.h, self.H, self.K, self.n
        nz, ny, nx = self.fine_shape
        bz, by, bx = self.base_shape
        F = self.face_of
        out = []
        if not 0 < K < n:
            return out
        cross = [(e, 0.5) for e in range(2)] if d == 3 else [(0, 1.0)]
        for j in range(by):
            for i in range(bx):
                fine = []
                if a == 2:
                    for e, we in cross:
                        for t in range(2):
                            fine.append((F[(2, "f", nz - 1, (2 * j + e) if d == 3 else 0, 2 * i + t)], 0.5 * we))
                    out.append((F[(2, "i", K, j, i)], fine, h))
                    continue
                for dt, wt in ((-1, 0.25), (0, 0.5), (1, 0.25)):
                    for e, we in cross:
                        if a == 0:
                            key = (0, "f", nz - 1, (2 * j + e) % ny, (2 * i + dt) % nx)
                        else:
                            key = (1, "f", nz - 1, (2 * j + dt) % ny, (2 * i + e) % nx)
                        fine.append((F[key], wt * we))
                out.append((F[(a, "c", K, j, i)], fine, 0.75 * H))
        return out

    def velocity_operator(self, mu=1.0):
        """A = -mu V L on the face unknowns, one composite operator per component
        (reading R22), assembled from its energy form

            u^T A u = mu sum_pairs (area / dist) (u_a - u_b)^2
                    + mu sum_walls (area / dist) u^2
                    + mu sum_groups (area_c / dist) (u_c - sum_f omega_f u_f)^2.

        Each velocity node owns the box between the centres of the two cells
        its face separates (along the face normal) and its cell's extent along
        the other axes.  Pairs are nodes of one level whose boxes share a face
        (area of the shared face, distance between the nodes).  A wall at a
        box face sets the node value against 0 at the wall (distance from the
        node to the wall).  Across the refinement interface a base node c
        faces the fine nodes under its box; omega_f is the part of c's box face
        that fine node f's box face covers (the flux-sum rule of Eq.
        equ_def_discr_div), and dist is the distance between the two rows of
        nodes: (3/4) H for the x and y components, as in Eq. equ_def_discr_grad,
        and h for the wall-normal component (its interface node sits on the
        interface).  For cell-centred components this is the paper's rule."""
        d, h, H, K, n = self.dim, self.h, self.H, self.K, self.n
        nz, ny, nx = self.fine_shape
        bz, by, bx = self.base_shape
        F = self.face_of
        rows, cols, vals = [], [], []

        def term(weight, coeffs):
            for a, ca in coeffs:
                for b, cb in coeffs:
                    rows.append(a)
                    cols.append(b)
                    vals.append(mu * weight * ca * cb)

        def pair(weight, a, b):
            term(weight, [(a, 1.0), (b, -1.0)])

        axes = [0, 1] if d == 3 else [0]
        # x and y components: cell-type across the walls
        for a in axes:
            o = 1 - a if d == 3 else None            # the other periodic axis
            for lev, s, rows_k, shape in (("f", h, range(nz), (ny, nx)), ("c", H, range(K, n), (by, bx))):
                area = s ** (d - 1)
                for k in rows_k:
                    for j in range(shape[0]):
                        for i in range(shape[1]):
                            me = F[(a, lev, k, j, i)]
                            # along the component's own axis (through the cell), then the other one
                            nxt = (k, j, i + 1) if a == 0 else (k, j + 1, i)
                            pair(area / s, me, F[(a, lev, nxt[0], nxt[1] % shape[0], nxt[2] % shape[1])])
                            if o is not None:
                                nb = (k, j, i + 1) if o == 0 else (k, j + 1, i)
                                pair(area / s, me, F[(a, lev, nb[0], nb[1] % shape[0], nb[2] % shape[1])])
                            top = nz - 1 if lev == "f" else n - 1
                            if k < top:
                                pair(area / s, me, F[(a, lev, k + 1, j, i)])
                            if lev == "f" and k == 0 or lev == "c" and k == 0:
                                term(area / (s / 2), [(me, 1.0)])           # bottom wall
                            if lev == "c" and k == n - 1 or lev == "f" and k == nz - 1 and K == n:
                                term(area / (s / 2), [(me, 1.0)])           # top wall
            for c, fine, dist in self.interface_groups(a):
                term(H ** (d - 1) / dist, [(c, 1.0)] + [(f, -w) for f, w in fine])
        # wall-normal component: vertex-type across the walls
        a = 2
        nodes = []                                  # (key, spacing along x/y, box height, z)
        for m in range(1, nz):
            for q in range(ny):
                for p in range(nx):
                    nodes.append(((2, "f", m, q, p), h, h, m * h))
        if 0 < K < n:
            for l in range(by):
                for i in range(bx):
                    nodes.append(((2, "i", K, l, i), H, 0.75 * H, K * H))
        for j in range(K + 1, n):
            for l in range(by):
                for i in range(bx):
                    nodes.append(((2, "c", j, l, i), H, H, j * H))
        for key, s, height, z in nodes:
            me = F[key]
            lev, k, j, i = key[1], key[2], key[3], key[4]
            dims = (ny, nx) if lev == "f" else (by, bx)
            side = s ** (d - 2) * height                    # area of a box face normal to x or y
            pair(side / s, me, F[(2, lev, k, j, (i + 1) % dims[1])])
            if d == 3:
                pair(side / s, me, F[(2, lev, k, (j + 1) % dims[0], i)])
            area = s ** (d - 1)                             # box face normal to z
            if lev == "f":
                if k + 1 < nz:
                    pair(area / h, me, F[(2, "f", k + 1, j, i)])
                elif K == n:
                    term(area / h, [(me, 1.0)])                                 # top wall
                if k == 1:
                    term(area / h, [(me, 1.0)])                                 # bottom wall
            else:
                up = (2, "c", (K + 1 if lev == "i" else k + 1), j, i)
                if up in F:
                    pair(area / H, me, F[up])
                else:
                    term(area / H, [(me, 1.0)])                                 # top wall
                if lev == "c" and k == 1:
                    term(area / H, [(me, 1.0)])                                 # bottom wall (K = 0)
        for c, fine, dist in self.interface_groups(2):   # interface node against the fine row below it
            term(H ** (d - 1) / dist, [(c, 1.0)] + [(f, -w) for f, w in fine])
        return sp.csr_matrix((vals, (rows, cols)), shape=(self.n_faces, self.n_faces))


# ---- stochastic FAC on the staggered composite grid (Algorithms 1-3) ----

# An off-diagonal entry below this fraction of its row's diagonal is the
# rounding residue of an exact cancellation in a Galerkin product (the exact
# entry is 0), not a coupling of the graph.
GRAPH_RTOL = 1e-12


def _greedy_colours(A):
    """Colour classes of the graph of A (a_ij != 0, i != j), each an independent
    set, by first fit in index order: a valid Gibbs visiting order.  Entries
    with |a_ij| <= GRAPH_RTOL |a_ii| are exact zeros up to rounding and are
    not edges, so the classes do not depend on the summation order of the
    Galerkin products."""
    A = sp.csr_matrix(A)
    if A.shape[0] == 0:
        return []
    diag = np.abs(A.diagonal())
    colour = -np.ones(A.shape[0], dtype=int)
    for i in range(A.shape[0]):
        lo, hi = A.indptr[i], A.indptr[i + 1]
        used = {colour[j] for j, a in zip(A.indices[lo:hi], A.data[lo:hi])
                if j != i and colour[j] >= 0 and abs(a) > GRAPH_RTOL * diag[i]}
        c = 0
        while c in used:
            c += 1
        colour[i] = c
    return [np.nonzero(colour == c)[0] for c in range(colour.max() + 1)]


def _kron3(Pz, Py, Px):
    return sp.kron(sp.csr_matrix(Pz), sp.kron(sp.csr_matrix(Py), sp.csr_matrix(Px))).tocsr()


class CompositeMACFAC:
    """FAC for the velocity of a composite MAC grid (reading R23).

    Base level (1) = the uniform MAC velocity grid of n cells, components
    (u, v, w) flattened (z, y, x) as in grid.velocity_system.  P maps the base
    unknowns to the composite ones: the identity on the base nodes that stay
    unknowns, and on the refined slab the uniform tri-linear interpolation of
    grid.prolongation (the component's lattice types) from the base nodes.
    The base operator is the Galerkin product A_1 = P^T A P, the levels below
    it P_l^T A_l P_l with the uniform tri-linear P_l, and the coarsest level is
    the exact block draw.  A cycle (Algorithm 1 around Algorithm 2):
        r = b - A z;  q_1 = V-Cycle(0, P^T r);  q = P q_1;
        nu Gibbs sweeps on the refined-slab unknowns of A q = r;  z += q,
    with every Gibbs sweep a heat-bath pass over colour classes of the
    operator's graph (first-fit colouring).
    """

    def __init__(self, g, mu=1.0, levels=None):
        self.g = g
        self.A = g.velocity_operator(mu).tocsr()
        n, d = g.n, g.dim
        self.base = grid.velocity_system(n, d, mu=mu, levels=levels)
        self.P = self._prolongation()
        self.fine = np.array([f[5][1] == "f" for f in g.faces])
        ops = [(self.P.T @ self.A @ self.P).tocsr()]
        self.Pl = []
        for lev in range(self.base.nlevels - 1):
            Pl = sp.block_diag([_kron3(Ps[2], Ps[1], Ps[0]) for Ps in self.base.P[lev]]).tocsr()
            self.Pl.append(Pl)
            ops.append((Pl.T @ ops[-1] @ Pl).tocsr())
        self.ops = ops
        self.colours = [_greedy_colours(A) for A in ops[:-1]]
        self.chol = np.linalg.cholesky(ops[-1].toarray())
        idx = np.nonzero(self.fine)[0]
        self.patch = idx
        self.patch_colours = [idx[c] for c in _greedy_colours(self.A[idx][:, idx])]

    def _prolongation(self):
        g, n, d, K = self.g, self.g.n, self.g.dim, self.g.K
        kinds = self.base.kinds
        offs = np.cumsum([0] + [cl.size for cl in self.base.levels[0]])
        shapes = [cl.shape for cl in self.base.levels[0]]
        comp_of_axis = {0: 0, 1: 1, 2: 2} if d == 3 else {0: 0, 2: 1}
        up = {}
        rows, cols, vals = [], [], []
        for f, (axis, plus, minus, area, dist, key) in enumerate(g.faces):
            _, lev, k, j, i = key
            c = comp_of_axis[axis]
            nz, ny, nx = shapes[c]
            if lev != "f":                                  # a base node that stays an unknown
                kk = k - 1 if axis == 2 else k
                rows.append(f)
                cols.append(offs[c] + (kk * ny + (j if d == 3 else 0)) * nx + i)
                vals.append(1.0)
                continue
            if c not in up:                                 # tri-linear n -> 2n of this component
                P1 = [grid.prolongation(kd, n if kd != "O" else 1) for kd in kinds[c]]
                up[c] = (_kron3(P1[2], P1[1], P1[0]).tocsr(), [p.shape[0] for p in P1])
            Pc, (fx, fy, fz) = up[c]
            kk = k - 1 if axis == 2 else k
            row = Pc.getrow((kk * fy + (j if d == 3 else 0)) * fx + i)
            for col, v in zip(row.indices, row.data):
                rows.append(f)
                cols.append(offs[c] + col)
                vals.append(v)
        return sp.csr_matrix((vals, (rows, cols)), shape=(g.n_faces, offs[-1]))

    # -- one V-cycle on the base hierarchy (Algorithm 3) --------------------
    def _sweep(self, lev, v, b, sweep, noise, sigma):
        A = self.ops[lev]
        diag = A.diagonal()
        for colour, idx in enumerate(self.colours[lev]):
            off = A[idx] @ v - diag[idx] * v[idx]
            new = (b[idx] - off) / diag[idx]
            if sigma != 0.0:
                new = new + sigma * noise.sweep(lev + 1, 0, colour, sweep, idx.size) / np.sqrt(diag[idx])
            v[idx] = new

    def vcycle(self, lev, v, b, noise, sigma, mu1=2, mu2=2):
        if lev == len(self.ops) - 1:
            y = np.linalg.solve(self.chol, b)
            if sigma != 0.0:
                y = y + sigma * noise.coarsest(lev + 1, 0, y.size)
            v[:] = np.linalg.solve(self.chol.T, y)
            return v
        for s in range(mu1):
            self._sweep(lev, v, b, s, noise, sigma)
        bc = self.Pl[lev].T @ (b - self.ops[lev] @ v)
        vc = np.zeros(bc.size)
        self.vcycle(lev + 1, vc, bc, noise, sigma, mu1, mu2)
        v += self.Pl[lev] @ vc
        for s in range(mu2):
            self._sweep(lev, v, b, mu1 + s, noise, sigma)
        return v

    # -- the composite cycle (Algorithms 1 and 2) ----------------------------
    def fac_cycle(self, z, b, noise, sigma, mu1=2, mu2=2, nu=2):
        r = b - self.A @ z
        qb = np.zeros(self.P.shape[1])
        self.vcycle(0, qb, self.P.T @ r, noise, sigma, mu1, mu2)
        q = self.P @ qb
        diag = self.A.diagonal()
        for s in range(nu):
            for colour, idx in enumerate(self.patch_colours):
                off = self.A[idx] @ q - diag[idx] * q[idx]
                new = (r[idx] - off) / diag[idx]
                if sigma != 0.0:
                    new = new + sigma * noise.patch(0, colour, s, idx) / np.sqrt(diag[idx])
                q[idx] = new
        z += q
        return z

    def solve(self, b, tol=1e-10, max_cycles=200):
        from .philox import ExplicitNoise
        z = np.zeros_like(b)
        bn = np.linalg.norm(b)
        cycles, rel = 0, np.linalg.norm(b - self.A @ z) / bn
        while rel > tol and cycles < max_cycles:
            self.fac_cycle(z, b, ExplicitNoise(), 0.0)
            cycles += 1
            rel = np.linalg.norm(b - self.A @ z) / bn
        return z, cycles, rel


# ---- particles on the composite MAC grid (Algorithm 4; reading R24) ----

class CompositeSELM:
    """Mobility and thermal velocities of particles on a composite MAC grid.

    kernel = "fine" (default): every particle uses the fine level's 4-point
    kernel, so its size does not change when it crosses the interface;
    kernel = "cover": a particle uses the level whose cells cover it, the fine
    level below the interface (z < K H) and the base level above (its
    self-mobility then jumps by about a fifth at the interface).  The 4^d
    Peskin nodes are nodes of that level's whole uniform MAC lattice; their
    values come from the composite field through
      R: base field = the composite value on base nodes that are unknowns,
         and on covered base nodes the mean of the 2^(d-1) fine faces that
         coincide with the base face;
      E: fine field = the composite value on the slab's fine nodes, and
         elsewhere the uniform tri-linear interpolation (grid.prolongation)
         of the base field R u.
    Gamma (interpolation) is the Peskin sum on that field (coupling.stencil),
    so Gamma = I_level(X) R or I_level(X) E.  With A = -mu V L the force
    density is Lambda F = V^-1 Gamma^T F, and
        M = Gamma P~ A^-1 P~^T Gamma^T,   g = sqrt(2 kT) Gamma P~ xi,
    P~^T = W P~ W^-1 the adjoint of the W-orthogonal projection acting on the
    spread forces; M is symmetric and Cov(g) = 2 kT M.
    """

    def __init__(self, n, K, dim, mu=1.0, kT=1.0, project=False, kernel="fine", seed=0, instance=0, tol=1e-10):
        assert kernel in ("cover", "fine")
        self.kernel = kernel
        self.n, self.K, self.dim, self.kT, self.project_on = n, K, dim, kT, project
        self.g = CompositeMAC(n, K, dim)
        self.fac = CompositeMACFAC(self.g, mu)
        self.coarse_sys = grid.velocity_system(n, dim, mu=mu, levels=1)
        self.fine_sys = grid.velocity_system(2 * n, dim, mu=mu, levels=1)
        self.R = self._restriction()
        self.E = self._extension()
        self.seed, self.instance, self.tol = seed, instance, tol
        self.xi = np.zeros(self.g.n_faces)     # persistent chain state
        self.cycle = 0                          # chain step counter (Philox counter words 2-3)

    @staticmethod
    def _offsets(system):
        return np.cumsum([0] + [cl.size for cl in system.levels[0]])

    def _comp_axes(self):
        return [0, 1, 2] if self.dim == 3 else [0, 2]

    def _restriction(self):
        g, d, K, n = self.g, self.dim, self.K, self.n
        F = g.face_of
        offs = self._offsets(self.coarse_sys)
        rows, cols, vals = [], [], []
        for c, axis in enumerate(self._comp_axes()):
            nz, ny, nx = self.coarse_sys.levels[0][c].shape
            for k in range(nz):
                for j in range(ny):
                    for i in range(nx):
                        row = offs[c] + (k * ny + j) * nx + i
                        kz = k + 1 if axis == 2 else k           # base row (w: node at kz H)
                        covered = kz < K
                        if not covered:
                            lev = "i" if axis == 2 and kz == K and 0 < K < n else "c"
                            rows.append(row)
                            cols.append(F[(axis, lev, kz, j, i)])
                            vals.append(1.0)
                            continue
                        kids = []
                        for e in (range(2) if d == 3 else [0]):
                            for t in range(2):
                                if axis == 0:
                                    key = (0, "f", 2 * kz + t, 2 * j + e if d == 3 else 0, 2 * i)
                                elif axis == 1:
                                    key = (1, "f", 2 * kz + t, 2 * j, 2 * i + e)
                                else:
                                    key = (2, "f", 2 * kz, 2 * j + e if d == 3 else 0, 2 * i + t)
                                kids.append(F[key])
                        for f in kids:
                            rows.append(row)
                            cols.append(f)
                            vals.append(1.0 / len(kids))
        return sp.csr_matrix((vals, (rows, cols)), shape=(offs[-1], g.n_faces))

    def _extension(self):
        g, d, K, n = self.g, self.dim, self.K, self.n
        F = g.face_of
        offs_f = self._offsets(self.fine_sys)
        offs_c = self._offsets(self.coarse_sys)
        rows, cols, vals = [], [], []
        ghost_rows, ghost_src = [], []
        for c, axis in enumerate(self._comp_axes()):
            kinds = self.coarse_sys.kinds[c]
            P1 = [grid.prolongation(kd, n if kd != "O" else 1) for kd in kinds]
            Pc = _kron3(P1[2], P1[1], P1[0]).tocsr()
            nz, ny, nx = self.fine_sys.levels[0][c].shape
            for k in range(nz):
                for j in range(ny):
                    for i in range(nx):
                        row = offs_f[c] + (k * ny + j) * nx + i
                        kz = k + 1 if axis == 2 else k
                        if kz < 2 * K:                                   # a slab unknown
                            rows.append(row)
                            cols.append(F[(axis, "f", kz, j, i)])
                            vals.append(1.0)
                        else:                                            # ghost: tri-linear from the base field
                            prow = Pc.getrow((k * ny + j) * nx + i)
                            for col, v in zip(prow.indices, prow.data):
                                ghost_rows.append(row)
                                ghost_src.append((offs_c[c] + col, v))
        E = sp.csr_matrix((vals, (rows, cols)), shape=(offs_f[-1], g.n_faces))
        if ghost_rows:
            Rr = sp.csr_matrix(([v for _, v in ghost_src], (ghost_rows, [s for s, _ in ghost_src])),
                               shape=(offs_f[-1], offs_c[-1]))
            E = E + Rr @ self.R
        return E.tocsr()

    def interpolation(self, X):
        """Gamma as a sparse (np d) x (faces) matrix."""
        rows, cols, vals = [], [], []
        cols_of = [0, 1, 2] if self.dim == 3 else [0, 1]
        for p_, x in enumerate(X):
            fine = self.kernel == "fine" or x[-1] < self.K * self.g.H
            system = self.fine_sys if fine else self.coarse_sys
            offs = self._offsets(system)
            lift = self.E if fine else self.R
            for c in range(system.ncomp):
                kk, jj, ii, W = coupling.stencil(system, c, x[None, :])
                nz, ny, nx = system.levels[0][c].shape
                idx = offs[c] + (kk.ravel() * ny + jj.ravel()) * nx + ii.ravel()
                w = W.ravel()
                keep = w != 0.0
                r = lift[idx[keep]].T @ w[keep]
                nzr = np.nonzero(r)[0]
                rows.extend([p_ * self.dim + cols_of[c]] * nzr.size)
                cols.extend(nzr.tolist())
                vals.extend(r[nzr].tolist())
        return sp.csr_matrix((vals, (rows, cols)), shape=(X.shape[0] * self.dim, self.g.n_faces))

    def _P(self, u):
        return self.g.project(u) if self.project_on else u

    def _PT(self, c):
        return self.g.weight * self.g.project(c / self.g.weight) if self.project_on else c

    def mobility_matrix(self, X, tol=1e-12):
        G = self.interpolation(X).toarray()
        M = np.zeros((G.shape[0], G.shape[0]))
        for col in range(G.shape[0]):
            u, cycles, rel = self.fac.solve(self._PT(G[col]), tol=tol)
            M[:, col] = G @ self._P(u)
        return M

    def thermal_operator(self, X):
        """K = sqrt(2 kT) Gamma P~ as a dense matrix (g = K xi); row r is P~^T of Gamma's row r."""
        G = self.interpolation(X).toarray()
        return np.sqrt(2.0 * self.kT) * np.array([self._PT(r) for r in G])

    # -- dynamics (Algorithm 4 on the composite grid) -----------------------
    def chain_cycles(self, ncycles):
        """Advance xi by ncycles stochastic FAC cycles with b = 0 (sigma = 1)."""
        from .philox import PhiloxNoise
        zero = np.zeros(self.g.n_faces)
        for _ in range(ncycles):
            self.fac.fac_cycle(self.xi, zero, PhiloxNoise(self.seed, self.instance, self.cycle), 1.0)
            self.cycle += 1
        return self.xi

    @staticmethod
    def wrap_reflect(X):
        X = X.copy()
        X[:, :-1] = np.mod(X[:, :-1], 1.0)
        z = X[:, -1]
        z = np.where(z < 0.0, -z, z)
        z = np.where(z > 1.0, 2.0 - z, z)
        X[:, -1] = z
        return X

    def em_step(self, X, F, dt, ncycles):
        """One Euler-Maruyama step (Algorithm 4): u = A^-1 P~^T Gamma^T F by FAC
        cycles to tol, the chain advanced by ncycles, then
        X <- X + Gamma P~ (dt u + sqrt(2 kT dt) xi), wrapped and reflected."""
        Gam = self.interpolation(X)
        rhs = self._PT(Gam.T @ F.ravel())
        u, cycles, rel = self.fac.solve(rhs, tol=self.tol)
        self.chain_cycles(ncycles)
        w = dt * u + np.sqrt(2.0 * self.kT * dt) * self.xi
        V = (Gam @ self._P(w)).reshape(X.shape)
        return self.wrap_reflect(X + V), cycles
