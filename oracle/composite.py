"""Composite-grid FAC (Algorithms 1 and 2) for one refined patch: oracle.

Test infrastructure (plain FP64 numpy/scipy, follows the paper step by step):
only tests and the benchmark's CPU baseline call it.

Geometry (readings R14, R15 and R17 of the design notes):

* Base grid: n cells along each periodic axis (x, and y in 3-D), H = 1/n.
  The wall axis z has its cell centres on the walls (Section 4: Dirichlet
  conditions put partition-cell centres on the boundary): nodes j = 0..n at
  z = jH, the wall nodes j = 0 and j = n are Dirichlet zeros, the unknowns are
  the rows j = 1..n-1 (array row r = j - 1).  One scalar field per component
  (cell-centred, no projection; the paper's adaptive discretization of the
  Laplacian in Section 4).
* Patch: the base rows j = 1..K over the whole periodic x-y extent are refined
  by 2 in every direction: fine cells (m, q, p), p, q in [0, 2n), m in
  [0, 2K), of width h = H/2, centred at z = (2m + 3) H / 4.  Base row j covers
  fine layers m = 2(j - 1) and 2(j - 1) + 1.  The covered base cells are not
  composite unknowns; the uncovered base rows j = K+1..n-1 are.
* The base wall cell j = 0 (centre on the wall, value 0) borders the patch's
  bottom layer across the face z = H/2, and the uncovered base row j = K+1
  borders its top layer across z = (K + 1/2) H.  Both are coarse-fine faces.

Operator (Section 4, Eqs. equ_def_discr_div to equ_def_L, L = DG, and the
symmetric form A = -mu V L of reading R16): the divergence is the
face-area-weighted flux sum over a cell's faces divided by its volume; the
gradient across a face between equal cells is the difference over the
spacing; across a coarse-fine face it is (mean of the 2^(d-1) fine values -
coarse value) over (3/4) H on every fine face, and the coarse face carries the
mean of the fine-face values (Eqs. equ_def_discr_grad to
equ_def_discr_grad_last, with the four fine neighbours B, C, D, E in 3-D,
reading R16).  Then A = -mu V L is the quadratic form
    c^T A c = mu * sum over faces  w_f * (delta_f c)^2
with w = h^(d-2) (delta = difference) on a face between two fine cells,
w = H^(d-2) between two base cells (and at the top wall, delta = c), and
w = (4/3) H^(d-2), delta = c_coarse - mean(c_fine), for each coarse-fine group
(the wall group has c_coarse = 0).  It is symmetric by construction and
positive definite.

FAC (Algorithm 1 around Algorithm 2, readings R6, R25, R17):
    r   = b - A z                                  (composite residual)
    r_b = P^T r                                    (restriction to the base)
    q_b = V-Cycle(0, r_b) on the base hierarchy    (Algorithm 3; level 1 = base)
    q   = P q_b                                    (prolongation into the patch)
    nu  Gibbs sweeps on the patch cells of A q = r (composite rows)
    z  += q
P (base -> composite) is the identity on uncovered base cells and gives each
fine cell its parent's value (piecewise constant, reading R17); the base
operator is the Galerkin product A_b = P^T A P, which is the 7-point operator
with z-dependent weights built in ``base_factors`` (pinned against the triple
product).  The base hierarchy below is the usual Galerkin hierarchy with
tri-linear transfers.  Level numbering: 0 = patch, 1 = base, 2.. = coarser.

Patch sweep order (reading R18): the patch rows of A couple a fine cell to
its 2^(d-1) siblings across a coarse-fine face, so a red-black order is not a
valid Gibbs order on the two interface layers (m = 0 and m = 2K-1).  A sweep
is four passes: red sites except the interface-layer sites with odd p, then
those, then the same for black (red = (p + q + m) even).  Noise: counter
stream kind 2; a patch row (m, q) is cut into segments of 8 cells along x,
and the four cells of one colour in a segment share one Philox block:
group = (m n_y + q) ceil(n_x / 8) + p // 8, lane = (p mod 8) // 2 (the two
cells of a lane have opposite colours, so they never share a pass).
"""

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import grid, multigrid, gibbs


class CompositeGrid:
    """Base grid + refined bottom patch for `ncomp` scalar components."""

    def __init__(self, n, K, dim, mu=1.0, ncomp=1, levels=None):
        assert dim in (2, 3) and n % 2 == 0 and 1 <= K <= n - 2
        self.n, self.K, self.dim, self.mu = n, K, dim, float(mu)
        self.ncomp = ncomp
        self.comp_ids = list(range(ncomp))
        self.H = 1.0 / n
        self.h = self.H / 2.0
        ny_b = n if dim == 3 else 1
        self.base_shape = (n - 1, ny_b, n)
        self.fine_shape = (2 * K, 2 * n if dim == 3 else 1, 2 * n)
        self.n_fine = int(np.prod(self.fine_shape))
        self.n_unc = (n - 1 - K) * ny_b * n           # uncovered base unknowns
        self.size = self.n_fine + self.n_unc
        self.A = self._assemble()
        self.P = self._prolongation()
        self.diag = self.A.diagonal()
        self.base = BaseHierarchy(self, levels)

    # -- indexing ----------------------------------------------------------
    def fine_index(self, m, q, p):
        nz, ny, nx = self.fine_shape
        return (m * ny + q) * nx + p

    def base_index(self, r, l, i):
        """Composite index of an uncovered base cell (row r >= K)."""
        _, ny, nx = self.base_shape
        return self.n_fine + ((r - self.K) * ny + l) * nx + i

    def to_vec(self, fine, base):
        return np.concatenate([fine.ravel(), base[self.K:].ravel()])

    def from_vec(self, vec):
        fine = vec[:self.n_fine].reshape(self.fine_shape).copy()
        base = np.zeros(self.base_shape)
        base[self.K:] = vec[self.n_fine:].reshape((self.base_shape[0] - self.K,) + self.base_shape[1:])
        return fine, base

    # -- operator ----------------------------------------------------------
    def _assemble(self):
        d, n, K = self.dim, self.n, self.K
        wf = self.mu * self.h ** (d - 2)
        wb = self.mu * self.H ** (d - 2)
        wcf = self.mu * (4.0 / 3.0) * self.H ** (d - 2)
        rows, cols, vals = [], [], []

        def face(w, a, b):
            a = np.asarray(a).ravel()
            b = np.asarray(b).ravel()
            for i_, j_, v_ in ((a, a, w), (b, b, w), (a, b, -w), (b, a, -w)):
                rows.append(i_)
                cols.append(j_)
                vals.append(np.full(i_.size, v_))

        def wall(w, a):
            a = np.asarray(a).ravel()
            rows.append(a)
            cols.append(a)
            vals.append(np.full(a.size, w))

        def group(w, coarse, children):
            """w (c_coarse - mean(children))^2; coarse None = wall (value 0)."""
            nch = len(children)
            g_idx = ([] if coarse is None else [np.asarray(coarse).ravel()]) + \
                    [np.asarray(c).ravel() for c in children]
            g_val = ([] if coarse is None else [1.0]) + [-1.0 / nch] * nch
            for a, va in zip(g_idx, g_val):
                for b, vb in zip(g_idx, g_val):
                    rows.append(a)
                    cols.append(b)
                    vals.append(np.full(a.size, w * va * vb))

        fz, fy, fx = self.fine_shape
        m, q, p = np.meshgrid(np.arange(fz), np.arange(fy), np.arange(fx), indexing="ij")
        F = self.fine_index(m, q, p)
        face(wf, F, self.fine_index(m, q, (p + 1) % fx))                  # x faces (periodic)
        if d == 3:
            face(wf, F, self.fine_index(m, (q + 1) % fy, p))              # y faces
        face(wf, F[:-1], F[1:])                                           # z faces inside the patch
        bz, by, bx = self.base_shape
        r, l, i = np.meshgrid(np.arange(K, bz), np.arange(by), np.arange(bx), indexing="ij")
        B = self.base_index(r, l, i)
        face(wb, B, self.base_index(r, l, (i + 1) % bx))
        if d == 3:
            face(wb, B, self.base_index(r, (l + 1) % by, i))
        face(wb, B[:-1], B[1:])                                           # z faces between base rows
        wall(wb, B[-1])                                                   # top wall
        # coarse-fine groups: children of base (l, i) in the top / bottom fine layer
        l2, i2 = np.meshgrid(np.arange(by), np.arange(bx), indexing="ij")
        offs = [(0, 0), (0, 1)] if d == 2 else [(0, 0), (0, 1), (1, 0), (1, 1)]
        for mlayer, coarse in ((2 * K - 1, self.base_index(K, l2, i2)), (0, None)):
            children = [self.fine_index(mlayer, (2 * l2 + dq) if d == 3 else 0 * l2, 2 * i2 + dp)
                        for dq, dp in offs]
            group(wcf, coarse, children)
        A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.size, self.size))
        A.sum_duplicates()
        return A

    def apply(self, vec):
        return self.A @ vec

    # -- transfers -----------------------------------------------------------
    def _prolongation(self):
        """P: base field (all rows, flattened) -> composite vector (reading R17)."""
        bz, by, bx = self.base_shape
        nb = bz * by * bx
        fz, fy, fx = self.fine_shape
        m, q, p = np.meshgrid(np.arange(fz), np.arange(fy), np.arange(fx), indexing="ij")
        parent = ((m >> 1) * by + (q >> 1)) * bx + (p >> 1)
        rows = [self.fine_index(m, q, p).ravel()]
        cols = [parent.ravel()]
        r, l, i = np.meshgrid(np.arange(self.K, bz), np.arange(by), np.arange(bx), indexing="ij")
        rows.append(self.base_index(r, l, i).ravel())
        cols.append(((r * by + l) * bx + i).ravel())
        rr = np.concatenate(rows)
        return sp.csr_matrix((np.ones(rr.size), (rr, np.concatenate(cols))), shape=(self.size, nb))

    def prolong(self, base):
        return self.P @ base.ravel()

    def restrict(self, vec):
        return (self.P.T @ vec).reshape(self.base_shape)

    # -- patch sweeps ---------------------------------------------------------
    def pass_sets(self):
        """Linear fine indices of the four passes of a patch sweep (reading R18)."""
        fz, fy, fx = self.fine_shape
        m, q, p = np.meshgrid(np.arange(fz), np.arange(fy), np.arange(fx), indexing="ij")
        red = ((m + q + p) & 1) == 0
        iface = (m == 0) | (m == fz - 1)
        late = iface & ((p & 1) == 1)
        sets = []
        for colour in (red, ~red):
            sets.append(np.nonzero((colour & ~late).ravel())[0])
            sets.append(np.nonzero((colour & late).ravel())[0])
        return sets

    def noise_index(self, idx):
        """Counter index of patch cells (linear indices idx): 4 group + lane."""
        fz, fy, fx = self.fine_shape
        row, p = idx // fx, idx % fx
        nseg = (fx + 7) // 8
        return 4 * (row * nseg + p // 8) + (p % 8) // 2

    def patch_sweep(self, qvec, rvec, comp, sweep_id, noise, sigma):
        """One Gibbs sweep of the patch cells of A q = r (composite rows), in place."""
        for pid, idx in enumerate(self.pass_sets()):
            Aq = self.A[idx] @ qvec
            dg = self.diag[idx]
            new = (rvec[idx] - (Aq - dg * qvec[idx])) / dg
            if sigma != 0.0:
                nrm = noise.patch(comp, pid, sweep_id, self.noise_index(idx))
                new = new + sigma * nrm / np.sqrt(dg)
            qvec[idx] = new
        return qvec


def base_factors(cg):
    """1-D factors of the Galerkin base operator A_b = P^T A P (unit mu H^(d-2)).

    x, y: the periodic second difference with unit mass.  z (rows r = j - 1):
    face weights between node f and f+1 are 4/3 at the bottom wall (the wall
    group), 2 between two covered rows, 4/3 across the interface, 1 between
    uncovered rows and at the top wall; the x-y mass is 2 on covered rows and
    1 on uncovered rows (2^(d-1) fine faces of weight h^(d-2) make one base
    face of weight 2 H^(d-2)).
    """
    n, K = cg.n, cg.K
    wz = np.ones(n)                     # face f between node f and f+1, f = 0..n-1
    wz[0] = 4.0 / 3.0
    wz[1:K] = 2.0
    wz[K] = 4.0 / 3.0
    Kz = np.zeros((n - 1, n - 1))
    for r in range(n - 1):
        Kz[r, r] = wz[r] + wz[r + 1]
        if r + 1 < n - 1:
            Kz[r, r + 1] = Kz[r + 1, r] = -wz[r + 1]
    Mz = np.diag(np.where(np.arange(n - 1) < K, 2.0, 1.0))
    Kx = grid.second_difference("P", n)
    if cg.dim == 3:
        Ky = grid.second_difference("P", n)
        My = np.eye(n)
    else:
        Ky = np.zeros((1, 1))
        My = np.ones((1, 1))
    return [Kx, Ky, Kz], [np.eye(n), My, Mz]


class BaseHierarchy(grid.System):
    """Galerkin hierarchy below the patch: level 1 = base grid, 2.. coarser.

    Level 1 is red-black (its operator is 7-point); coarser levels use the
    colour-modulus rule.  Index 0 of ``levels`` is the patch and is not used
    by the V-cycle.
    """

    def __init__(self, cg, levels=None):
        n, dim = cg.n, cg.dim
        self.dim = dim
        self.n = n
        nb = grid.default_levels(n, dim) if levels is None else levels
        self.nlevels = nb + 1
        self.comp_ids = list(cg.comp_ids)
        kinds = ("P", "P", "V") if dim == 3 else ("P", "O", "V")
        self.kinds = [kinds] * cg.ncomp
        self.scale = cg.mu * cg.H ** (dim - 2)
        self.levels = [[None] * cg.ncomp]
        self.P = [[None] * cg.ncomp]
        self._Psp = {}
        K0, M0 = base_factors(cg)
        for l in range(1, self.nlevels):
            self.levels.append([])
            self.P.append([])
        for c in range(cg.ncomp):
            K, M = [k.copy() for k in K0], [m.copy() for m in M0]
            ncells = [n, n if dim == 3 else 1, n]
            for l in range(1, self.nlevels):
                self.levels[l].append(grid.CompLevel(self.comp_ids[c], l, kinds, list(ncells), K, M, self.scale,
                                                     red_black=(l == 1)))
                if l == self.nlevels - 1:
                    break
                Ps = []
                for a in range(3):
                    if kinds[a] == "O":
                        Ps.append(np.ones((1, 1)))
                        continue
                    assert ncells[a] % 2 == 0, "cells per axis must be divisible by 2^(levels-1)"
                    Ps.append(grid.prolongation(kinds[a], ncells[a] // 2))
                self.P[l].append(Ps)
                K = [Ps[a].T @ K[a] @ Ps[a] for a in range(3)]
                M = [Ps[a].T @ M[a] @ Ps[a] for a in range(3)]
                ncells = [nn // 2 if k != "O" else 1 for k, nn in zip(kinds, ncells)]


def residual(cg, z, b):
    """Composite residual r = b - A z per component (vectors)."""
    return [bb - cg.apply(zz) for zz, bb in zip(z, b)]


def fac_cycle(cg, z, b, noise, sigma, mu1=2, mu2=2, nu=2, coarse_mode="cholesky", coarsest=None):
    """One composite FAC iteration (Algorithm 1 with Algorithm 2), in place.

    z, b: lists (one per component) of composite vectors.
    """
    r = residual(cg, z, b)
    rb = [cg.restrict(x) for x in r]                                   # Alg. 2 step 2
    qb = cg.base.zeros(1)
    multigrid.vcycle(cg.base, 1, qb, rb, noise, sigma, mu1, mu2, coarse_mode, coarsest)  # step 3
    for c in range(cg.ncomp):
        q = cg.prolong(qb[c])                                          # step 4 (reading R25)
        for s in range(nu):                                            # step 5
            cg.patch_sweep(q, r[c], cg.comp_ids[c], s, noise, sigma)
        z[c] += q                                                      # Alg. 1 step 4
    return z


def solve(cg, b, tol=1e-10, max_cycles=200, v0=None, mu1=2, mu2=2, nu=2, coarse_mode="cholesky"):
    """Deterministic composite FAC until ||b - A z|| <= tol ||b|| (reading R9)."""
    from .philox import ExplicitNoise
    coarsest = multigrid.Coarsest(cg.base) if coarse_mode == "cholesky" else None
    z = [np.zeros(cg.size) for _ in range(cg.ncomp)] if v0 is None else [x.copy() for x in v0]
    bn = multigrid.norm(b)
    if bn == 0.0:
        return z, 0, 0.0
    cycles = 0
    rel = multigrid.norm(residual(cg, z, b)) / bn
    while rel > tol and cycles < max_cycles:
        fac_cycle(cg, z, b, ExplicitNoise(), 0.0, mu1, mu2, nu, coarse_mode, coarsest)
        cycles += 1
        rel = multigrid.norm(residual(cg, z, b)) / bn
    return z, cycles, rel


def direct_solve(cg, b):
    """Sparse direct solve of A z = b (for pins)."""
    return [spla.spsolve(cg.A.tocsc(), x) for x in b]


def cell_centres_z(cg):
    """z coordinate of every composite unknown (fine cells, then uncovered base)."""
    fz, fy, fx = cg.fine_shape
    zf = np.broadcast_to(((2 * np.arange(fz) + 3) * cg.H / 4.0)[:, None, None], cg.fine_shape)
    bz, by, bx = cg.base_shape
    zb = np.broadcast_to(((np.arange(cg.K, bz) + 1) * cg.H)[:, None, None], (bz - cg.K, by, bx))
    return np.concatenate([zf.ravel(), zb.ravel()])
