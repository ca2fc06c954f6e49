"""MAC lattices, separable 1-D factors and the Galerkin multigrid hierarchy.

Discretization (Section 4, Eq. equ_def_L, L = DG; Dirichlet / Neumann rules
for rectangular domains): the domain is the unit box, periodic in x (and y in
3-D) with no-slip walls at z = 0 and z = 1 ("z" is the wall axis; in 2-D the
paper's y axis is called z here and the y axis has one trivial node).

Each scalar unknown field ("component") is separable: along every axis it is
one of the 1-D lattice types

  'P'  periodic, n nodes
  'V'  wall-normal ("vertex") lattice: nodes at k h, k = 0..n, the two wall
       nodes are Dirichlet values (cell centres on the boundary, Section 4),
       unknowns are the n-1 interior nodes
  'C'  cell lattice between Dirichlet walls: n nodes at (k + 1/2) h; the
       ghost value beyond a wall is the odd reflection (reading R1)
  'N'  cell lattice with Neumann walls (pressure): ghost = even reflection
  'O'  trivial axis of a 2-D problem: one node, no coupling

Operator: with K_d the integer 1-D second-difference matrix of axis d and
M_d = I, the top-level operator is A = s * sum_d K_d (x) prod_{e != d} M_e,
i.e. A = mu h^d (-L_h) for the velocity (s = mu h^(d-2)), which is symmetric
positive definite (Section 2.1 requires L = L^T).

Multigrid transfers (Section 3.2): prolongation is the tensor product of 1-D
linear interpolation ("tri-linear", Eq. equ_restr_prolong_variation context);
restriction is its transpose; coarse operators are Galerkin,
A^(l) = P^T A^(l-1) P (variational property), which for a tensor-product P
keeps the separable form with K_d <- P_d^T K_d P_d and M_d <- P_d^T M_d P_d.
"""

import numpy as np
import scipy.sparse as sp

WALL_TYPES = ("V", "C", "N")


def lattice_size(kind, n):
    """Number of unknowns of a 1-D lattice with n cells."""
    if kind == "O":
        return 1
    if kind == "V":
        return n - 1
    return n


def node_positions(kind, n, length=1.0):
    """Physical coordinates of the unknowns of a 1-D lattice.

    'P' lattices are given by the caller's offset (see ``component_offsets``);
    here they are returned for offset 0.
    """
    h = length / n
    if kind == "V":
        return (np.arange(n - 1) + 1.0) * h
    if kind in ("C", "N"):
        return (np.arange(n) + 0.5) * h
    if kind == "P":
        return np.arange(n) * h
    return np.zeros(1)


def second_difference(kind, n):
    """Top-level 1-D factor K (integer second difference, h = 1 units)."""
    m = lattice_size(kind, n)
    if kind == "O":
        return np.zeros((1, 1))
    K = 2.0 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)
    if kind == "P":
        K[0, m - 1] -= 1.0
        K[m - 1, 0] -= 1.0
    elif kind == "C":  # ghost = -u: the wall-adjacent diagonal becomes 3
        K[0, 0] += 1.0
        K[m - 1, m - 1] += 1.0
    elif kind == "N":  # ghost = +u: the wall-adjacent diagonal becomes 1
        K[0, 0] -= 1.0
        K[m - 1, m - 1] -= 1.0
    return K


def prolongation(kind, nc):
    """1-D linear interpolation from a lattice of nc cells to one of 2 nc cells.

    'P': coarse node J sits on fine node 2J; odd fine nodes take the mean of
         their two coarse neighbours (periodic wrap).
    'V': same rule on interior nodes; the coarse wall nodes are 0.
    'C'/'N': coarse cell J (centre (2J+1) h_f) interpolates linearly to the
         fine cells 2J and 2J+1 (weights 3/4 near, 1/4 far); beyond a wall the
         coarse ghost is the odd ('C', reading R3) or even ('N') reflection.
    Returns the dense matrix P with shape (fine unknowns, coarse unknowns).
    """
    if kind == "O":
        return np.ones((1, 1))
    nf = 2 * nc
    mf, mc = lattice_size(kind, nf), lattice_size(kind, nc)
    P = np.zeros((mf, mc))
    if kind == "P":
        for J in range(nc):
            P[2 * J, J] += 1.0
            P[2 * J + 1, J] += 0.5
            P[2 * J + 1, (J + 1) % nc] += 0.5
    elif kind == "V":
        # fine unknown k is node k+1; coarse unknown J is coarse node J+1 = fine node 2J+2
        for k in range(mf):
            node = k + 1
            if node % 2 == 0:
                P[k, node // 2 - 1] += 1.0
            else:
                for cn in ((node - 1) // 2, (node + 1) // 2):
                    if 1 <= cn <= nc - 1:
                        P[k, cn - 1] += 0.5
    else:
        ghost = -1.0 if kind == "C" else 1.0
        for J in range(nc):
            for f, far in ((2 * J, J - 1), (2 * J + 1, J + 1)):
                P[f, J] += 0.75
                if 0 <= far < nc:
                    P[f, far] += 0.25
                else:  # reflection of coarse cell J across the wall
                    P[f, J] += 0.25 * ghost
    return P


def bandwidth(mat, periodic):
    """Largest |offset| (cyclic for periodic factors) with a non-zero entry."""
    m = mat.shape[0]
    bw = 0
    rows, cols = np.nonzero(mat)
    for r, c in zip(rows, cols):
        d = abs(int(c) - int(r))
        if periodic:
            d = min(d, m - d)
        bw = max(bw, d)
    return bw


class CompLevel:
    """One scalar component on one multigrid level (separable operator)."""

    def __init__(self, comp, level, kinds, ncells, K, M, scale, red_black=None):
        self.comp = comp            # component id (axis of the velocity it carries)
        self.level = level
        # red-black colouring (the 5/7-point top level); else colour moduli
        self.red_black = (level == 0) if red_black is None else bool(red_black)
        self.kinds = kinds          # (kind_x, kind_y, kind_z)
        self.ncells = ncells        # cells per axis at this level
        self.K = K                  # dense 1-D factors, axis order x, y, z
        self.M = M
        self.scale = scale
        self.shape = tuple(K[a].shape[0] for a in (2, 1, 0))   # array shape (nz, ny, nx)
        self.size = int(np.prod(self.shape))
        self._Ks = [sp.csr_matrix(k) for k in K]
        self._Ms = [sp.csr_matrix(m) for m in M]
        self._M_is_identity = [bool(np.array_equal(m, np.eye(m.shape[0]))) for m in M]
        self.bw = [bandwidth(K[a] + M[a], kinds[a] == "P") for a in range(3)]
        self._classes = None
        self._diag = None

    # -- operator -------------------------------------------------------
    @staticmethod
    def _apply_axis(mat, v, axis):
        """(mat applied along array axis `axis`) v, v of shape (nz, ny, nx)."""
        w = np.moveaxis(v, axis, 0)
        sh = w.shape
        out = mat @ w.reshape(sh[0], -1)
        return np.moveaxis(np.asarray(out).reshape((mat.shape[0],) + sh[1:]), 0, axis)

    def apply(self, v):
        """A v = s * sum_d K_d (x) prod_{e != d} M_e  v."""
        out = np.zeros_like(v)
        for d in range(3):
            t = v
            for a in range(3):
                if a != d and self._M_is_identity[a]:
                    continue                          # identity factor
                mat = self._Ks[a] if a == d else self._Ms[a]
                t = self._apply_axis(mat, t, 2 - a)   # axis a of space is array axis 2-a
            out += t
        return self.scale * out

    def diagonal(self):
        if self._diag is None:
            self._diag = self._diagonal()
        return self._diag

    def _diagonal(self):
        dk = [np.diag(k) for k in self.K]
        dm = [np.diag(m) for m in self.M]
        out = np.zeros(self.shape)
        for d in range(3):
            f = [dk[a] if a == d else dm[a] for a in range(3)]
            out += f[2][:, None, None] * f[1][None, :, None] * f[0][None, None, :]
        return self.scale * out

    def dense(self):
        """Assembled matrix in the flattening order of arrays (nz, ny, nx)."""
        K, M = self.K, self.M
        terms = [np.kron(M[2], np.kron(M[1], K[0])),
                 np.kron(M[2], np.kron(K[1], M[0])),
                 np.kron(K[2], np.kron(M[1], M[0]))]
        return self.scale * sum(terms)

    # -- colour classes for the Gibbs sweeps ------------------------------
    def colour_classes(self):
        if self._classes is None:
            self._classes = self._colour_classes()
        return self._classes

    def _colour_classes(self):
        """List of (colour id, index tuple) in visiting order, sites in rank order.

        Level 0 (or a level flagged red-black): colour = (i + j + k) mod 2,
        red (0) first; valid because the operator is the 5/7-point stencil
        (reading R2).
        Level >= 1: the Galerkin stencil couples offsets up to the factor
        bandwidths b_d, so colour = (i mod m_x, j mod m_y, k mod m_z) with
        m_d = b_d + 1 and colour id c_x + m_x (c_y + m_y c_z), visited in
        increasing id.  Within a class, sites are ranked row-major (x fastest).
        """
        nz, ny, nx = self.shape
        classes = []
        if self.red_black:
            assert nx % 2 == 0
            for c in (0, 1):
                k, j, m = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx // 2),
                                      indexing="ij")
                i = 2 * m + ((j + k + c) & 1)
                classes.append((c, (k.ravel(), j.ravel(), i.ravel())))
            return classes
        mods = self.moduli()
        mx, my, mz = mods
        for cz in range(mz):
            for cy in range(my):
                for cx in range(mx):
                    cid = cx + mx * (cy + my * cz)
                    kk = np.arange(cz, nz, mz)
                    jj = np.arange(cy, ny, my)
                    ii = np.arange(cx, nx, mx)
                    if kk.size == 0 or jj.size == 0 or ii.size == 0:
                        continue
                    k, j, i = np.meshgrid(kk, jj, ii, indexing="ij")
                    classes.append((cid, (k.ravel(), j.ravel(), i.ravel())))
        return classes

    def moduli(self):
        mods = []
        for a in range(3):
            n = self.K[a].shape[0]
            if n == 1:
                mods.append(1)
                continue
            m = self.bw[a] + 1
            if self.kinds[a] == "P":
                assert n % m == 0 and n > 2 * self.bw[a] or n == 2, \
                    "periodic axis too short for a valid colouring"
            mods.append(m)
        return tuple(mods)


class System:
    """A block-diagonal system of scalar components with a Galerkin hierarchy.

    kinds_per_comp : list of (kind_x, kind_y, kind_z) tuples
    comp_ids       : component ids (used in noise counters)
    n              : cells per axis at the finest level (same for every axis)
    dim            : 2 or 3
    scale          : s of the top-level operator
    levels         : number of multigrid levels (level 0 = finest)
    """

    def __init__(self, kinds_per_comp, comp_ids, n, dim, scale, levels):
        self.dim = dim
        self.n = n
        self.nlevels = levels
        self.comp_ids = list(comp_ids)
        self.kinds = [tuple(k) for k in kinds_per_comp]
        self.scale = scale
        self.levels = []       # levels[l][c] -> CompLevel
        self.P = []            # P[l][c] -> list of 1-D prolongations (level l+1 -> l)
        self._Psp = {}
        for c, kinds in enumerate(self.kinds):
            ncells = [n if k != "O" else 1 for k in kinds]
            K = [second_difference(k, nn) for k, nn in zip(kinds, ncells)]
            M = [np.eye(k_.shape[0]) for k_ in K]
            for l in range(levels):
                if len(self.levels) <= l:
                    self.levels.append([])
                    self.P.append([])
                self.levels[l].append(CompLevel(self.comp_ids[c], l, kinds, list(ncells),
                                                K, M, scale))
                if l == levels - 1:
                    break
                Ps = []
                for a in range(3):
                    if kinds[a] == "O":
                        Ps.append(np.ones((1, 1)))
                        continue
                    assert ncells[a] % 2 == 0, "cells per axis must be divisible by 2^(levels-1)"
                    Ps.append(prolongation(kinds[a], ncells[a] // 2))
                self.P[l].append(Ps)
                K = [Ps[a].T @ K[a] @ Ps[a] for a in range(3)]
                M = [Ps[a].T @ M[a] @ Ps[a] for a in range(3)]
                ncells = [nn // 2 if k != "O" else 1 for k, nn in zip(kinds, ncells)]

    @property
    def ncomp(self):
        return len(self.kinds)

    def shapes(self, level=0):
        return [cl.shape for cl in self.levels[level]]

    def zeros(self, level=0):
        return [np.zeros(s) for s in self.shapes(level)]

    def apply(self, level, v):
        return [cl.apply(x) for cl, x in zip(self.levels[level], v)]

    # -- transfers --------------------------------------------------------
    def _sparse_P(self, level, c, a, transpose):
        key = (level, c, a, transpose)
        if key not in self._Psp:
            m = self.P[level][c][a]
            self._Psp[key] = sp.csr_matrix(m.T if transpose else m)
        return self._Psp[key]

    def prolong(self, level, vc):
        """P vc: level+1 -> level (tensor product of the 1-D interpolations)."""
        out = []
        for c, x in enumerate(vc):
            t = x
            for a in range(3):
                t = CompLevel._apply_axis(self._sparse_P(level, c, a, False), t, 2 - a)
            out.append(t)
        return out

    def restrict(self, level, r):
        """P^T r: level -> level+1 (adjoint of prolongation, Eq. equ_restr_prolong_variation)."""
        out = []
        for c, x in enumerate(r):
            t = x
            for a in range(3):
                t = CompLevel._apply_axis(self._sparse_P(level, c, a, True), t, 2 - a)
            out.append(t)
        return out


def default_levels(n, dim):
    """Coarsen while the edge stays even and at least 4 after halving (reading R8)."""
    levels = 1
    m = n
    while m % 2 == 0 and m // 2 >= 4:
        m //= 2
        levels += 1
    return levels


def velocity_system(n, dim, mu=1.0, levels=None):
    """MAC velocity components; their ids are the axes of their face normals."""
    h = 1.0 / n
    if levels is None:
        levels = default_levels(n, dim)
    if dim == 3:
        kinds = [("P", "P", "C"), ("P", "P", "C"), ("P", "P", "V")]
        ids = [0, 1, 2]
    else:
        kinds = [("P", "O", "C"), ("P", "O", "V")]
        ids = [0, 2]
    return System(kinds, ids, n, dim, mu * h ** (dim - 2), levels)


def pressure_system(n, dim, levels=None):
    """Cell-centred pressure with Neumann walls: A_p = D^ D^T (integer form)."""
    if levels is None:
        levels = default_levels(n, dim)
    kinds = [("P", "P", "N")] if dim == 3 else [("P", "O", "N")]
    return System(kinds, [3], n, dim, 1.0, levels)


def component_offsets(comp, dim):
    """Offsets (in cells) of a velocity component's lattice along x, y, z.

    The component normal to axis a lives on faces normal to a: offset 0 along
    a and 1/2 along the other axes.  For the wall axis the 'V' lattice is
    described by ``node_positions`` (unknown k at (k+1) h).
    """
    off = [0.5, 0.5, 0.5]
    off[comp] = 0.0
    if dim == 2:
        off[1] = 0.0
    return off
