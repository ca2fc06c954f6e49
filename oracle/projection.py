"""Discrete divergence, gradient and projection on the MAC grid (Section 4).

Divergence (Eq. equ_def_discr_div): the cell-centred sum of outward normal
face values divided by the cell width.  Gradient at a face between two cells
of the same level (Eq. equ_def_discr_grad0): difference of the two cell
values divided by the width.  With D^ = h D (integer differences) the
gradient restricted to the unknown faces is G = -D^T / h (no value is defined
on wall faces, which carry Dirichlet velocity), so the Neumann pressure
operator is D G = -D^ D^T / h^2 (Eq. equ_def_L, L = DG, Neumann rule).

Projection (Section 2.1 wants P~ = P~^T): P~ = I - G (D G)^+ D
= I - D^T (D^ D^T)^+ D^, the orthogonal projection onto discretely
divergence-free fields.  The pressure Poisson problem is solved by the
deterministic FAC iteration of ``multigrid`` on the 'N' system.
"""

import numpy as np

from . import grid, multigrid


def divergence(w, dim):
    """D^ w (integer-difference divergence), shape (nz, ny, nx) of cells."""
    if dim == 3:
        u, v, ww = w
    else:
        u, ww = w
        v = None
    nz = u.shape[0]
    out = np.roll(u, -1, axis=2) - u
    if v is not None:
        out = out + (np.roll(v, -1, axis=1) - v)
    # wall-normal faces: unknown k is the face between cells k and k+1
    top = np.zeros_like(out)
    top[:nz - 1] = ww
    bottom = np.zeros_like(out)
    bottom[1:] = ww
    return out + top - bottom


def divergence_transpose(phi, dim):
    """D^T phi on the velocity unknowns (the negative scaled gradient)."""
    gx = np.roll(phi, 1, axis=2) - phi                 # face i: phi[i-1] - phi[i]
    gz = phi[:-1] - phi[1:]                             # face k+1: phi[k] - phi[k+1]
    if dim == 3:
        gy = np.roll(phi, 1, axis=1) - phi
        return [gx, gy, gz]
    return [gx, gz]


class Projector:
    """P~ w with the pressure solved by the FAC iteration (Algorithm 1).

    Algorithm 1 starts from a given initial value.  ``slot=None`` starts from
    zero; an integer slot starts from the pressure that slot produced last
    time (a warm start for repeated projections of slowly changing fields)."""

    def __init__(self, n, dim, tol=1e-12, levels=None):
        self.dim = dim
        self.psys = grid.pressure_system(n, dim, levels)
        self.coarsest = multigrid.Coarsest(self.psys)
        self.tol = tol
        self.warm = {}

    def pressure(self, w, slot=None):
        div = divergence(w, self.dim)
        # D^ w sums to zero exactly (flux form); removing the rounding-level
        # mean keeps the singular Neumann system consistent.
        rhs = [div - np.mean(div)]
        v0 = None if slot is None or slot not in self.warm else [self.warm[slot]]
        phi, cycles, rel = multigrid.solve(self.psys, rhs, tol=self.tol, max_cycles=200,
                                           coarsest=self.coarsest, v0=v0)
        if slot is not None:
            self.warm[slot] = phi[0].copy()
        return phi[0], cycles

    def project(self, w, slot=None):
        phi, _ = self.pressure(w, slot)
        g = divergence_transpose(phi, self.dim)
        return [a - b for a, b in zip(w, g)]
