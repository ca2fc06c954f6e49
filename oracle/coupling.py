"""Fluid-structure coupling: interpolation Gamma and spreading Gamma^T.

Section 2.1 requires coupling operators with Lambda = alpha Gamma^T; the paper
points to the immersed boundary method (Peskin, Acta Numerica 2002) for a
realisation but does not print the kernel.  This is the Peskin 4-point
function from that reference:

    phi(r) = (3 - 2|r| + sqrt(1 + 4|r| - 4 r^2)) / 8     for |r| <= 1
           = (5 - 2|r| - sqrt(-7 + 12|r| - 4 r^2)) / 8    for 1 <= |r| <= 2
           = 0                                            otherwise

Gamma interpolates each velocity component at a particle from the 4^d nodes
of that component's staggered lattice with weights prod_d phi((X_d - x_d)/h)
(Eq. equ_dX_dt_Gamma, U = Gamma u).  Weights that fall on nodes that are not
unknowns (wall nodes or beyond the walls) are dropped in both Gamma and
Gamma^T (reading R11), which keeps the two exactly adjoint.  With A scaled by
h^d, spreading with Gamma^T is the force density Lambda F = h^-d Gamma^T F
multiplied by h^d (alpha = h^-d).
"""

import numpy as np

from .grid import component_offsets


def peskin_phi(r):
    r = np.abs(np.asarray(r, dtype=np.float64))
    out = np.zeros_like(r)
    m1 = r <= 1.0
    m2 = (r > 1.0) & (r <= 2.0)
    out[m1] = (3.0 - 2.0 * r[m1] + np.sqrt(1.0 + 4.0 * r[m1] - 4.0 * r[m1] ** 2)) / 8.0
    r2 = r[m2]
    out[m2] = (5.0 - 2.0 * r2 - np.sqrt(np.maximum(-7.0 + 12.0 * r2 - 4.0 * r2 ** 2, 0.0))) / 8.0
    return out


def _axis_nodes(x, kind, offset, n):
    """Indices (np, 4), weights (np, 4) and validity (np, 4) along one axis.

    x: particle coordinates in units of h.
    """
    if kind == "O":
        idx = np.zeros((x.shape[0], 4), dtype=np.int64)
        w = np.zeros((x.shape[0], 4))
        w[:, 0] = 1.0
        return idx, w, w > 0
    if kind == "V":
        off = 0.0      # node m at m h; unknown index m - 1
    elif kind in ("C", "N"):
        off = 0.5
    else:
        off = offset
    base = np.floor(x - off).astype(np.int64) - 1
    a = base[:, None] + np.arange(4)[None, :]
    w = peskin_phi(x[:, None] - off - a)
    if kind == "P":
        return np.mod(a, n), w, np.ones_like(w, dtype=bool)
    if kind == "V":
        valid = (a >= 1) & (a <= n - 1)
        return np.where(valid, a - 1, 0), w, valid
    valid = (a >= 0) & (a <= n - 1)
    return np.where(valid, a, 0), w, valid


def stencil(system, comp_index, X):
    """Per-particle node indices and tensor weights for one component.

    Returns (kk, jj, ii, W): arrays of shape (np, 4, 4, 4) (unused axes of a
    2-D problem have weight 1 at slot 0 only); invalid nodes get weight 0.
    """
    cl = system.levels[0][comp_index]
    n = system.n
    dim = system.dim
    comp = cl.comp
    offs = component_offsets(comp, dim)
    cols = [0, 1, 2] if dim == 3 else [0, None, 1]
    per_axis = []
    for a in range(3):
        if cl.kinds[a] == "O":
            per_axis.append(_axis_nodes(np.zeros(X.shape[0]), "O", 0.0, 1))
        else:
            per_axis.append(_axis_nodes(X[:, cols[a]] * n, cl.kinds[a], offs[a], n))
    (ix, wx, vx), (iy, wy, vy), (iz, wz, vz) = per_axis
    wx = np.where(vx, wx, 0.0)
    wy = np.where(vy, wy, 0.0)
    wz = np.where(vz, wz, 0.0)
    W = wz[:, :, None, None] * wy[:, None, :, None] * wx[:, None, None, :]
    kk = np.broadcast_to(iz[:, :, None, None], W.shape)
    jj = np.broadcast_to(iy[:, None, :, None], W.shape)
    ii = np.broadcast_to(ix[:, None, None, :], W.shape)
    return kk, jj, ii, W


def particle_columns(dim):
    return [0, 1, 2] if dim == 3 else [0, 1]


def interpolate(system, u, X):
    """U = Gamma u: (np, dim) velocities of the particles."""
    U = np.zeros((X.shape[0], system.dim))
    for c in range(system.ncomp):
        kk, jj, ii, W = stencil(system, c, X)
        vals = u[c][kk, jj, ii]
        U[:, particle_columns(system.dim)[c]] = np.sum(W * vals, axis=(1, 2, 3))
    return U


def spread(system, F, X):
    """b = Gamma^T F: one field per component."""
    b = system.zeros(0)
    for c in range(system.ncomp):
        kk, jj, ii, W = stencil(system, c, X)
        f = F[:, particle_columns(system.dim)[c]]
        np.add.at(b[c], (kk.ravel(), jj.ravel(), ii.ravel()),
                  (W * f[:, None, None, None]).ravel())
    return b
