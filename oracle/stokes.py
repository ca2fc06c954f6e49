"""Exact discrete Stokes mobility near walls and the Ito drift kT div_X M.

TEST INFRASTRUCTURE ONLY (see the package header).  Two corrections to the
paper's effective dynamics (reading R28), written from their definitions:

1. Stokes mobility.  Section 2.1 forms the mobility as
   M = Gamma P~ A^-1 P~ Gamma^T, the discrete Stokes mobility only when P~
   commutes with A.  Next to no-slip walls it does not (reading R13).  The
   steady discrete Stokes problem on the MAC grid is the saddle point

       A u + D^T p = f,    D u = 0          (D the integer MAC divergence),

   whose velocity is u = S f, S = Z (Z^T A Z)^-1 Z^T for any basis Z of
   ker D.  S is symmetric positive semidefinite, S A S = S, and
   P~ A^-1 P~ - S is positive semidefinite (both are the maximisers of
   2 f^T u - u^T A u, S over the smaller set ker D).  Thermal velocities with
   covariance 2 kT Gamma S Gamma^T follow from the chain xi ~ N(0, A^-1):
   Cov(S A xi) = S A A^-1 A S = S.

2. Ito drift.  M depends on the positions (walls, lattice), so the Ito form of
   the overdamped dynamics carries kT div_X M, which reading R12 leaves out.
   The random finite difference
       d = (kT / delta) [M(X + delta W / 2) - M(X - delta W / 2)] W
   has E_W d = kT div_X M + O(delta^2) for W ~ N(0, I).

The Euler-Maruyama step with both corrections (Algorithm 4 with S in place of
P~ A^-1 P~):
    X <- X + Gamma S (dt Gamma^T F + sqrt(2 kT dt) A xi) + dt d,
with xi the persistent chain after its cycles of the step and d the drift at
the step's start positions.
"""

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import coupling, grid, multigrid, projection
from .philox import PhiloxNoise, make_key, normals_for_ranks, pack_ctr1

KIND_RFD = 3   # Philox counter kind of the random-finite-difference directions


def velocity_matrix(system):
    """A of the velocity system's level 0 as a sparse block-diagonal matrix."""
    return sp.block_diag([sp.csr_matrix(cl.dense()) for cl in system.levels[0]]).tocsr()


def divergence_matrix(n, dim):
    """D (integer MAC divergence, cells x velocity unknowns), column by column."""
    system = grid.velocity_system(n, dim, levels=1)
    shapes = system.shapes(0)
    sizes = [int(np.prod(s)) for s in shapes]
    cols = []
    for c, (shape, size) in enumerate(zip(shapes, sizes)):
        for q in range(size):
            w = [np.zeros(s) for s in shapes]
            w[c].flat[q] = 1.0
            cols.append(sp.csr_matrix(projection.divergence(w, dim).ravel()).T)
    return sp.hstack(cols).tocsr()


class StokesSolver:
    """u = S f by a sparse direct solve of the saddle point, pressure of cell 0
    pinned to zero (the constants are the kernel of D^T)."""

    def __init__(self, n, dim, mu=1.0):
        self.n, self.dim = n, dim
        self.system = grid.velocity_system(n, dim, mu=mu, levels=1)
        self.A = velocity_matrix(self.system)
        self.D = divergence_matrix(n, dim)
        nv, nc = self.A.shape[0], self.D.shape[0]
        K = sp.bmat([[self.A, self.D.T], [self.D, None]]).tocsc()
        keep = np.r_[0:nv, nv + 1:nv + nc]
        self.nv, self.nc = nv, nc
        self._keep = keep
        self._lu = spla.splu(K[keep][:, keep].tocsc())

    def solve(self, f):
        """(u, p) for a flat velocity right-hand side f (p has zero mean)."""
        rhs = np.zeros(self._keep.size)
        rhs[:self.nv] = f
        x = self._lu.solve(rhs)
        u = x[:self.nv]
        p = np.concatenate([[0.0], x[self.nv:]])
        return u, p - p.mean()


def _flat(fields):
    return np.concatenate([f.ravel() for f in fields])


def _fields(system, vec):
    out, o = [], 0
    for s in system.shapes(0):
        k = int(np.prod(s))
        out.append(vec[o:o + k].reshape(s))
        o += k
    return out


def rfd_directions(seed, instance, step, npart, dim):
    """W ~ N(0, I) of one step's drift estimate, [npart][dim] (Philox kind 3,
    rank = p dim + axis, counter words 2-3 = the step index)."""
    c1 = pack_ctr1(0, 0, 0, 0, KIND_RFD)
    return normals_for_ranks(make_key(seed, instance), c1, step, npart * dim).reshape(npart, dim)


class StokesModel:
    """Particles with the exact Stokes mobility and the Ito drift (FP64)."""

    def __init__(self, n, dim, mu=1.0, kT=1.0, seed=0, instance=0, tol=1e-12, delta=1e-4, drift=True):
        self.n, self.dim, self.kT = n, dim, kT
        self.stokes = StokesSolver(n, dim, mu)
        self.sys = self.stokes.system
        self.chain_sys = grid.velocity_system(n, dim, mu=mu)
        self.coarsest = multigrid.Coarsest(self.chain_sys)
        self.seed, self.instance, self.tol = seed, instance, tol
        self.delta, self.drift_on = delta, drift
        self.xi = self.chain_sys.zeros(0)
        self.cycle = 0
        self.step_count = 0

    def S(self, f):
        return self.stokes.solve(f)[0]

    def mobility_apply(self, X, F):
        f = _flat(coupling.spread(self.sys, F, X))
        return coupling.interpolate(self.sys, _fields(self.sys, self.S(f)), X)

    def mobility_matrix(self, X):
        npart, dim = X.shape
        M = np.zeros((npart * dim, npart * dim))
        for col in range(npart * dim):
            F = np.zeros((npart, dim))
            F[col // dim, col % dim] = 1.0
            M[:, col] = self.mobility_apply(X, F).ravel()
        return M

    def rfd_drift(self, X, W):
        """(kT / delta) [M(X + delta W/2) - M(X - delta W/2)] W."""
        h = 0.5 * self.delta
        up = self.mobility_apply(X + h * W, W)
        dn = self.mobility_apply(X - h * W, W)
        return self.kT / self.delta * (up - dn)

    def chain_cycles(self, ncycles):
        zero = self.chain_sys.zeros(0)
        for _ in range(ncycles):
            noise = PhiloxNoise(self.seed, self.instance, self.cycle)
            multigrid.fac_cycle(self.chain_sys, self.xi, zero, noise, 1.0, coarsest=self.coarsest)
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
        d = np.zeros_like(X)
        if self.drift_on and self.kT > 0.0:
            W = rfd_directions(self.seed, self.instance, self.step_count, X.shape[0], X.shape[1])
            d = self.rfd_drift(X, W)
        self.chain_cycles(ncycles)
        f = _flat(coupling.spread(self.sys, F, X))
        axi = _flat(self.chain_sys.apply(0, self.xi))
        w = self.S(dt * f + np.sqrt(2.0 * self.kT * dt) * axi)
        V = coupling.interpolate(self.sys, _fields(self.sys, w), X)
        self.step_count += 1
        return self.wrap_reflect(X + V + dt * d)
