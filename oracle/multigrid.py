"""Stochastic multigrid: V-cycle (Algorithm 3) and FAC iteration (Algorithm 1).

On a uniform grid the hierarchy has no refined patches, so Full-Sweep
(Algorithm 2) reduces to one V-cycle on the base level and FAC-Multigrid is

    r = b - A v            (Algorithm 1 step 1; sign read as b - Av, reading R6)
    q <- 0                 (step 2)
    q <- V-Cycle(q, r)     (step 3)
    v <- v + q             (step 4)

V-Cycle(v, b) at level l (Algorithm 3):
    1. mu1 stochastic smoothing sweeps on A^(l) v = b^(l)
    2. at the coarsest level go to 5
    3. b^(l+1) <- P^T (b^(l) - A^(l) v^(l)),  v^(l+1) <- 0,  V-Cycle on level l+1
       (reading R5 of the garbled formula)
    4. v^(l) <- v^(l) + P v^(l+1)
    5. mu2 stochastic smoothing sweeps

Coarsest level (reading R7): the paper only smooths there.  The default here
("cholesky") replaces steps 1 and 5 at the coarsest level by an exact draw
from the level's conditional distribution, v = A_c^-1 b + sigma L_c^-T n with
A_c = L_c L_c^T, an exact block heat-bath update that keeps the invariant
measure.  ``coarse_mode="smooth"`` runs steps 1 and 5 literally.
For a singular pure-Neumann coarse operator (pressure) the factor is taken of
A_c + (mean diag / N_c) 1 1^T, which returns the zero-mean solution for a
consistent right-hand side.
"""

import numpy as np
import scipy.linalg as sla

from . import gibbs


class Coarsest:
    """Dense Cholesky factors of the coarsest-level operators."""

    def __init__(self, system):
        self.L = []
        lev = system.nlevels - 1
        for cl in system.levels[lev]:
            A = cl.dense()
            if cl.kinds[2] == "N" and all(k in ("P", "O", "N") for k in cl.kinds):
                nrm = np.mean(np.diag(A)) / A.shape[0]
                A = A + nrm * np.ones_like(A)
            self.L.append(np.linalg.cholesky(A))

    def apply(self, system, b, noise, sigma):
        lev = system.nlevels - 1
        out = []
        for c, cl in enumerate(system.levels[lev]):
            L = self.L[c]
            y = sla.solve_triangular(L, b[c].ravel(), lower=True)
            if sigma != 0.0:
                y = y + sigma * noise.coarsest(lev, cl.comp, y.size)
            x = sla.solve_triangular(L.T, y, lower=False)
            out.append(x.reshape(cl.shape))
        return out


def vcycle(system, level, v, b, noise, sigma, mu1=2, mu2=2, coarse_mode="cholesky",
           coarsest=None):
    """Algorithm 3 on lists of per-component arrays; v is updated in place."""
    last = system.nlevels - 1
    if level == last and coarse_mode == "cholesky":
        if coarsest is None:
            coarsest = Coarsest(system)
        x = coarsest.apply(system, b, noise, sigma)
        for c in range(len(v)):
            v[c][...] = x[c]
        return v
    for s in range(mu1):                                     # step 1
        gibbs.sweep(system, level, v, b, s, noise, sigma)
    if level < last:                                         # steps 2-4
        Av = system.apply(level, v)
        bc = system.restrict(level, [bb - a for bb, a in zip(b, Av)])
        vc = system.zeros(level + 1)
        vcycle(system, level + 1, vc, bc, noise, sigma, mu1, mu2, coarse_mode, coarsest)
        corr = system.prolong(level, vc)
        for c in range(len(v)):
            v[c] += corr[c]
    for s in range(mu2):                                     # step 5
        gibbs.sweep(system, level, v, b, mu1 + s, noise, sigma)
    return v


def fac_cycle(system, v, b, noise, sigma, mu1=2, mu2=2, coarse_mode="cholesky",
              coarsest=None):
    """Algorithm 1 (uniform grid): v <- v + V-Cycle(0, b - A v)."""
    Av = system.apply(0, v)
    r = [bb - a for bb, a in zip(b, Av)]
    q = system.zeros(0)
    vcycle(system, 0, q, r, noise, sigma, mu1, mu2, coarse_mode, coarsest)
    for c in range(len(v)):
        v[c] += q[c]
    return v


def norm(fields):
    return float(np.sqrt(sum(float(np.sum(f * f)) for f in fields)))


def residual_norm(system, v, b):
    Av = system.apply(0, v)
    return norm([bb - a for bb, a in zip(b, Av)])


def solve(system, b, tol=1e-10, max_cycles=100, v0=None, mu1=2, mu2=2,
          coarse_mode="cholesky", coarsest=None):
    """Deterministic FAC iteration until ||b - A v||_2 <= tol ||b||_2 (reading R9).

    Returns (v, cycles, relative residual).
    """
    from .philox import ExplicitNoise
    if coarsest is None and coarse_mode == "cholesky":
        coarsest = Coarsest(system)
    v = system.zeros(0) if v0 is None else [x.copy() for x in v0]
    bn = norm(b)
    if bn == 0.0:
        return v, 0, 0.0
    cycles = 0
    rel = residual_norm(system, v, b) / bn
    while rel > tol and cycles < max_cycles:
        fac_cycle(system, v, b, ExplicitNoise(), 0.0, mu1, mu2, coarse_mode, coarsest)
        cycles += 1
        rel = residual_norm(system, v, b) / bn
    return v, cycles, rel
