"""Decorrelation of the stochastic samplers: multigrid against Gauss-Seidel.

TEST INFRASTRUCTURE ONLY (see the package header).

Section 5 compares the two stochastic iterations by how strongly the random
variates they generate stay correlated after a given number of iterations,
in 2-D and 3-D, and finds that the multigrid sampler needs O(1) iterations
while Gauss-Seidel stays correlated for many (the figure comparing the
multigrid and Gauss-Seidel samplers).  The figure's data are not printed, so
the measure is fixed here (reading R20):

* Each sampler is an affine iteration z' = M z + N b + B n whose invariant
  law is N(A^-1 b, C), C = A^-1 (Section 3.1 for Gauss-Seidel, Section 3.2
  for the multigrid cycle).  Section 3.1 gives the lag covariance of the
  stochastic iteration by the recurrence C^(0,k) = R^k C^(0,0) (and bounds
  its norm by ||R||^k ||C^(0,0)||); the same argument holds for the
  multigrid cycle's map M: z_k is M^k z_0 plus noise drawn after z_0, so in
  the stationary state with b = 0, Cov(z_k, z_0) = M^k C.
* For a linear observable phi^T z the lag-k correlation is therefore
      rho(k) = phi^T M^k C phi / phi^T C phi.
  It is computed without sampling: w = C phi by a solve, then k noiseless
  iterations with b = 0 (z <- M z), then the inner product with phi.
* One iteration of the multigrid sampler is one stochastic FAC cycle
  (Algorithm 1, V-cycle of Algorithm 3, mu1 = mu2 = 2).  One iteration of
  the Gauss-Seidel sampler is one full red-black stochastic sweep of the
  fine grid (Section 3.1): the same FAC form on a one-level hierarchy whose
  only level is smoothed (coarse_mode "smooth", mu1 = 1, mu2 = 0).
* Observables: the lowest wall mode of component 0 (uniform along the
  periodic axes, sin(pi z) across the channel; an eigenvector of A, the
  slowest mode of Gauss-Seidel) and a point probe at the channel centre.
* The integrated autocorrelation time 1 + 2 sum_{k>=1} rho(k) converts a
  correlation curve into iterations per independent variate.
"""

import numpy as np

from . import grid, multigrid
from .philox import ExplicitNoise


def mg_sampler(n, dim, mu=1.0, levels=None):
    """The multigrid sampler's hierarchy and its exact coarsest step."""
    s = grid.velocity_system(n, dim, mu=mu, levels=levels)
    return dict(system=s, mu=mu, mu1=2, mu2=2, coarse_mode="cholesky", coarsest=multigrid.Coarsest(s))


def gs_sampler(n, dim, mu=1.0):
    """The Gauss-Seidel sampler: one red-black sweep of the fine grid per iteration."""
    s = grid.velocity_system(n, dim, mu=mu, levels=1)
    return dict(system=s, mu=mu, mu1=1, mu2=0, coarse_mode="smooth", coarsest=None)


def iterate(sampler, z, b, noise, sigma):
    """One iteration of a sampler (Algorithm 1 with the sampler's V-cycle), in place."""
    return multigrid.fac_cycle(sampler["system"], z, b, noise, sigma, sampler["mu1"], sampler["mu2"],
                               sampler["coarse_mode"], sampler["coarsest"])


def wall_mode(system):
    """Component 0 = sin(pi z) at its nodes, uniform in x (and y); other components 0."""
    out = system.zeros(0)
    cl = system.levels[0][0]
    z = grid.node_positions(cl.kinds[2], system.n)
    out[0][...] = np.sin(np.pi * z)[:, None, None]
    return out


def point_probe(system):
    """Unit vector at the centre node of component 0."""
    out = system.zeros(0)
    nz, ny, nx = out[0].shape
    out[0][nz // 2, ny // 2, nx // 2] = 1.0
    return out


def dot(a, b):
    return float(sum(float(np.sum(x * y)) for x, y in zip(a, b)))


def covariance_image(sampler, phi, tol=1e-13):
    """w = C phi = A^-1 phi: the deterministic FAC solve on the full hierarchy
    of the sampler's fine-grid operator (both samplers share that operator)."""
    s = sampler["system"]
    full = grid.velocity_system(s.n, s.dim, mu=sampler["mu"])
    w, cycles, rel = multigrid.solve(full, phi, tol=tol, max_cycles=200)
    return w


def lag_correlations(sampler, phi, K, w=None):
    """rho(0..K) of the observable phi for the sampler (reading R20)."""
    s = sampler["system"]
    if w is None:
        w = covariance_image(sampler, phi)
    z = [x.copy() for x in w]
    zero = s.zeros(0)
    var = dot(phi, w)
    rho = [1.0]
    for _ in range(K):
        iterate(sampler, z, zero, ExplicitNoise(), 0.0)
        rho.append(dot(phi, z) / var)
    return np.array(rho)


def integrated_time(rho):
    """1 + 2 sum_{k>=1} rho(k) over the computed lags."""
    return 1.0 + 2.0 * float(np.sum(rho[1:]))


def lags_below(rho, threshold=0.05):
    """First lag k with |rho(j)| < threshold for all j >= k among the computed lags, else None."""
    above = np.nonzero(np.abs(rho) >= threshold)[0]
    k = int(above[-1]) + 1 if above.size else 0
    return k if k < len(rho) else None
