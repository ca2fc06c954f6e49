"""SELM driver: mobility, thermal field and Euler-Maruyama steps (Algorithm 4).

Notation (Sections 2.1 and 3): A = mu h^d (-L) (SPD), Gamma = Peskin
interpolation, Lambda = h^-d Gamma^T, P~ = discrete projection.  Then the
discrete coupling tensor of Eq. equ_H_selm_discr is

    M = Gamma P~ A^-1 P~ Gamma^T                (mobility, U = M F)

and with xi ~ N(0, A^-1) the thermal term g = sqrt(2 kT) Gamma P~ xi has
covariance 2 kT M (Eq. equ_G_special_form, equ_g_gen_xi).  xi is the state of
a persistent stochastic multigrid chain advanced by FAC cycles with noise.

Euler-Maruyama step (Algorithm 4 step 4):
    X <- X + dt M F + sqrt(dt) g
       = X + Gamma P~ ( dt A^-1 P~ Gamma^T F + sqrt(2 kT dt) xi )
followed by periodic wrap in x (and y) and reflection at the walls
(reading R12).  No drift correction is added (the paper assumes
div_X H = 0, reading R12).
"""

import numpy as np

from . import grid, multigrid, coupling, projection
from .philox import PhiloxNoise


class Model:
    def __init__(self, n, dim, mu=1.0, kT=1.0, levels=None, project=False,
                 seed=0, instance=0, tol=1e-10, mu1=2, mu2=2, coarse_mode="cholesky"):
        self.n, self.dim, self.mu, self.kT = n, dim, mu, kT
        self.sys = grid.velocity_system(n, dim, mu, levels)
        self.coarsest = multigrid.Coarsest(self.sys) if coarse_mode == "cholesky" else None
        self.proj = projection.Projector(n, dim) if project else None
        self.seed, self.instance = seed, instance
        self.tol = tol
        self.mu1, self.mu2, self.coarse_mode = mu1, mu2, coarse_mode
        self.xi = self.sys.zeros(0)        # persistent chain state
        self.cycle = 0                      # chain step counter (Philox counter words 2-3)

    # projection slots (warm starts of the pressure solve): 0 = Gamma^T F,
    # 1 = the step's combined field, 2 = the sampled field
    def P(self, w, slot=None):
        return w if self.proj is None else self.proj.project(w, slot)

    # -- deterministic part ---------------------------------------------
    def rhs(self, X, F):
        return self.P(coupling.spread(self.sys, F, X), 0)

    def solve_field(self, b):
        u, cycles, rel = multigrid.solve(self.sys, b, tol=self.tol, mu1=self.mu1, mu2=self.mu2,
                                         coarse_mode=self.coarse_mode, coarsest=self.coarsest)
        return u, cycles, rel

    def mobility_apply(self, X, F):
        u, cycles, rel = self.solve_field(self.rhs(X, F))
        return coupling.interpolate(self.sys, self.P(u, 1), X), cycles, rel

    def mobility_matrix(self, X):
        """Dense M (columns = responses to unit forces), d np x d np."""
        npart, dim = X.shape
        Mm = np.zeros((npart * dim, npart * dim))
        for col in range(npart * dim):
            F = np.zeros((npart, dim))
            F[col // dim, col % dim] = 1.0
            U, _, _ = self.mobility_apply(X, F)
            Mm[:, col] = U.ravel()
        return Mm

    # -- stochastic part ------------------------------------------------
    def chain_cycles(self, ncycles):
        """Advance xi by ncycles stochastic FAC cycles with b = 0."""
        zero = self.sys.zeros(0)
        for _ in range(ncycles):
            noise = PhiloxNoise(self.seed, self.instance, self.cycle)
            multigrid.fac_cycle(self.sys, self.xi, zero, noise, 1.0, self.mu1, self.mu2,
                                self.coarse_mode, self.coarsest)
            self.cycle += 1
        return self.xi

    def thermal(self, X, ncycles):
        self.chain_cycles(ncycles)
        g = coupling.interpolate(self.sys, self.P(self.xi, 2), X)
        return np.sqrt(2.0 * self.kT) * g

    # -- dynamics -------------------------------------------------------
    def wrap_reflect(self, X):
        X = X.copy()
        X[:, :-1] = np.mod(X[:, :-1], 1.0)
        z = X[:, -1]
        z = np.where(z < 0.0, -z, z)
        z = np.where(z > 1.0, 2.0 - z, z)
        X[:, -1] = z
        return X

    def em_step(self, X, F, dt, ncycles):
        u, cycles, rel = self.solve_field(self.rhs(X, F))
        self.chain_cycles(ncycles)
        a = dt
        c = np.sqrt(2.0 * self.kT * dt)
        w = [a * uu + c * xx for uu, xx in zip(u, self.xi)]
        V = coupling.interpolate(self.sys, self.P(w, 1), X)
        return self.wrap_reflect(X + V), cycles
