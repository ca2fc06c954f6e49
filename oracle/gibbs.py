"""Stochastic Gauss-Seidel (Gibbs heat-bath) sweeps, Section 3.1.

With A = D - L - U (Eq. equ_R_GS context) the stochastic Gauss-Seidel
iteration Z <- R Z + s + Q n with R = (D - L)^-1 U and Q = (D - L)^-1 D^(1/2)
(Eq. equ_def_Q_GS) is, written site by site in the visiting order,

    z_i <- ( b_i - sum_{j != i} A_ij z_j ) / A_ii  +  sigma * n_i / sqrt(A_ii)

with n_i independent standard normals.  sigma = 1 samples N(A^-1 b, A^-1)
(the invariant measure, Eq. equ_J_cov_GS); sigma = 0 is plain Gauss-Seidel.
Sites of one colour class are mutually uncoupled, so updating them together
equals updating them one after another.
"""

import numpy as np


def sweep(system, level, v, b, sweep_id, noise, sigma):
    """One full sweep (all colours) of every component at `level`, in place.

    v, b : lists of arrays (one per component)
    noise: object with ``sweep(level, comp, colour, sweep, nsites)``
    """
    for c, cl in enumerate(system.levels[level]):
        diag = cl.diagonal()
        x = v[c]
        for colour, idx in cl.colour_classes():
            Ax = cl.apply(x)
            off = Ax[idx] - diag[idx] * x[idx]          # sum_{j != i} A_ij z_j
            new = (b[c][idx] - off) / diag[idx]
            if sigma != 0.0:
                n = noise.sweep(level, cl.comp, colour, sweep_id, idx[0].size)
                new = new + sigma * n / np.sqrt(diag[idx])
            x[idx] = new
    return v
