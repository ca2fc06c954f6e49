"""Pins for one stochastic Gauss-Seidel sweep (oracle/gibbs.py), Section 3.1.

The sweep is the affine map z' = R z + S b + Q n.  With A = D - L - U in the
sweep's visiting order the paper states R = (D - L)^-1 U (Eq. equ_R_GS),
Q = (D - L)^-1 D^(1/2) (Eq. equ_def_Q_GS), QQ^T = (D-L)^-1 D (D-U)^-1
(Eq. equ_J_cov_GS) and the stationarity condition J = C - R C R^T with
C = A^-1 (Eq. equ_J_eq_C_R).
"""

import numpy as np
import pytest

from oracle import gibbs, grid
from tests.affine import block_diag, extract


def _visiting_permutation(system, level):
    perm, off = [], 0
    for cl in system.levels[level]:
        nz, ny, nx = cl.shape
        for colour, (k, j, i) in cl.colour_classes():
            perm.append(off + (k * ny + j) * nx + i)
        off += cl.size
    return np.concatenate(perm)


CASES = [("velocity", 2, 8, 2, 0), ("velocity", 2, 8, 2, 1), ("velocity", 3, 4, 2, 0),
         ("velocity", 3, 8, 2, 1), ("pressure", 2, 8, 2, 1)]


@pytest.mark.parametrize("which,dim,n,levels,level", CASES)
def test_sweep_matches_paper_factors(which, dim, n, levels, level):
    s = (grid.velocity_system(n, dim, mu=1.3, levels=levels) if which == "velocity"
         else grid.pressure_system(n, dim, levels=levels))
    shapes = s.shapes(level)

    def step(z, b, noise):
        return gibbs.sweep(s, level, z, b, 0, noise, 1.0)

    R, S, Q, c = extract(step, shapes)
    assert np.allclose(c, 0.0)
    A = block_diag([cl.dense() for cl in s.levels[level]])
    perm = _visiting_permutation(s, level)
    Ap = A[np.ix_(perm, perm)]
    D = np.diag(np.diag(Ap))
    L = -np.tril(Ap, -1)
    U = -np.triu(Ap, 1)
    DL_inv = np.linalg.inv(D - L)
    Rp = DL_inv @ U
    Qp = DL_inv @ np.sqrt(D)
    assert np.allclose(R[np.ix_(perm, perm)], Rp, atol=1e-12)
    assert np.allclose(Q[perm, :], Qp, atol=1e-12)
    assert np.allclose(S[np.ix_(perm, perm)], DL_inv, atol=1e-12)
    J = Q @ Q.T
    Jp = DL_inv @ D @ np.linalg.inv(D - U)
    assert np.allclose(J[np.ix_(perm, perm)], Jp, atol=1e-12)
    if which == "velocity":  # SPD: stationarity J = C - R C R^T with C = A^-1
        C = np.linalg.inv(A)
        err = np.abs(C - R @ C @ R.T - J).max() / np.abs(C).max()
        assert err < 1e-12
        # the mean A^-1 b is a fixed point of the noiseless sweep
        b = np.random.default_rng(0).standard_normal(A.shape[0])
        x = np.linalg.solve(A, b)
        assert np.allclose(R @ x + S @ b, x, atol=1e-11)


def test_sweep_uses_each_site_once():
    s = grid.velocity_system(8, 3, levels=2)
    for level in range(2):
        from oracle.philox import ExplicitNoise
        z = s.zeros(level)
        noise = ExplicitNoise(None)
        gibbs.sweep(s, level, z, s.zeros(level), 0, noise, 1.0)
        assert noise.count == sum(cl.size for cl in s.levels[level])
