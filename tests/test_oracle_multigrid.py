"""Pins for the stochastic V-cycle / FAC iteration (oracle/multigrid.py).

The paper's central claim (Section 3.2): with Galerkin coarse operators and
restriction = prolongation^T, the target N(A^-1 b, A^-1) is invariant under
the stochastic multigrid cycle.  The FAC cycle is affine,
z' = M z + N b + B n, so invariance is the exact identity
    A^-1 = M A^-1 M^T + B B^T   and   A^-1 b = M A^-1 b + N b.
"""

import numpy as np
import pytest

from oracle import grid, multigrid
from oracle.philox import ExplicitNoise, PhiloxNoise
from tests import closed_forms as cf
from tests.affine import block_diag, extract, flatten, unflatten


@pytest.mark.parametrize("dim,n,levels,mode", [
    (2, 8, 3, "cholesky"), (2, 8, 3, "smooth"), (3, 4, 2, "cholesky"), (2, 4, 1, "cholesky"),
])
def test_cycle_invariance_exact(dim, n, levels, mode):
    s = grid.velocity_system(n, dim, mu=0.9, levels=levels)
    co = multigrid.Coarsest(s) if mode == "cholesky" else None
    shapes = s.shapes(0)

    def step(z, b, noise):
        return multigrid.fac_cycle(s, z, b, noise, 1.0, 2, 2, mode, co)

    M, N, B, c = extract(step, shapes)
    A = block_diag([cl.dense() for cl in s.levels[0]])
    C = np.linalg.inv(A)
    err = np.abs(M @ C @ M.T + B @ B.T - C).max() / np.abs(C).max()
    assert err < 1e-12
    b = np.random.default_rng(5).standard_normal(A.shape[0])
    x = C @ b
    assert np.allclose(M @ x + N @ b + c, x, atol=1e-11)
    # contraction: spectral radius of M below 1 (deterministic convergence)
    assert np.max(np.abs(np.linalg.eigvals(M))) < 0.5


def test_wrong_restriction_scaling_breaks_invariance():
    # A plausible slip (restriction = P^T / 2 with Galerkin A_c = P^T A P)
    # must be caught by the invariance identity used above.
    s = grid.velocity_system(8, 2, levels=2)
    co = multigrid.Coarsest(s)
    orig = s.restrict
    s.restrict = lambda level, r: [0.5 * x for x in orig(level, r)]
    try:
        M, N, B, c = extract(lambda z, b, nz: multigrid.fac_cycle(s, z, b, nz, 1.0, 2, 2,
                                                                 "cholesky", co), s.shapes(0))
    finally:
        s.restrict = orig
    A = block_diag([cl.dense() for cl in s.levels[0]])
    C = np.linalg.inv(A)
    assert np.abs(M @ C @ M.T + B @ B.T - C).max() / np.abs(C).max() > 1e-4


def test_coarsest_exact_sample_covariance():
    s = grid.velocity_system(4, 2, levels=2)
    co = multigrid.Coarsest(s)
    lev = 1
    shapes = s.shapes(lev)

    def step(z, b, noise):
        return co.apply(s, b, noise, 1.0)

    M, N, B, c = extract(step, shapes)
    A = block_diag([cl.dense() for cl in s.levels[lev]])
    assert np.allclose(M, 0.0)
    assert np.allclose(N, np.linalg.inv(A), atol=1e-13)
    assert np.allclose(B @ B.T, np.linalg.inv(A), atol=1e-13)


@pytest.mark.parametrize("dim,n,levels", [(2, 64, 6), (3, 16, 3), (3, 32, 4)])
def test_solve_matches_spectral_closed_form(dim, n, levels):
    s = grid.velocity_system(n, dim, mu=1.0, levels=levels)
    rng = np.random.default_rng(11)
    b = [rng.standard_normal(sh) for sh in s.shapes()]
    v, cycles, rel = multigrid.solve(s, b, tol=1e-10)
    assert rel <= 1e-10 and cycles <= 12
    for c, cl in enumerate(s.levels[0]):
        x = cf.spectral_solve(cl.kinds, n, cl.scale, b[c])
        assert np.linalg.norm(v[c] - x) / np.linalg.norm(x) < 1e-8


def test_pressure_solve_matches_spectral_closed_form():
    s = grid.pressure_system(16, 3, levels=3)
    rng = np.random.default_rng(12)
    b = rng.standard_normal(s.shapes()[0])
    b -= b.mean()
    v, cycles, rel = multigrid.solve(s, [b], tol=1e-11)
    x = cf.spectral_solve(s.levels[0][0].kinds, 16, 1.0, b)
    assert rel <= 1e-11
    assert np.linalg.norm(v[0] - v[0].mean() - x) / np.linalg.norm(x) < 1e-9


def test_chain_sample_covariance():
    # Statistical pin: the chain's sample covariance approaches A^-1.
    s = grid.velocity_system(4, 2, levels=2)
    co = multigrid.Coarsest(s)
    A = block_diag([cl.dense() for cl in s.levels[0]])
    C = np.linalg.inv(A)
    z = s.zeros(0)
    zero = s.zeros(0)
    samples = []
    for cyc in range(2000):
        multigrid.fac_cycle(s, z, zero, PhiloxNoise(0, 0, cyc), 1.0, coarsest=co)
        samples.append(flatten(z))
    X = np.array(samples[20:])
    nb = 20                                    # batch means for the standard error
    batches = np.array_split(X, nb)
    covs = np.array([b.T @ b / b.shape[0] for b in batches])
    mean_cov = covs.mean(0)
    se = covs.std(0, ddof=1) / np.sqrt(nb)
    z_scores = (mean_cov - C) / se
    diag = np.arange(C.shape[0])
    assert np.all(np.abs(z_scores[diag, diag]) < 5.0)
    # batch-means z-scores are t(19)-distributed: E[z^2] = 19/17
    assert np.mean(z_scores ** 2) < 1.6


def test_refinement_form_equals_direct_cycle():
    # V(z, b, n) = z + V(0, b - A z, n): the FAC form of Algorithm 1 equals a
    # V-cycle applied to z directly (affine cycle, additive noise).
    s = grid.velocity_system(8, 2, levels=3)
    co = multigrid.Coarsest(s)
    rng = np.random.default_rng(4)
    z0 = [rng.standard_normal(sh) for sh in s.shapes()]
    b = [rng.standard_normal(sh) for sh in s.shapes()]
    z1 = [x.copy() for x in z0]
    multigrid.fac_cycle(s, z1, b, PhiloxNoise(3, 0, 17), 1.0, coarsest=co)
    z2 = [x.copy() for x in z0]
    multigrid.vcycle(s, 0, z2, b, PhiloxNoise(3, 0, 17), 1.0, coarsest=co)
    assert np.allclose(flatten(z1), flatten(z2), atol=1e-12)
