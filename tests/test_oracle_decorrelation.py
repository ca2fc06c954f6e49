"""Pins for the sampler decorrelation measure (oracle/decorrelation.py), Section 5.

rho(k) = phi^T M^k C phi / phi^T C phi, C = A^-1, is the lag-k correlation of
phi^T z for a stationary affine sampler z' = M z + B n.  The oracle computes
it by noiseless iterations from C phi.  It is pinned against
* the dense matrix form, with M probed from the noisy iteration as an affine
  map and C the inverse of the assembled operator;
* the exact sampler (one level, exact block step): M = 0, so rho(k) = 0 for
  every k >= 1;
* closed forms of the observables: the wall mode is an eigenvector of A
  (discrete sine transform of the cell lattice) and C phi = phi / lambda;
* the empirical lag correlation of long seeded noisy chains;
and the paper's statement (multigrid: O(1) iterations; Gauss-Seidel: strong
correlation after many) is checked on 2-D and 3-D grids.
"""

import numpy as np
import pytest

from oracle import decorrelation as D
from oracle import grid, multigrid
from oracle.philox import PhiloxNoise
from tests.affine import block_diag, extract, flatten


def _dense(sampler):
    s = sampler["system"]
    shapes = s.shapes(0)

    def step(z, b, noise):
        return D.iterate(sampler, z, b, noise, 1.0)

    M, N, B, c = extract(step, shapes)
    A = block_diag([cl.dense() for cl in s.levels[0]])
    return M, B, np.linalg.inv(A)


def _rho_dense(M, C, phi, K):
    p = flatten(phi)
    x = C @ p
    var = p @ x
    out = []
    for _ in range(K + 1):
        out.append(p @ x / var)
        x = M @ x
    return np.array(out)


@pytest.mark.parametrize("kind,dim,n", [("mg", 2, 8), ("gs", 2, 8), ("mg", 3, 4), ("gs", 3, 4)])
def test_lag_correlations_equal_matrix_form(kind, dim, n):
    smp = D.mg_sampler(n, dim, mu=0.8) if kind == "mg" else D.gs_sampler(n, dim, mu=0.8)
    M, B, C = _dense(smp)
    # the sampler leaves N(0, C) invariant (Sections 3.1, 3.2)
    assert np.abs(M @ C @ M.T + B @ B.T - C).max() / np.abs(C).max() < 1e-12
    s = smp["system"]
    rng = np.random.default_rng(3)
    for phi in (D.wall_mode(s), D.point_probe(s), [rng.standard_normal(sh) for sh in s.shapes(0)]):
        rho = D.lag_correlations(smp, phi, 6)
        assert np.abs(rho - _rho_dense(M, C, phi, 6)).max() < 1e-11


def test_forgetting_the_covariance_is_caught():
    # A plausible slip: iterating from phi instead of C phi (the lag correlation
    # of a white-noise start, not of the stationary chain).
    smp = D.gs_sampler(8, 2)
    M, B, C = _dense(smp)
    phi = D.point_probe(smp["system"])
    wrong = D.lag_correlations(smp, phi, 4, w=[x.copy() for x in phi])
    assert np.abs(wrong - _rho_dense(M, C, phi, 4)).max() > 1e-2


@pytest.mark.parametrize("dim,n", [(2, 8), (3, 4)])
def test_exact_sampler_decorrelates_in_one_iteration(dim, n):
    s = grid.velocity_system(n, dim, levels=1)
    smp = dict(system=s, mu=1.0, mu1=2, mu2=2, coarse_mode="cholesky", coarsest=multigrid.Coarsest(s))
    for phi in (D.wall_mode(s), D.point_probe(s)):
        rho = D.lag_correlations(smp, phi, 3)
        assert rho[0] == 1.0 and np.abs(rho[1:]).max() < 1e-13
        assert D.integrated_time(rho) == pytest.approx(1.0, abs=1e-12)
        assert D.lags_below(rho) == 1


@pytest.mark.parametrize("dim,n,mu", [(2, 16, 1.0), (3, 8, 0.7)])
def test_wall_mode_is_an_eigenvector(dim, n, mu):
    # cell lattice between Dirichlet walls: sin(pi (k + 1/2) / n) is the first
    # DST-II vector, eigenvalue 4 sin^2(pi / 2n) of the second difference;
    # the operator scale is mu h^(d-2)
    s = grid.velocity_system(n, dim, mu=mu)
    phi = D.wall_mode(s)
    lam = mu * (1.0 / n) ** (dim - 2) * 4.0 * np.sin(np.pi / (2 * n)) ** 2
    Aphi = s.apply(0, phi)
    assert np.abs(flatten(Aphi) - lam * flatten(phi)).max() < 1e-12
    w = D.covariance_image(D.mg_sampler(n, dim, mu=mu), phi)
    assert np.abs(flatten(w) - flatten(phi) / lam).max() < 1e-9 * np.abs(flatten(phi) / lam).max()


def _empirical(smp, phi, iters, burn, seed):
    s = smp["system"]
    z = s.zeros(0)
    zero = s.zeros(0)
    x = []
    for k in range(burn + iters):
        D.iterate(smp, z, zero, PhiloxNoise(seed, 0, k), 1.0)
        if k >= burn:
            x.append(D.dot(phi, z))
    return np.array(x)


def _acf(x, lags):
    x = x - x.mean()
    v = x @ x / x.size
    return np.array([(x[:-k] @ x[k:]) / (x.size - k) / v for k in lags])


@pytest.mark.parametrize("kind", ["mg", "gs"])
def test_lag_correlations_match_sampled_chains(kind):
    # Statistical pin: the lag correlations of the noisy seeded chain agree
    # with rho(k) within batch-means standard errors.
    n, dim = 8, 2
    smp = D.mg_sampler(n, dim) if kind == "mg" else D.gs_sampler(n, dim)
    phi = D.point_probe(smp["system"])
    lags = [1, 2, 4]
    rho = D.lag_correlations(smp, phi, max(lags))
    x = _empirical(smp, phi, 2500 if kind == "mg" else 6000, 50, seed=7 if kind == "mg" else 8)
    batches = np.array_split(x, 10)
    est = np.array([_acf(b, lags) for b in batches])
    mean, se = est.mean(0), est.std(0, ddof=1) / np.sqrt(len(batches))
    assert np.all(np.abs(mean - rho[lags]) < 5.0 * se), (mean, rho[lags], se)
    # and the stationary variance of phi^T z is phi^T C phi
    var = D.dot(phi, D.covariance_image(smp, phi))
    assert abs(x.var() / var - 1.0) < 0.15


@pytest.mark.parametrize("dim,n", [(2, 32), (3, 16)])
def test_multigrid_needs_O1_iterations_gauss_seidel_many(dim, n):
    # Section 5's finding, on both observables: the multigrid sampler's
    # correlation is below 5 % after one iteration, Gauss-Seidel's wall mode
    # is still above 40 % after 40 sweeps.
    mg, gs = D.mg_sampler(n, dim), D.gs_sampler(n, dim)
    for phi_of in (D.wall_mode, D.point_probe):
        r_mg = D.lag_correlations(mg, phi_of(mg["system"]), 4)
        assert D.lags_below(r_mg) == 1
        assert D.integrated_time(r_mg) < 1.1
    r_gs = D.lag_correlations(gs, D.wall_mode(gs["system"]), 40)
    assert r_gs[40] > 0.4 and D.lags_below(r_gs) is None
    assert np.all(np.diff(r_gs) < 0)          # monotone decay of the slow mode
