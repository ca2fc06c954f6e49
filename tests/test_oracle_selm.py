"""Pins for the SELM driver (oracle/selm.py): Sections 2.1, 3 and Algorithm 4."""

import numpy as np
import pytest

import selm_inputs
from oracle import coupling, selm
from tests.affine import block_diag, flatten, unflatten


@pytest.mark.parametrize("project", [False, True])
def test_mobility_symmetric_positive(project):
    m = selm.Model(16, 2, mu=1.0, kT=1.0, levels=4, project=project, tol=1e-12)
    X = selm_inputs.particles(4, 2, 16, seed=0)
    M = m.mobility_matrix(X)
    assert np.abs(M - M.T).max() < 1e-9 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def _thermal_operator(m, X):
    """K = sqrt(2 kT) Gamma P~ as a matrix (columns = responses to unit xi)."""
    shapes = m.sys.shapes()
    nv = sum(int(np.prod(s)) for s in shapes)
    K = np.zeros((X.size, nv))
    for i in range(nv):
        e = np.zeros(nv)
        e[i] = 1.0
        K[:, i] = np.sqrt(2 * m.kT) * coupling.interpolate(m.sys, m.P(unflatten(e, shapes)), X).ravel()
    return K


@pytest.mark.parametrize("project", [False, True])
def test_fluctuation_dissipation_identity(project):
    # G = K C K^T with C = A^-1 equals 2 kT M (Eq. equ_G_special_form)
    m = selm.Model(8, 2, mu=0.7, kT=1.9, levels=3, project=project, tol=1e-13)
    X = selm_inputs.particles(3, 2, 8, seed=1)
    K = _thermal_operator(m, X)
    A = block_diag([cl.dense() for cl in m.sys.levels[0]])
    G = K @ np.linalg.inv(A) @ K.T
    M = m.mobility_matrix(X)
    assert np.allclose(G, 2 * m.kT * M, atol=1e-9 * np.abs(G).max())


def test_em_step_without_noise_is_mobility_drift():
    m = selm.Model(16, 2, kT=0.0, levels=4, tol=1e-12)
    X = selm_inputs.particles(5, 2, 16, seed=2)
    F = selm_inputs.forces(5, 2, seed=2)
    U, _, _ = m.mobility_apply(X, F)
    X1, _ = m.em_step(X, F, 1e-3, ncycles=2)
    assert np.allclose(X1, m.wrap_reflect(X + 1e-3 * U), atol=1e-13)


def test_wrap_and_reflect():
    m = selm.Model(8, 3, levels=2)
    X = np.array([[1.25, -0.5, -0.1], [0.5, 0.5, 1.2]])
    Y = m.wrap_reflect(X)
    assert np.allclose(Y, [[0.25, 0.5, 0.1], [0.5, 0.5, 0.8]])


def test_chain_counter_advances_and_reproduces():
    a = selm.Model(8, 2, levels=3, seed=5)
    b = selm.Model(8, 2, levels=3, seed=5)
    a.chain_cycles(3)
    b.chain_cycles(1)
    b.chain_cycles(2)          # resume: same counter sequence, same chain
    assert a.cycle == b.cycle == 3
    assert np.array_equal(flatten(a.xi), flatten(b.xi))


def test_em_displacement_statistics_without_force():
    # Algorithm 4 with F = 0: the displacement X1 - X0 = sqrt(2 kT dt) Gamma xi
    # has mean 0 and covariance 2 kT dt M (statistical pin; consecutive samples
    # of the multigrid chain are practically independent, lag-1 correlation ~2 %)
    kT, dt = 1.3, 1e-4
    m = selm.Model(8, 2, mu=1.0, kT=kT, levels=3, seed=3, instance=1, tol=1e-13)
    X0 = np.array([[0.31, 0.42], [0.77, 0.58]])
    M = m.mobility_matrix(X0)
    m.chain_cycles(10)
    F = np.zeros_like(X0)
    D = np.array([(m.em_step(X0, F, dt, ncycles=1)[0] - X0).ravel() for _ in range(1200)])
    target = 2 * kT * dt * M
    nb = 10
    batches = np.array_split(D, nb)
    covs = np.array([b.T @ b / b.shape[0] for b in batches])
    means = np.array([b.mean(0) for b in batches])
    se_cov = covs.std(0, ddof=1) / np.sqrt(nb)
    assert np.all(np.abs(covs.mean(0) - target) < 5 * se_cov + 1e-3 * np.abs(target).max())
    se_mean = means.std(0, ddof=1) / np.sqrt(nb)
    assert np.all(np.abs(means.mean(0)) < 5 * se_mean)
    assert np.abs(covs.mean(0) - target).max() < 0.2 * np.abs(target).max()


def test_config1_mobility_matches_direct_solves():
    # 2-D 64^2, 16 particles: the 32 x 32 mobility from FAC solves equals the
    # one from sparse direct solves of the same operator, and is symmetric
    # positive definite
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    m = selm.Model(64, 2, mu=1.0, kT=1.0, levels=6, tol=1e-12)
    X = selm_inputs.particles(16, 2, 64, seed=0)
    M = m.mobility_matrix(X)
    blocks = []
    for cl in m.sys.levels[0]:
        K, Mm = [sp.csr_matrix(k) for k in cl.K], [sp.csr_matrix(x) for x in cl.M]
        blocks.append(cl.scale * (sp.kron(Mm[2], sp.kron(Mm[1], K[0])) + sp.kron(Mm[2], sp.kron(K[1], Mm[0]))
                                  + sp.kron(K[2], sp.kron(Mm[1], Mm[0]))))
    lu = spla.splu(sp.block_diag(blocks).tocsc())
    shapes = m.sys.shapes()
    Md = np.zeros_like(M)
    for col in range(32):
        F = np.zeros((16, 2))
        F[col // 2, col % 2] = 1.0
        u = unflatten(lu.solve(flatten(coupling.spread(m.sys, F, X))), shapes)
        Md[:, col] = coupling.interpolate(m.sys, u, X).ravel()
    assert np.abs(M - Md).max() < 1e-9 * np.abs(Md).max()
    assert np.abs(M - M.T).max() < 1e-9 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0
