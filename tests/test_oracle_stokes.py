"""Pins of the exact discrete Stokes mobility and the Ito drift (oracle/stokes.py).

Each pin checks the oracle against something other than its own formula:
closed forms of flows that vary only along z (a shear flow needs no pressure,
a wall-normal body force is balanced by pressure alone), the variational
ordering of the two mobilities, the projection identity S A S = S, and the
random finite difference against a numerical derivative of the mobility.
"""

import numpy as np
import pytest

from oracle.stokes import StokesModel, StokesSolver, _fields, _flat, rfd_directions


def _column_operator(n, s):
    """1-D operator of a tangential component along z, built from the no-slip
    ghost rule (ghost = -value beyond the wall): diagonal 2, off-diagonals -1,
    wall rows 3, times s."""
    K = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    K[0, 0] = K[-1, -1] = 3.0
    return s * K


@pytest.mark.parametrize("dim,n", [(2, 8), (3, 6)])
def test_shear_flow_needs_no_pressure(dim, n):
    # f = (g(z), 0, 0): u = (A_z^-1 g, 0, 0), p = const
    mu = 0.7
    st = StokesSolver(n, dim, mu)
    shapes = st.system.shapes(0)
    g = np.sin(np.linspace(0.3, 2.9, n)) + 0.2
    f = [np.zeros(s) for s in shapes]
    f[0][:] = g[:, None, None]
    u, p = st.solve(_flat(f))
    U = _fields(st.system, u)
    s = mu * (1.0 / n) ** (dim - 2)
    col = np.linalg.solve(_column_operator(n, s), g)
    assert np.abs(U[0] - col[:, None, None]).max() < 1e-12 * np.abs(col).max()
    for c in range(1, len(U)):
        assert np.abs(U[c]).max() < 1e-12 * np.abs(col).max()
    assert np.abs(p).max() < 1e-10


@pytest.mark.parametrize("dim,n", [(2, 8), (3, 4)])
def test_wall_normal_body_force_is_hydrostatic(dim, n):
    # a uniform wall-normal force is the gradient of a linear pressure: no flow
    st = StokesSolver(n, dim)
    f = [np.zeros(s) for s in st.system.shapes(0)]
    f[-1][:] = 1.3
    u, p = st.solve(_flat(f))
    assert np.abs(u).max() < 1e-12
    # D^T p = f: (D^T p) on the face between cells k and k+1 is p_k - p_(k+1),
    # so p falls linearly along z by the force per face, uniform in x and y
    P = p.reshape(n, -1)
    assert np.abs(P - P[:, :1]).max() < 1e-10
    assert np.allclose(np.diff(P[:, 0]), -1.3, atol=1e-10)


@pytest.mark.parametrize("dim,n", [(2, 6), (3, 4)])
def test_stokes_operator_is_a_constrained_inverse(dim, n):
    st = StokesSolver(n, dim, mu=1.1)
    N = st.nv
    S = np.column_stack([st.solve(e)[0] for e in np.eye(N)])
    A = st.A.toarray()
    assert np.abs(S - S.T).max() < 1e-12 * np.abs(S).max()
    assert np.abs(S @ A @ S - S).max() < 1e-11 * np.abs(S).max()
    assert np.abs(st.D @ S).max() < 1e-12
    # P~ A^-1 P~ - S is positive semidefinite, and strictly so near walls
    # P~ = Z Z^T, Z an orthonormal basis of ker D (from the SVD of D)
    _, sv, Vt = np.linalg.svd(st.D.toarray())
    Z = Vt[(sv > 1e-10 * sv.max()).sum():].T
    P = Z @ Z.T
    gap = np.linalg.eigvalsh(P @ np.linalg.inv(A) @ P - S)
    assert gap.min() > -1e-12 * np.abs(S).max()
    assert gap.max() > 1e-6 * np.abs(S).max()


def test_wrong_pressure_sign_is_caught():
    # a plausible slip: A u - D^T p = f solved instead; D u = 0 still holds but
    # u differs from the constrained minimiser for a force with a gradient part
    st = StokesSolver(6, 2)
    rng = np.random.default_rng(3)
    f = rng.standard_normal(st.nv)
    u, p = st.solve(f)
    assert np.abs(st.A @ u + st.D.T @ p - f).max() < 1e-12
    assert np.abs(st.A @ u - st.D.T @ p - f).max() > 1e-3


def test_rfd_drift_matches_the_derivative_of_the_mobility():
    # one particle near the bottom wall: the mean of the random finite
    # difference over W equals kT * sum_j dM_ij/dX_j, the latter from central
    # differences of the mobility along each axis
    m = StokesModel(8, 2, kT=1.7, delta=1e-4)
    X = np.array([[0.37, 0.21]])
    div = np.zeros(2)
    e = 1e-4
    for j in range(2):
        dX = np.zeros((1, 2))
        dX[0, j] = e
        for i in range(2):
            F = np.zeros((1, 2))
            F[0, j] = 1.0
            div[i] += (m.mobility_apply(X + dX, F)[0, i] - m.mobility_apply(X - dX, F)[0, i]) / (2 * e)
    rng = np.random.default_rng(4)
    samples = np.array([m.rfd_drift(X, rng.standard_normal((1, 2)))[0] for _ in range(400)])
    mean, se = samples.mean(axis=0), samples.std(axis=0, ddof=1) / np.sqrt(len(samples))
    assert np.all(np.abs(mean - 1.7 * div) < 4 * se + 1e-9)
    # the wall-normal component dominates and points away from the wall
    assert 1.7 * div[1] > 10 * abs(1.7 * div[0])


def test_rfd_directions_are_standard_normals():
    W = rfd_directions(5, 2, 7, 2000, 3)
    assert W.shape == (2000, 3)
    assert abs(W.mean()) < 4 / np.sqrt(W.size) and abs(W.var() - 1) < 0.05
    assert not np.array_equal(W, rfd_directions(5, 2, 8, 2000, 3))


def test_em_step_deterministic_part_is_the_stokes_mobility():
    # kT = 0: X moves by dt M_S F
    m = StokesModel(8, 2, kT=0.0)
    X = np.array([[0.3, 0.33], [0.6, 0.41]])
    F = np.array([[0.5, -1.0], [0.1, 0.4]])
    Xn = m.em_step(X, F, 0.01, 1)
    M = m.mobility_matrix(X)
    assert np.abs((Xn - X).ravel() - 0.01 * M @ F.ravel()).max() < 1e-12
