"""Pins for the MAC divergence / gradient / projection (oracle/projection.py)."""

import numpy as np
import pytest

from oracle import grid, projection
from tests.affine import flatten, unflatten


def _dense_divergence(n, dim):
    vs = grid.velocity_system(n, dim, levels=1)
    shapes = vs.shapes()
    nv = sum(int(np.prod(s)) for s in shapes)
    cols = []
    for i in range(nv):
        e = np.zeros(nv)
        e[i] = 1.0
        cols.append(projection.divergence(unflatten(e, shapes), dim).ravel())
    return np.array(cols).T, shapes


@pytest.mark.parametrize("dim,n", [(2, 8), (3, 4)])
def test_divergence_and_gradient_are_adjoint(dim, n):
    D, shapes = _dense_divergence(n, dim)
    rng = np.random.default_rng(0)
    phi = rng.standard_normal(D.shape[0]).reshape(shapes[0] if dim == 2 else (n, n, n))
    phi = phi.reshape((n, 1, n) if dim == 2 else (n, n, n))
    G = flatten(projection.divergence_transpose(phi, dim))
    assert np.allclose(G, D.T @ phi.ravel(), atol=1e-13)


@pytest.mark.parametrize("dim,n", [(2, 8), (3, 4)])
def test_divergence_of_cell_fluxes(dim, n):
    # (D^ u)_m = sum over faces of the outward normal value (Eq. equ_def_discr_div):
    # check one interior and one wall cell by hand
    vs = grid.velocity_system(n, dim, levels=1)
    rng = np.random.default_rng(1)
    w = [rng.standard_normal(s) for s in vs.shapes()]
    div = projection.divergence(w, dim)
    u = w[0]
    wz = w[-1]
    k, j, i = 1, 0, 2
    expect = u[k, j, i + 1] - u[k, j, i] + wz[k, j, i] - wz[k - 1, j, i]
    if dim == 3:
        expect += w[1][k, j + 1, i] - w[1][k, j, i]
    assert div[k, j, i] == pytest.approx(expect)
    k = 0                                   # bottom wall face carries no flux
    expect = u[k, j, i + 1] - u[k, j, i] + wz[k, j, i]
    if dim == 3:
        expect += w[1][k, j + 1, i] - w[1][k, j, i]
    assert div[k, j, i] == pytest.approx(expect)


@pytest.mark.parametrize("dim,n", [(2, 8), (3, 4)])
def test_pressure_operator_is_DDt(dim, n):
    D, _ = _dense_divergence(n, dim)
    ps = grid.pressure_system(n, dim, levels=1)
    assert np.allclose(ps.levels[0][0].dense(), D @ D.T, atol=1e-13)


@pytest.mark.parametrize("dim,n", [(2, 8), (3, 4)])
def test_projection_dense_properties(dim, n):
    D, shapes = _dense_divergence(n, dim)
    pr = projection.Projector(n, dim, tol=1e-13, levels=2)
    nv = D.shape[1]
    Pm = np.zeros((nv, nv))
    for i in range(nv):
        e = np.zeros(nv)
        e[i] = 1.0
        Pm[:, i] = flatten(pr.project(unflatten(e, shapes)))
    want = np.eye(nv) - D.T @ np.linalg.pinv(D @ D.T, rcond=1e-10, hermitian=True) @ D
    assert np.allclose(Pm, want, atol=1e-10)
    assert np.allclose(Pm, Pm.T, atol=1e-10)
    assert np.allclose(Pm @ Pm, Pm, atol=1e-10)
    assert np.abs(D @ Pm).max() < 1e-10


def test_projection_removes_divergence_16():
    pr = projection.Projector(16, 3)
    vs = grid.velocity_system(16, 3, levels=1)
    rng = np.random.default_rng(2)
    w = [rng.standard_normal(s) for s in vs.shapes()]
    pw = pr.project(w)
    assert np.abs(projection.divergence(pw, 3)).max() < 1e-9 * np.abs(projection.divergence(w, 3)).max()
    ppw = pr.project(pw)
    assert np.linalg.norm(flatten(ppw) - flatten(pw)) < 1e-9 * np.linalg.norm(flatten(pw))
