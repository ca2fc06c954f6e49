"""Pins for Peskin 4-point interpolation / spreading (oracle/coupling.py)."""

import numpy as np
import pytest

from oracle import coupling, grid


def test_peskin_moment_identities():
    # Peskin (2002): sum_j phi(r - j) = 1, sum_j (r - j) phi(r - j) = 0,
    # even and odd sums are 1/2 each, sum_j phi(r - j)^2 = 3/8, for any r.
    r = np.random.default_rng(0).uniform(-3, 3, size=200)
    j = np.arange(-6, 7)
    phi = coupling.peskin_phi(r[:, None] - j[None, :])
    assert np.allclose(phi.sum(1), 1.0, atol=1e-14)
    assert np.allclose(((r[:, None] - j[None, :]) * phi).sum(1), 0.0, atol=1e-14)
    assert np.allclose(phi[:, (j % 2) == 0].sum(1), 0.5, atol=1e-14)
    assert np.allclose(phi[:, (j % 2) == 1].sum(1), 0.5, atol=1e-14)
    assert np.allclose((phi ** 2).sum(1), 3.0 / 8.0, atol=1e-14)
    assert np.all(coupling.peskin_phi(np.array([2.0, 2.5, -7.0])) == 0.0)


def _particles(npart, dim, n, clearance, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.uniform(0, 1, size=(npart, dim))
    X[:, -1] = rng.uniform(clearance / n, 1 - clearance / n, size=npart)
    return X


@pytest.mark.parametrize("dim,n", [(2, 16), (3, 8)])
def test_interpolation_reproduces_linear_fields(dim, n):
    s = grid.velocity_system(n, dim, levels=1)
    X = _particles(40, dim, n, clearance=2.5)
    # constant and x-linear fields (periodic direction: linear modulo wrap, so
    # keep particles away from the seam) are reproduced exactly away from walls
    X[:, 0] = np.random.default_rng(1).uniform(0.3, 0.7, size=X.shape[0])
    for c, cl in enumerate(s.levels[0]):
        from oracle.grid import component_offsets
        off = component_offsets(cl.comp, dim)[0]
        nz, ny, nx = cl.shape
        xnodes = (np.arange(nx) + off) / n
        u_const = [np.zeros(sh) for sh in s.shapes()]
        u_const[c][...] = 1.0
        u_lin = [np.zeros(sh) for sh in s.shapes()]
        u_lin[c][...] = xnodes[None, None, :]
        col = coupling.particle_columns(dim)[c]
        assert np.allclose(coupling.interpolate(s, u_const, X)[:, col], 1.0, atol=1e-13)
        assert np.allclose(coupling.interpolate(s, u_lin, X)[:, col], X[:, 0], atol=1e-13)


@pytest.mark.parametrize("dim,n", [(2, 16), (3, 8)])
def test_spread_is_adjoint_of_interpolation(dim, n):
    s = grid.velocity_system(n, dim, levels=1)
    rng = np.random.default_rng(3)
    X = _particles(25, dim, n, clearance=0.0, seed=4)   # includes near-wall particles
    F = rng.standard_normal(X.shape)
    u = [rng.standard_normal(sh) for sh in s.shapes()]
    lhs = np.sum(coupling.interpolate(s, u, X) * F)
    b = coupling.spread(s, F, X)
    rhs = sum(np.sum(uu * bb) for uu, bb in zip(u, b))
    assert lhs == pytest.approx(rhs, rel=1e-13)


def test_spread_total_force_away_from_walls():
    # sum of weights is 1 in each direction, so spreading conserves the force
    s = grid.velocity_system(16, 3, levels=1)
    X = _particles(10, 3, 16, clearance=2.5, seed=7)
    F = np.random.default_rng(8).standard_normal(X.shape)
    b = coupling.spread(s, F, X)
    assert np.allclose([bb.sum() for bb in b], F.sum(0), atol=1e-12)
