"""Pins for the discretization and the Galerkin hierarchy (oracle/grid.py)."""

import numpy as np
import pytest

from oracle import grid
from tests import closed_forms as cf


@pytest.mark.parametrize("kind", ["P", "V", "C", "N"])
@pytest.mark.parametrize("n", [4, 8, 16])
def test_1d_factor_eigenvalues(kind, n):
    K = grid.second_difference(kind, n)
    got = np.sort(np.linalg.eigvalsh(K))
    want = np.sort(cf.eigenvalues_1d(kind, n))
    assert np.allclose(got, want, atol=1e-12)


@pytest.mark.parametrize("dim,n", [(2, 8), (3, 4)])
def test_top_operator_matches_explicit_stencil(dim, n):
    s = grid.velocity_system(n, dim, mu=1.7, levels=1)
    rng = np.random.default_rng(0)
    for cl in s.levels[0]:
        v = rng.standard_normal(cl.shape)
        want = cf.stencil_apply_3d(cl.kinds, cl.scale, v)
        assert np.allclose(cl.apply(v), want, atol=1e-13)
    # scale = mu h^(d-2)
    assert s.scale == pytest.approx(1.7 * (1.0 / n) ** (dim - 2))


@pytest.mark.parametrize("dim,n", [(2, 6), (3, 4)])
def test_top_operator_spectrum(dim, n):
    s = grid.velocity_system(n, dim, levels=1)
    for cl in s.levels[0]:
        lam = [cf.eigenvalues_1d(k, n if k != "O" else 1) for k in cl.kinds]
        want = np.sort((lam[2][:, None, None] + lam[1][None, :, None]
                        + lam[0][None, None, :]).ravel() * cl.scale)
        got = np.sort(np.linalg.eigvalsh(cl.dense()))
        assert np.allclose(got, want, atol=1e-11)
        assert got.min() > 0  # SPD


@pytest.mark.parametrize("kind", ["P", "V", "C", "N"])
@pytest.mark.parametrize("nc", [1, 2, 3, 4, 8])
def test_prolongation_is_linear_interpolation(kind, nc):
    if kind == "V" and nc < 2:
        pytest.skip("no interior coarse node")
    P = grid.prolongation(kind, nc)
    assert np.allclose(P, cf.hat_prolongation(kind, nc), atol=1e-15)


def _dense_P(s, level, c):
    """Tensor-product interpolation from positions (independent of oracle P)."""
    cl = s.levels[level][c]
    mats = []
    for a in range(3):
        kind = cl.kinds[a]
        if kind == "O":
            mats.append(np.ones((1, 1)))
        else:
            mats.append(cf.hat_prolongation(kind, cl.ncells[a] // 2))
    return np.kron(mats[2], np.kron(mats[1], mats[0]))


@pytest.mark.parametrize("dim,n,levels", [(2, 16, 4), (3, 8, 3)])
@pytest.mark.parametrize("which", ["velocity", "pressure"])
def test_galerkin_coarse_operators(dim, n, levels, which):
    s = (grid.velocity_system(n, dim, mu=0.8, levels=levels) if which == "velocity"
         else grid.pressure_system(n, dim, levels=levels))
    for l in range(1, levels):
        for c in range(s.ncomp):
            P = _dense_P(s, l - 1, c)
            A_fine = s.levels[l - 1][c].dense()
            A_coarse = s.levels[l][c].dense()
            assert np.allclose(P.T @ A_fine @ P, A_coarse, atol=1e-12)


@pytest.mark.parametrize("dim,n,levels", [(2, 16, 3), (3, 8, 3)])
def test_restriction_is_transpose(dim, n, levels):
    s = grid.velocity_system(n, dim, levels=levels)
    rng = np.random.default_rng(2)
    for l in range(levels - 1):
        r = [rng.standard_normal(sh) for sh in s.shapes(l)]
        vc = [rng.standard_normal(sh) for sh in s.shapes(l + 1)]
        R = s.restrict(l, r)
        Pv = s.prolong(l, vc)
        for c in range(s.ncomp):
            P = _dense_P(s, l, c)
            assert np.allclose(R[c].ravel(), P.T @ r[c].ravel(), atol=1e-13)
            assert np.allclose(Pv[c].ravel(), P @ vc[c].ravel(), atol=1e-13)


def test_energy_identity():
    # E(P v) = 1/2 v^T A^(l) v - v^T b^(l) with A^(l) = P^T A P, b^(l) = P^T b
    # (the variational property of Section 3.2, Eq. equ_energy_v)
    s = grid.velocity_system(16, 2, levels=3)
    rng = np.random.default_rng(3)
    for c in range(s.ncomp):
        A = s.levels[0][c].dense()
        P = _dense_P(s, 0, c)
        b = rng.standard_normal(A.shape[0])
        v = rng.standard_normal(P.shape[1])
        x = P @ v
        E_fine = 0.5 * x @ A @ x - x @ b
        Ac = s.levels[1][c].dense()
        E_coarse = 0.5 * v @ Ac @ v - v @ (P.T @ b)
        assert E_fine == pytest.approx(E_coarse, rel=1e-12)


@pytest.mark.parametrize("dim,n,levels", [(2, 16, 4), (3, 8, 3)])
def test_colour_classes_partition_and_decouple(dim, n, levels):
    s = grid.velocity_system(n, dim, levels=levels)
    for l in range(levels):
        for cl in s.levels[l]:
            A = cl.dense()
            nz, ny, nx = cl.shape
            seen = np.zeros(cl.size, dtype=int)
            for colour, (k, j, i) in cl.colour_classes():
                flat = (k * ny + j) * nx + i
                seen[flat] += 1
                sub = A[np.ix_(flat, flat)]
                assert np.count_nonzero(sub - np.diag(np.diag(sub))) == 0
            assert np.all(seen == 1)


def test_coarse_level_counts_128():
    s = grid.velocity_system(128, 3)
    assert s.nlevels == 6
    assert s.shapes(0) == [(128, 128, 128), (128, 128, 128), (127, 128, 128)]
    assert s.shapes(5) == [(4, 4, 4), (4, 4, 4), (3, 4, 4)]
    s2 = grid.velocity_system(64, 2, levels=6)
    assert s2.shapes(0) == [(64, 1, 64), (63, 1, 64)]
    assert s2.shapes(5) == [(2, 1, 2), (1, 1, 2)]
