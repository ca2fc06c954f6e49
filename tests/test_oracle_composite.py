"""Pins of the composite-grid oracle (refined patch, Algorithms 1-2).

Each pin checks the oracle against something other than itself:
* the operator against a literal construction L = D G from the paper's
  divergence and gradient formulas (Section 4), cell by cell;
* symmetry and positive definiteness of A = -mu V L (reading R22);
* the closed form for a field linear in z (the coarse-fine gradient rule is
  exact on linear fields, so only the top-wall rows are non-zero);
* the Galerkin identity P^T A P = analytic base factors;
* exact invariance of N(A^-1 b, A^-1) under one stochastic FAC cycle
  (M A^-1 M^T + B B^T = A^-1, the paper's invariance claim, Section 3.2);
* the deterministic FAC solve against a sparse direct solve;
* validity of the patch pass order (no two coupled sites in one pass).
"""

import numpy as np
import pytest

from oracle import composite as C, multigrid
from oracle.philox import PhiloxNoise

from tests import affine


def literal_DG(cg):
    """-mu V L with L = D G built from the paper's formulas, cell by cell.

    Cells: fine cells (width h) and uncovered base cells (width H); the wall
    base cells (centre on the wall, value 0) and the covered base cells are not
    unknowns.  Gradient on a face between equal cells: difference over the
    spacing.  Across a coarse-fine face: on every one of the 2^(d-1) fine faces
    (mean of the fine values - coarse value) / ((3/4) H), oriented along +axis;
    the coarse face carries the mean of its fine faces.  Divergence of a cell:
    sum over its faces of area * G * outward sign, divided by the volume.
    """
    d, n, K, H, h, mu = cg.dim, cg.n, cg.K, cg.H, cg.h, cg.mu
    fz, fy, fx = cg.fine_shape
    bz, by, bx = cg.base_shape
    N = cg.size
    L = np.zeros((N, N))
    vol = np.zeros(N)

    def fine(m, q, p):
        return cg.fine_index(m, q % fy, p % fx)

    def base(r, l, i):
        return cg.base_index(r, l % by, i % bx)

    axes = [(0, 0, 1), (0, 1, 0)] if d == 3 else [(0, 0, 1)]   # in-plane offsets (dm, dq, dp)
    # fine cells
    for m in range(fz):
        for q in range(fy):
            for p in range(fx):
                row = fine(m, q, p)
                vol[row] = h ** d
                area = h ** (d - 1)
                # in-plane faces: neighbours at the same level
                for _, dq, dp in axes:
                    for sgn in (1, -1):
                        nb = fine(m, q + sgn * dq, p + sgn * dp)
                        # flux out = area * (c_nb - c_row) / h
                        L[row, nb] += area / h / vol[row]
                        L[row, row] -= area / h / vol[row]
                # z faces
                for sgn in (1, -1):
                    mm = m + sgn
                    if 0 <= mm < fz:
                        nb = fine(mm, q, p)
                        L[row, nb] += area / h / vol[row]
                        L[row, row] -= area / h / vol[row]
                        continue
                    # coarse-fine face: the group of siblings sharing the coarse neighbour
                    q0, p0 = (q // 2) * 2, (p // 2) * 2
                    sibs = [fine(m, q0 + a, p0 + c) for a in (range(2) if d == 3 else [0]) for c in range(2)]
                    coarse = None if sgn < 0 else base(K, q // 2, p // 2)
                    # G along +z at this fine face
                    g = {}
                    if sgn > 0:     # coarse above: G = (c_A - mean(fine)) / (3/4 H)
                        g[coarse] = g.get(coarse, 0.0) + 1.0 / (0.75 * H)
                        for s_ in sibs:
                            g[s_] = g.get(s_, 0.0) - 1.0 / len(sibs) / (0.75 * H)
                    else:           # wall below: G = (mean(fine) - 0) / (3/4 H)
                        for s_ in sibs:
                            g[s_] = g.get(s_, 0.0) + 1.0 / len(sibs) / (0.75 * H)
                    for col, val in g.items():
                        L[row, col] += sgn * area * val / vol[row]
    # uncovered base cells
    for r in range(K, bz):
        for l in range(by):
            for i in range(bx):
                row = base(r, l, i)
                vol[row] = H ** d
                area = H ** (d - 1)
                for _, dq, dp in axes:
                    for sgn in (1, -1):
                        nb = base(r, l + sgn * dq, i + sgn * dp)
                        L[row, nb] += area / H / vol[row]
                        L[row, row] -= area / H / vol[row]
                # above: base row or the top wall (value 0)
                if r + 1 < bz:
                    L[row, base(r + 1, l, i)] += area / H / vol[row]
                L[row, row] -= area / H / vol[row]
                # below: base row or the patch (coarse face = mean of the fine faces)
                if r > K:
                    L[row, base(r - 1, l, i)] += area / H / vol[row]
                    L[row, row] -= area / H / vol[row]
                else:
                    sibs = [fine(fz - 1, 2 * l + a, 2 * i + c) for a in (range(2) if d == 3 else [0]) for c in range(2)]
                    # G along +z = (c_A - mean(fine)) / (3/4 H); outward normal of the bottom face is -z
                    L[row, row] -= area / (0.75 * H) / vol[row]
                    for s_ in sibs:
                        L[row, s_] += area / len(sibs) / (0.75 * H) / vol[row]
    return -mu * vol[:, None] * L


GEOMS = [(2, 8, 2), (2, 8, 1), (3, 4, 1), (3, 8, 2)]


@pytest.mark.parametrize("dim,n,K", GEOMS)
def test_operator_is_literal_DG(dim, n, K):
    cg = C.CompositeGrid(n, K, dim, mu=1.7)
    ref = literal_DG(cg)
    A = cg.A.toarray()
    assert np.abs(A - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("dim,n,K", GEOMS)
def test_symmetric_positive_definite(dim, n, K):
    cg = C.CompositeGrid(n, K, dim, mu=0.9)
    A = cg.A.toarray()
    assert np.array_equal(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0.0


@pytest.mark.parametrize("dim,n,K", GEOMS + [(3, 16, 3)])
def test_linear_field_closed_form(dim, n, K):
    """c = z: the rows vanish except the top-wall rows, which equal mu H^(d-2)."""
    mu = 1.3
    cg = C.CompositeGrid(n, K, dim, mu=mu)
    Az = cg.A @ C.cell_centres_z(cg)
    bz, by, bx = cg.base_shape
    top = np.array([cg.base_index(bz - 1, l, i) for l in range(by) for i in range(bx)])
    mask = np.ones(cg.size, bool)
    mask[top] = False
    assert np.abs(Az[mask]).max() < 1e-13
    assert np.allclose(Az[top], mu * cg.H ** (dim - 2), rtol=1e-13)


@pytest.mark.parametrize("dim,n,K", GEOMS + [(3, 16, 3)])
def test_galerkin_base_operator(dim, n, K):
    cg = C.CompositeGrid(n, K, dim, mu=1.1)
    Ab = (cg.P.T @ cg.A @ cg.P).toarray()
    assert np.abs(Ab - cg.base.levels[1][0].dense()).max() <= 1e-13 * np.abs(Ab).max()


def test_prolongation_is_parent_copy_and_restriction_its_transpose():
    cg = C.CompositeGrid(8, 2, 3)
    rng = np.random.default_rng(3)
    base = rng.standard_normal(cg.base_shape)
    fine, b2 = cg.from_vec(cg.prolong(base))
    assert np.array_equal(fine, np.repeat(np.repeat(np.repeat(base[:2], 2, 0), 2, 1), 2, 2))
    assert np.array_equal(b2[2:], base[2:])
    v = rng.standard_normal(cg.size)
    assert np.isclose(v @ cg.prolong(base), np.sum(cg.restrict(v) * base), rtol=1e-13)


@pytest.mark.parametrize("dim,n,K", [(2, 8, 2), (3, 8, 1)])
def test_patch_passes_are_valid_gibbs_order(dim, n, K):
    cg = C.CompositeGrid(n, K, dim)
    sets = cg.pass_sets()
    allidx = np.sort(np.concatenate(sets))
    assert np.array_equal(allidx, np.arange(cg.n_fine))
    A = cg.A.tocsr()
    for idx in sets:
        sub = A[idx][:, idx].toarray()
        assert np.count_nonzero(sub - np.diag(np.diag(sub))) == 0


@pytest.mark.parametrize("coarse_mode", ["cholesky", "smooth"])
def test_stochastic_fac_keeps_the_gaussian_invariant(coarse_mode):
    cg = C.CompositeGrid(8, 2, 2, mu=0.7)
    coarsest = multigrid.Coarsest(cg.base)

    def step(z, b, noise):
        zz = [z[0].copy()]
        C.fac_cycle(cg, zz, [b[0]], noise, 1.0, coarse_mode=coarse_mode, coarsest=coarsest)
        return zz

    M, N, B, c = affine.extract(step, [(cg.size,)])
    Ainv = np.linalg.inv(cg.A.toarray())
    assert np.abs(M @ Ainv @ M.T + B @ B.T - Ainv).max() <= 1e-12 * np.abs(Ainv).max()
    assert np.abs((np.eye(cg.size) - M) @ Ainv - N).max() <= 1e-12 * np.abs(N).max()
    assert np.abs(np.linalg.eigvals(M)).max() < 0.5     # it contracts


@pytest.mark.parametrize("dim,n,K", [(2, 16, 3), (3, 8, 2)])
def test_deterministic_fac_solve_matches_direct_solve(dim, n, K):
    cg = C.CompositeGrid(n, K, dim, ncomp=2)
    rng = np.random.default_rng(5)
    b = [rng.standard_normal(cg.size) for _ in range(2)]
    z, cycles, rel = C.solve(cg, b, tol=1e-10)
    ref = C.direct_solve(cg, b)
    assert rel <= 1e-10 and cycles < 60
    for a, r in zip(z, ref):
        assert np.abs(a - r).max() <= 1e-8 * np.abs(r).max()


def test_patch_noise_stream_is_indexed_by_site():
    """Patch normals depend on the linear index only through (index >> 2, index & 3)."""
    nz = PhiloxNoise(4, 1, 9)
    idx = np.array([0, 1, 2, 3, 4, 9, 17])
    a = nz.patch(1, 2, 0, idx)
    b = np.concatenate([nz.patch(1, 2, 0, np.array([i])) for i in idx])
    assert np.array_equal(a, b)
    assert not np.array_equal(nz.patch(1, 3, 0, idx), a)


def test_probe_block_script_matches_dense_inverse():
    """The stored probe covariance of the composite sampler is written by
    tests/golden/make_composite_probe_cov.py from ten FAC solves and the grid's
    translation invariance.  On a small grid its block equals the block of
    the dense inverse of the composite operator (Section 3: the chain samples
    N(0, A^-1)), so the shift bookkeeping and the probe addressing are right."""
    import os
    import sys
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
    import make_composite_probe_cov as mk
    n, K = 8, 2
    B = mk.block(n, K)
    cg = C.CompositeGrid(n, K, 3, mu=1.0, ncomp=1)
    Ainv = np.linalg.inv(cg.A.toarray())
    idx = [cg.fine_index(z, y, x) if part == 0 else cg.base_index(z, y, x) for part, z, y, x in mk.probe_sites(n, K)]
    want = Ainv[np.ix_(idx, idx)]
    assert np.abs(B - want).max() < 1e-7 * np.abs(want).max()
    assert np.abs(B - B.T).max() < 1e-7 * np.abs(want).max()
