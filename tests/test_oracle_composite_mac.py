"""Pins for the composite MAC divergence, gradient and projection (oracle/composite_mac.py).

* The two uniform limits (no refined rows, every row refined) equal the
  uniform MAC projection of oracle/projection.py (pinned on its own).
* A pressure linear in z: L z vanishes in every cell but the wall cells,
  where it is +1/h (bottom, fine) and -1/H (top, base) -- the interface
  rule with the (3/4) H distance is exact on linear fields.
* A pressure that depends on z only reduces L to a 1-D operator on the
  column of 2K fine and n-K base cells, built here by hand.
* sum |c| p (D u) = - sum w_f u_f (G p); V L is symmetric negative
  semidefinite with the constants as its kernel.
* P~ is idempotent, W-symmetric, leaves divergence-free fields alone,
  annihilates gradients, and its output is divergence-free.
* A planted slip (distance H instead of (3/4) H across the interface) breaks
  the linear-field closed form.
"""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import projection
from oracle.composite_mac import CompositeMAC


def _to_components(g, u):
    """Face vector of a uniform composite (K = 0 or K = n) -> [u, (v), w] arrays."""
    nz, ny, nx = g.fine_shape if g.K == g.n else g.base_shape
    comps = [np.zeros((nz, ny, nx)) for _ in range(g.dim - 1)] + [np.zeros((nz - 1, ny, nx))]
    shape = (nz, ny, nx)
    off = 0 if g.K == g.n else g.n_fine
    for f, (axis, plus, minus, area, dist, _) in enumerate(g.faces):
        k, j, i = np.unravel_index(plus - off, shape)
        if axis == 2:
            comps[-1][k - 1, j, i] = u[f]
        else:
            comps[axis if g.dim == 3 else 0][k, j, i] = u[f]
    return comps


@pytest.mark.parametrize("dim,n,K", [(2, 8, 0), (2, 8, 8), (3, 4, 0), (3, 4, 4)])
def test_uniform_limits_match_uniform_projection(dim, n, K):
    g = CompositeMAC(n, K, dim)
    rng = np.random.default_rng(1)
    u = rng.standard_normal(g.n_faces)
    got = _to_components(g, g.project(u))
    want = projection.Projector(n if K == 0 else 2 * n, dim, tol=1e-13).project(_to_components(g, u))
    for a, b in zip(got, want):
        assert np.abs(a - b).max() < 1e-10


@pytest.mark.parametrize("dim,n,K", [(2, 8, 3), (3, 4, 1), (3, 8, 3), (2, 16, 1)])
def test_linear_pressure_closed_form(dim, n, K):
    g = CompositeMAC(n, K, dim)
    z = g.cell_centres()[:, 2]
    Lz = g.laplacian() @ z
    want = np.zeros(g.n_cells)
    nz, ny, nx = g.fine_shape
    want[:ny * nx] = 1.0 / g.h                               # fine cells on the bottom wall
    bz, by, bx = g.base_shape
    want[g.n_cells - by * bx:] = -1.0 / g.H                  # base cells under the top wall
    assert np.abs(Lz - want).max() < 1e-10 * (1.0 / g.h)


def _column_operator(n, K):
    """1-D L on a z-column: 2K fine cells (height h), then n-K base cells (H)."""
    H, h = 1.0 / n, 0.5 / n
    heights = [h] * (2 * K) + [H] * (n - K)
    N = len(heights)
    L = np.zeros((N, N))
    for k in range(N - 1):               # face between cells k and k+1, centres dist apart
        dist = 0.5 * (heights[k] + heights[k + 1])
        for a, b in ((k, k + 1), (k + 1, k)):
            L[a, b] += 1.0 / dist / heights[a]
            L[a, a] -= 1.0 / dist / heights[a]
    return L


@pytest.mark.parametrize("dim,n,K", [(2, 8, 3), (3, 8, 2), (2, 16, 5)])
def test_z_only_fields_reduce_to_the_column_operator(dim, n, K):
    g = CompositeMAC(n, K, dim)
    rng = np.random.default_rng(2)
    col = rng.standard_normal(2 * K + n - K)
    zc = g.cell_centres()[:, 2]
    heights_z = np.concatenate([(np.arange(2 * K) + 0.5) * g.h, (np.arange(K, n) + 0.5) * g.H])
    idx = np.array([np.argmin(np.abs(heights_z - z)) for z in zc])
    p = col[idx]
    got = g.laplacian() @ p
    want = (_column_operator(n, K) @ col)[idx]
    assert np.abs(got - want).max() < 1e-10 * np.abs(want).max()


@pytest.mark.parametrize("dim,n,K", [(2, 8, 3), (3, 4, 1)])
def test_adjoint_symmetric_semidefinite(dim, n, K):
    g = CompositeMAC(n, K, dim)
    rng = np.random.default_rng(3)
    u, p = rng.standard_normal(g.n_faces), rng.standard_normal(g.n_cells)
    lhs = g.vol @ (p * (g.D @ u))
    rhs = -(g.weight * u) @ (g.G @ p)
    assert abs(lhs - rhs) < 1e-13 * (abs(lhs) + 1.0)
    S = (sp.diags(g.vol) @ g.laplacian()).toarray()
    assert np.abs(S - S.T).max() < 1e-13 * np.abs(S).max()
    ev = np.linalg.eigvalsh(S)
    assert ev[-1] < 1e-12 * np.abs(ev).max() and abs(ev[-1]) < 1e-12 * np.abs(ev).max()
    assert ev[-2] < -1e-6 * np.abs(ev).max()                  # one-dimensional kernel
    assert np.abs(S @ np.ones(g.n_cells)).max() < 1e-12 * np.abs(S).max()


@pytest.mark.parametrize("dim,n,K", [(2, 8, 3), (3, 4, 1), (3, 8, 3)])
def test_projection_properties(dim, n, K):
    g = CompositeMAC(n, K, dim)
    rng = np.random.default_rng(4)
    u, v = rng.standard_normal(g.n_faces), rng.standard_normal(g.n_faces)
    pu, pv = g.project(u), g.project(v)
    scale = np.abs(u).max()
    assert np.abs(g.D @ pu).max() < 1e-10 * scale / g.h
    assert np.abs(g.project(pu) - pu).max() < 1e-11 * scale
    assert abs((g.weight * pu) @ v - (g.weight * u) @ pv) < 1e-12 * np.abs(g.weight * u).sum() * scale
    grad = g.G @ rng.standard_normal(g.n_cells)
    assert np.abs(g.project(grad)).max() < 1e-10 * np.abs(grad).max()
    flow = np.array([1.0 if f[0] == 0 else 0.0 for f in g.faces])   # uniform x-flow
    assert np.abs(g.D @ flow).max() < 1e-12
    assert np.abs(g.project(flow) - flow).max() < 1e-11


def test_wrong_interface_distance_is_caught():
    g = CompositeMAC(8, 3, 2)
    g.faces = [f if f[4] != 0.75 * g.H else f[:4] + (g.H,) + f[5:] for f in g.faces]
    g.dist = np.array([f[4] for f in g.faces])
    g.G = g._gradient()
    z = g.cell_centres()[:, 2]
    Lz = g.laplacian() @ z
    interior = np.ones(g.n_cells, bool)
    nz, ny, nx = g.fine_shape
    interior[:ny * nx] = False
    bz, by, bx = g.base_shape
    interior[g.n_cells - by * bx:] = False
    assert np.abs(Lz[interior]).max() > 1.0


# ---- velocity operators on the staggered composite grid (reading R22) ----

from oracle import grid  # noqa: E402


def _uniform_velocity(g, mu):
    """Dense uniform velocity operator of grid.py, mapped to the composite's face order."""
    N = g.n if g.K == 0 else 2 * g.n
    osys = grid.velocity_system(N, g.dim, mu=mu, levels=1)
    comps = [cl.dense() for cl in osys.levels[0]]
    shapes = [cl.shape for cl in osys.levels[0]]
    index = []
    for axis, plus, minus, area, dist, key in g.faces:
        _, lev, k, j, i = key
        c = axis if g.dim == 3 else (0 if axis == 0 else 1)
        nz, ny, nx = shapes[c]
        kk = k - 1 if axis == 2 else k
        index.append((c, (kk * ny + (j if g.dim == 3 else 0)) * nx + i))
    A = np.zeros((g.n_faces, g.n_faces))
    for a, (ca, ia) in enumerate(index):
        for b, (cb, ib) in enumerate(index):
            if ca == cb:
                A[a, b] = comps[ca][ia, ib]
    return A


@pytest.mark.parametrize("dim,n,K", [(2, 8, 0), (2, 8, 8), (3, 4, 0), (3, 4, 4)])
def test_velocity_uniform_limits_match_grid_operator(dim, n, K):
    g = CompositeMAC(n, K, dim)
    A = g.velocity_operator(mu=0.7).toarray()
    assert np.abs(A - _uniform_velocity(g, 0.7)).max() < 1e-13 * np.abs(A).max()


@pytest.mark.parametrize("dim,n,K", [(2, 8, 3), (3, 4, 1), (3, 8, 3), (2, 16, 1)])
def test_velocity_linear_field_closed_form(dim, n, K):
    # u = z: every row vanishes but the rows under the top wall, where the
    # cell-type components give 2 mu H^(d-2) and the wall-normal one mu H^(d-2)
    mu = 1.3
    g = CompositeMAC(n, K, dim)
    pos = g.face_positions()
    Az = g.velocity_operator(mu) @ pos[:, 2]
    want = np.zeros(g.n_faces)
    for f, (axis, plus, minus, area, dist, key) in enumerate(g.faces):
        top = abs(pos[f, 2] - (1.0 - (g.H if axis == 2 else 0.5 * g.H))) < 1e-12
        if top:
            want[f] = mu * g.H ** (dim - 2) * (1.0 if axis == 2 else 2.0)
    assert np.abs(Az - want).max() < 1e-12 * mu * g.H ** (dim - 2)


def _column(positions):
    """1-D operator on nodes at the given heights, Dirichlet 0 at z = 0 and z = 1:
    row k = sum over the neighbours of (u_k - u_nb) / distance."""
    zs = [0.0] + list(positions) + [1.0]
    N = len(positions)
    A = np.zeros((N, N))
    for k in range(N):
        for nb in (k - 1, k + 1):
            dist = abs(zs[k + 1] - zs[nb + 1])
            A[k, k] += 1.0 / dist
            if 0 <= nb < N:
                A[k, nb] -= 1.0 / dist
    return A


@pytest.mark.parametrize("dim,n,K", [(2, 8, 3), (3, 8, 2), (2, 16, 5), (3, 4, 1)])
def test_velocity_z_only_fields_reduce_to_column_operators(dim, n, K):
    # For a field that varies along z only, a row of A is the node's box face
    # area times a row of the 1-D operator on its column (distances between
    # consecutive node heights, walls at 0 and 1).
    g = CompositeMAC(n, K, dim)
    pos = g.face_positions()
    A = g.velocity_operator(1.0)
    rng = np.random.default_rng(5)
    for axis in ([0, 1] if dim == 3 else [0]) + [2]:
        sel = np.array([f[0] == axis for f in g.faces])
        heights = np.unique(np.round(pos[sel, 2], 12))
        col = rng.standard_normal(heights.size)
        u = np.zeros(g.n_faces)
        k_of = np.searchsorted(heights, np.round(pos[:, 2], 12))
        u[sel] = col[k_of[sel]]
        got = (A @ u)[sel]
        area = np.where(pos[sel, 2] < g.K * g.H - 1e-12, g.h, g.H) ** (dim - 1)
        want = area * (_column(heights) @ col)[k_of[sel]]
        assert np.abs(got - want).max() < 1e-11 * np.abs(want).max(), axis


@pytest.mark.parametrize("dim,n,K", [(2, 8, 3), (3, 4, 1)])
def test_interface_group_weights(dim, n, K):
    # each group's weights sum to 1 and reproduce its base node's position along
    # x and y (first moments, periodic distances); every fine node of the row
    # below is covered by the groups with its own box-face area
    g = CompositeMAC(n, K, dim)
    pos = g.face_positions()
    for axis in ([0, 1] if dim == 3 else [0]) + [2]:
        cover = {}
        for c, fine, dist in g.interface_groups(axis):
            w = np.array([x for _, x in fine])
            assert abs(w.sum() - 1.0) < 1e-15
            for ax in ([0, 1] if dim == 3 else [0]):
                dx = np.array([(pos[f, ax] - pos[c, ax] + 0.5) % 1.0 - 0.5 for f, _ in fine])
                assert abs(w @ dx) < 1e-15
            for f, x in fine:
                cover[f] = cover.get(f, 0.0) + x * g.H ** (dim - 1)
        assert cover and all(abs(v - g.h ** (dim - 1)) < 1e-15 for v in cover.values())


@pytest.mark.parametrize("dim,n,K", [(2, 8, 3), (3, 4, 1)])
def test_velocity_operator_symmetric_positive_definite(dim, n, K):
    A = CompositeMAC(n, K, dim).velocity_operator(0.9).toarray()
    assert np.abs(A - A.T).max() == 0.0
    assert np.linalg.eigvalsh(A)[0] > 0.0


def test_velocity_wrong_group_distance_is_caught():
    g = CompositeMAC(8, 3, 2)
    orig = g.interface_groups
    g.interface_groups = lambda a: [(c, f, g.H if a != 2 else d) for c, f, d in orig(a)]
    Az = g.velocity_operator(1.0) @ g.face_positions()[:, 2]
    below_top = g.face_positions()[:, 2] < 1.0 - g.H
    assert np.abs(Az[below_top]).max() > 0.2 * g.H          # (1/4) H^(d-1) at the interface rows


# ---- stochastic FAC on the staggered composite grid (reading R23) ----

import scipy.sparse.linalg as spla  # noqa: E402

from oracle.composite_mac import CompositeMACFAC  # noqa: E402
from tests.affine import extract  # noqa: E402


def _affine(F):
    def step(z, b, noise):
        return [F.fac_cycle(z[0].copy(), b[0], noise, 1.0)]
    return extract(step, [(F.g.n_faces,)])


@pytest.mark.parametrize("dim,n,K", [(2, 4, 1), (2, 8, 2), (3, 4, 1)])
def test_composite_mac_cycle_invariance_exact(dim, n, K):
    # the paper's claim (Section 3.2) for the composite cycle: N(A^-1 b, A^-1)
    # is invariant, A^-1 = M A^-1 M^T + B B^T, and A^-1 b is the fixed point
    F = CompositeMACFAC(CompositeMAC(n, K, dim), mu=0.8)
    M, N, B, c = _affine(F)
    C = np.linalg.inv(F.A.toarray())
    assert np.abs(M @ C @ M.T + B @ B.T - C).max() < 1e-12 * np.abs(C).max()
    b = np.random.default_rng(6).standard_normal(C.shape[0])
    x = C @ b
    assert np.abs(M @ x + N @ b + c - x).max() < 1e-11 * np.abs(x).max()
    assert np.max(np.abs(np.linalg.eigvals(M))) < 0.5


def test_composite_mac_wrong_restriction_breaks_invariance():
    # A plausible slip: the residual restricted by P^T / 2 while the base
    # operator stays the Galerkin P^T A P.
    F = CompositeMACFAC(CompositeMAC(4, 1, 2))

    def cycle(z, b, noise, sigma, mu1=2, mu2=2, nu=2):
        r = b - F.A @ z
        qb = np.zeros(F.P.shape[1])
        F.vcycle(0, qb, 0.5 * (F.P.T @ r), noise, sigma, mu1, mu2)
        q = F.P @ qb
        diag = F.A.diagonal()
        for s in range(nu):
            for colour, idx in enumerate(F.patch_colours):
                off = F.A[idx] @ q - diag[idx] * q[idx]
                q[idx] = (r[idx] - off) / diag[idx] + sigma * noise.patch(0, colour, s, idx) / np.sqrt(diag[idx])
        return z + q

    F.fac_cycle = cycle
    M, N, B, c = _affine(F)
    C = np.linalg.inv(F.A.toarray())
    assert np.abs(M @ C @ M.T + B @ B.T - C).max() > 1e-4 * np.abs(C).max()


@pytest.mark.parametrize("dim,n,K", [(2, 16, 4), (3, 8, 2)])
def test_composite_mac_solve_matches_direct(dim, n, K):
    F = CompositeMACFAC(CompositeMAC(n, K, dim), mu=1.2)
    b = np.random.default_rng(7).standard_normal(F.g.n_faces)
    z, cycles, rel = F.solve(b, tol=1e-11)
    assert rel <= 1e-11 and cycles <= 20
    x = spla.spsolve(F.A.tocsc(), b)
    assert np.linalg.norm(z - x) / np.linalg.norm(x) < 1e-9


@pytest.mark.parametrize("dim,n,K", [(2, 16, 5), (3, 8, 3), (3, 16, 4)])
def test_colour_classes_are_independent_sets(dim, n, K):
    # Every class of every level is an independent set of the operator's graph
    # (no coupling between two sites of one class), and the graph threshold
    # separates couplings from rounding residues by many orders of magnitude,
    # so the classes cannot depend on the summation order of the products.
    from oracle.composite_mac import GRAPH_RTOL
    F = CompositeMACFAC(CompositeMAC(n, K, dim))
    levels = [(A, cl) for A, cl in zip(F.ops, F.colours)] + [(F.A, F.patch_colours)]
    for A, classes in levels:
        A = A.tocsr()
        d = np.abs(A.diagonal())
        rel = np.abs(A.multiply(sp.csr_matrix(1.0 / d[:, None]))).tocsr()
        rel.setdiag(0.0)
        vals = rel.data[rel.data > 0]
        assert not np.any((vals > 1e3 * GRAPH_RTOL) & (vals < 1e-6))
        assert sorted(np.concatenate(classes).tolist()) == sorted(set(np.concatenate(classes).tolist()))
        for idx in classes:
            blk = rel[idx][:, idx]
            assert blk.max() <= GRAPH_RTOL if blk.nnz else True


def test_more_than_sixteen_colours_keep_distinct_streams():
    # 3-D Galerkin levels of the composite grid need more than 16 classes;
    # colours 16.. continue in the counter's top byte, colours below 16 keep
    # the counters of the uniform levels.
    from oracle import philox
    F = CompositeMACFAC(CompositeMAC(8, 3, 3))
    assert len(F.colours[0]) > 16
    c1 = {philox.pack_ctr1(1, 0, c, 0, 0) for c in range(40)}
    assert len(c1) == 40
    assert philox.pack_ctr1(2, 1, 3, 1, 0) == 2 | (1 << 4) | (3 << 8) | (1 << 12)
    assert philox.pack_ctr1(1, 0, 17, 2, 0) == 1 | (1 << 8) | (2 << 12) | (1 << 24)


# ---- particles on the composite MAC grid (reading R24) ----

from oracle import selm as oselm  # noqa: E402
from oracle.composite_mac import CompositeSELM  # noqa: E402

PARTICLES_2D = np.array([[0.31, 0.42], [0.77, 0.58], [0.12, 0.2]])


@pytest.mark.parametrize("K", [0, 8])
@pytest.mark.parametrize("project", [False, True])
def test_composite_selm_uniform_limits(K, project):
    # no row refined: the base grid's SELM; every row refined: the fine grid's
    n = 8
    cs = CompositeSELM(n, K, 2, mu=0.9, project=project, kernel="cover")
    M = cs.mobility_matrix(PARTICLES_2D)
    m = oselm.Model(n if K == 0 else 2 * n, 2, mu=0.9, project=project, tol=1e-13)
    Mu = m.mobility_matrix(PARTICLES_2D)
    assert np.abs(M - Mu).max() < 1e-10 * np.abs(Mu).max()
    if K == 8:
        Mf = CompositeSELM(n, K, 2, mu=0.9, project=project, kernel="fine").mobility_matrix(PARTICLES_2D)
        assert np.abs(Mf - Mu).max() < 1e-10 * np.abs(Mu).max()


@pytest.mark.parametrize("kernel", ["cover", "fine"])
def test_composite_interpolation_reproduces_linear_fields(kernel):
    # away from the walls Gamma reproduces fields linear in z on both sides of
    # the interface and across it (R and E are exact on them)
    n, K = 16, 6
    cs = CompositeSELM(n, K, 2, kernel=kernel)
    pos = cs.g.face_positions()
    u = np.where([f[0] == 0 for f in cs.g.faces], 0.3 + 2 * pos[:, 2], -1 + 0.5 * pos[:, 2])
    zs = np.linspace((K - 3) / n, (K + 3) / n, 25)
    X = np.column_stack([np.full(zs.size, 0.37), zs])
    U = (cs.interpolation(X) @ u).reshape(-1, 2)
    assert np.abs(U[:, 0] - (0.3 + 2 * zs)).max() < 1e-13
    assert np.abs(U[:, 1] - (-1 + 0.5 * zs)).max() < 1e-13


@pytest.mark.parametrize("project", [False, True])
def test_composite_fluctuation_dissipation(project):
    # K A^-1 K^T = 2 kT M with K = sqrt(2 kT) Gamma P~ (Eq. equ_G_special_form)
    cs = CompositeSELM(8, 3, 2, mu=0.8, kT=1.7, project=project, kernel="fine")
    X = np.array([[0.3, 0.33], [0.6, 0.41], [0.45, 0.7]])       # below, at and above the interface
    M = cs.mobility_matrix(X)
    Kt = cs.thermal_operator(X)
    G = Kt @ np.linalg.inv(cs.fac.A.toarray()) @ Kt.T
    assert np.abs(G - 2 * cs.kT * M).max() < 1e-9 * np.abs(G).max()
    assert np.abs(M - M.T).max() < 1e-10 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


def test_fine_kernel_mobility_is_continuous_across_the_interface():
    # The particle keeps its kernel (its size) when it crosses the interface:
    # between sample heights H/4 apart its self-mobility changes by at most 5 %
    # (about 2 % per step from the wall effect below, a dip of 4 % at the
    # interface, lattice ripples of 1-2 % above).  Switching to the coarse
    # kernel above the interface ("cover") makes it jump by about a fifth.
    n, K = 16, 6
    zz = np.linspace((K - 2.5) / n, (K + 2.5) / n, 21)
    steps = {}
    for kernel in ("fine", "cover"):
        cs = CompositeSELM(n, K, 2, kernel=kernel)
        vals = np.array([np.diag(cs.mobility_matrix(np.array([[0.37, z]]))) for z in zz])
        steps[kernel] = np.abs(np.diff(vals, axis=0)) / vals.mean(0)
    assert steps["fine"].max() < 0.05
    assert steps["cover"].max() > 0.15 and steps["cover"].max() > 4 * steps["fine"].max()


@pytest.mark.parametrize("K", [0, 4])
@pytest.mark.parametrize("project", [False, True])
def test_composite_selm_uniform_limits_3d(K, project):
    X = np.array([[0.31, 0.42, 0.55], [0.77, 0.58, 0.3]])
    M = CompositeSELM(4, K, 3, mu=0.9, project=project, kernel="cover").mobility_matrix(X)
    Mu = oselm.Model(4 if K == 0 else 8, 3, mu=0.9, project=project, tol=1e-13).mobility_matrix(X)
    assert np.abs(M - Mu).max() < 1e-10 * np.abs(Mu).max()


@pytest.mark.parametrize("project", [False, True])
def test_composite_em_step_uniform_limit(project):
    # No row refined and the covering level's kernel: one deterministic
    # Euler-Maruyama step (kT = 0) moves the particles as the uniform grid's
    # step does (Algorithm 4 on the base grid); both solves stop at 1e-12.
    n = 8
    X = PARTICLES_2D.copy()
    F = np.array([[1.0, -0.4], [0.2, 0.7], [-0.5, 0.3]])
    cs = CompositeSELM(n, 0, 2, mu=0.9, kT=0.0, project=project, kernel="cover", tol=1e-12)
    Xc, _ = cs.em_step(X, F, 0.05, 2)
    m = oselm.Model(n, 2, mu=0.9, kT=0.0, project=project, tol=1e-12)
    Xu, _ = m.em_step(X, F, 0.05, 2)
    assert np.abs(Xc - Xu).max() < 1e-9 * np.abs(Xu - X).max()


def test_composite_em_step_deterministic_part_is_the_mobility():
    # kT = 0: the step is X + dt M F (before wrapping), M from unit-force solves.
    cs = CompositeSELM(8, 3, 2, mu=0.8, kT=0.0, project=True, tol=1e-12)
    X = np.array([[0.3, 0.33], [0.6, 0.41], [0.45, 0.7]])
    F = np.array([[0.5, -1.0], [0.1, 0.4], [-0.3, 0.2]])
    Xn, _ = cs.em_step(X, F, 0.01, 1)
    M = cs.mobility_matrix(X, tol=1e-12)
    assert np.abs((Xn - X).ravel() - 0.01 * M @ F.ravel()).max() < 1e-9 * np.abs(Xn - X).max()
