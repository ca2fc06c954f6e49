"""GPU parity of the staggered composite grid (selm_mac.h) against the oracle.

The oracle (oracle/composite_mac.py, readings R21-R24) defines the composite
MAC operators, the projection, the stochastic FAC cycle (Algorithms 1-3 with
first-fit colour classes and Philox noise) and the particle coupling with
its Euler-Maruyama step (Algorithm 4).  Each CUDA entry point is compared
with it on the same seeded inputs: FP64 to 1e-12, FP32 inner cycles to 1e-5,
as field norms and element by element (max |a - b| / max |b|).
"""

import numpy as np
import pytest
import torch

from oracle.composite_mac import CompositeMAC, CompositeMACFAC, CompositeSELM
from oracle.philox import ExplicitNoise, PhiloxNoise
from tests.gpu_util import maxrel, rel

pytestmark = pytest.mark.gpu

GRIDS = [(2, 16, 5), (3, 8, 3), (3, 16, 4)]
EDGE = [(2, 8, 0), (2, 8, 8), (3, 8, 1)]          # no row refined, every row refined, one refined row


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_2680_gb300 import selm as mod
    mod.lib()
    return mod


_ORACLE = {}


def _fac(dim, n, K, mu):
    key = (dim, n, K, mu)
    if key not in _ORACLE:
        _ORACLE[key] = CompositeMACFAC(CompositeMAC(n, K, dim), mu=mu)
    return _ORACLE[key]


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _host(t):
    return t.double().cpu().numpy()


def _tol(prec, S):
    return 1e-12 if prec == S.SELM_FP64 else 1e-5


def _handle(S, dim, n, K, mu=0.9, prec=None, **kw):
    prec = S.SELM_FP64 if prec is None else prec
    return S.selm_mac_create(S.make_mac_desc(dim, n, K, mu=mu, precision=prec, **kw))


@pytest.mark.parametrize("dim,n,K", GRIDS + EDGE)
def test_operators(S, dim, n, K):
    F = _fac(dim, n, K, 0.9)
    g = F.g
    h = _handle(S, dim, n, K)
    try:
        rng = np.random.default_rng(1)
        u = rng.standard_normal(g.n_faces)
        p = rng.standard_normal(g.n_cells)
        Au = torch.zeros(g.n_faces, dtype=torch.float64, device="cuda")
        div = torch.zeros(g.n_cells, dtype=torch.float64, device="cuda")
        grad = torch.zeros(g.n_faces, dtype=torch.float64, device="cuda")
        assert S.selm_mac_faces(h) == g.n_faces and S.selm_mac_cells(h) == g.n_cells
        S.selm_mac_apply(h, _dev(u), Au)
        S.selm_mac_divergence(h, _dev(u), div)
        S.selm_mac_gradient(h, _dev(p), grad)
        for got, want in ((Au, F.A @ u), (div, g.D @ u), (grad, g.G @ p)):
            assert maxrel(_host(got), want) < 1e-13
    finally:
        S.selm_mac_destroy(h)


@pytest.mark.parametrize("dim,n,K", GRIDS + EDGE)
@pytest.mark.parametrize("adjoint", [0, 1])
def test_projection(S, dim, n, K, adjoint):
    g = _fac(dim, n, K, 0.9).g
    h = _handle(S, dim, n, K, proj_tol=1e-14)
    try:
        u = np.random.default_rng(2).standard_normal(g.n_faces)
        out = torch.zeros(g.n_faces, dtype=torch.float64, device="cuda")
        it, res = S.selm_mac_project(h, _dev(u), out, adjoint=bool(adjoint))
        want = g.project(u) if not adjoint else g.weight * g.project(u / g.weight)
        got = _host(out)
        assert rel(got, want) < 1e-12 and maxrel(got, want) < 1e-12, (it, res)
        # projected fields are discretely divergence-free
        if not adjoint:
            assert np.abs(g.D @ got).max() < 1e-10 * np.abs(g.D @ u).max()
    finally:
        S.selm_mac_destroy(h)


@pytest.mark.parametrize("dim,n,K", GRIDS + EDGE)
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("sigma", [0.0, 1.0])
def test_fac_cycle(S, dim, n, K, prec, sigma):
    F = _fac(dim, n, K, 0.9)
    h = _handle(S, dim, n, K, prec=prec, seed=5, instance=2)
    try:
        rng = np.random.default_rng(3)
        z0, b = rng.standard_normal(F.g.n_faces), rng.standard_normal(F.g.n_faces)
        want = z0.copy()
        F.fac_cycle(want, b, PhiloxNoise(5, 2, 11) if sigma else ExplicitNoise(), sigma)
        z = _dev(z0)
        S.selm_mac_fac_cycle(h, z, _dev(b), sigma, 11)
        got = _host(z)
        tol = _tol(prec, S)
        # the correction q = z - z0 carries the cycle's arithmetic
        assert rel(got - z0, want - z0) < tol and maxrel(got - z0, want - z0) < 10 * tol
    finally:
        S.selm_mac_destroy(h)


@pytest.mark.parametrize("dim,n,K", GRIDS)
@pytest.mark.parametrize("prec", [0, 1])
def test_solve(S, dim, n, K, prec):
    F = _fac(dim, n, K, 1.2)
    h = _handle(S, dim, n, K, mu=1.2, prec=prec)
    try:
        b = np.random.default_rng(4).standard_normal(F.g.n_faces)
        want, cyc_o, _ = F.solve(b, tol=1e-11)
        z = torch.zeros(F.g.n_faces, dtype=torch.float64, device="cuda")
        cycles, r = S.selm_mac_solve(h, z, _dev(b), 1e-11, 100)
        assert r <= 1e-11
        if prec == S.SELM_FP64:
            assert cycles == cyc_o
            assert rel(_host(z), want) < 1e-12 and maxrel(_host(z), want) < 1e-12
        else:
            assert cycles <= cyc_o + 2
            assert rel(_host(z), want) < 1e-9
    finally:
        S.selm_mac_destroy(h)


@pytest.mark.parametrize("dim,n,K", GRIDS)
@pytest.mark.parametrize("prec", [0, 1])
def test_chain(S, dim, n, K, prec):
    F = _fac(dim, n, K, 0.9)
    h = _handle(S, dim, n, K, prec=prec, seed=9, instance=4)
    try:
        xi = torch.zeros(F.g.n_faces, dtype=torch.float64, device="cuda")
        S.selm_mac_sample(h, 3, xi)
        want = np.zeros(F.g.n_faces)
        zero = np.zeros(F.g.n_faces)
        for k in range(3):
            F.fac_cycle(want, zero, PhiloxNoise(9, 4, k), 1.0)
        tol = _tol(prec, S)
        assert rel(_host(xi), want) < tol and maxrel(_host(xi), want) < 10 * tol
        assert S.selm_mac_chain(h)[1] == 3
        # graph replays (from the third cycle on) continue the same chain
        S.selm_mac_sample(h, 2, xi)
        for k in range(3, 5):
            F.fac_cycle(want, zero, PhiloxNoise(9, 4, k), 1.0)
        assert rel(_host(xi), want) < tol
    finally:
        S.selm_mac_destroy(h)


PARTS_2D = np.array([[0.31, 0.12], [0.77, 0.33], [0.12, 0.2], [0.5, 0.61]])
PARTS_3D = np.array([[0.31, 0.52, 0.12], [0.77, 0.1, 0.33], [0.45, 0.8, 0.61]])


@pytest.mark.parametrize("dim,n,K", [(2, 16, 5), (3, 8, 3)])
def test_interp_spread(S, dim, n, K):
    cs = CompositeSELM(n, K, dim, mu=0.9)
    X = PARTS_2D if dim == 2 else PARTS_3D
    Gam = cs.interpolation(X).toarray()
    h = _handle(S, dim, n, K)
    try:
        rng = np.random.default_rng(5)
        u = rng.standard_normal(cs.g.n_faces)
        Fp = rng.standard_normal(X.shape)
        U = torch.zeros(X.shape, dtype=torch.float64, device="cuda")
        f = torch.zeros(cs.g.n_faces, dtype=torch.float64, device="cuda")
        S.selm_mac_interp(h, _dev(X), _dev(u), U)
        S.selm_mac_spread(h, _dev(X), _dev(Fp), f)
        assert maxrel(_host(U).ravel(), Gam @ u) < 1e-13
        assert maxrel(_host(f), Gam.T @ Fp.ravel()) < 1e-13
    finally:
        S.selm_mac_destroy(h)


@pytest.mark.parametrize("dim,n,K", [(2, 16, 5), (3, 8, 3)])
@pytest.mark.parametrize("project", [0, 1])
def test_mobility(S, dim, n, K, project):
    cs = CompositeSELM(n, K, dim, mu=0.9, project=bool(project))
    X = PARTS_2D if dim == 2 else PARTS_3D
    Fp = np.random.default_rng(6).standard_normal(X.shape)
    want = cs.mobility_matrix(X, tol=1e-12) @ Fp.ravel()
    h = _handle(S, dim, n, K, projection=project, tol=1e-12, proj_tol=1e-14)
    try:
        U = torch.zeros(X.shape, dtype=torch.float64, device="cuda")
        S.selm_mac_mobility(h, _dev(X), _dev(Fp), U)
        assert maxrel(_host(U).ravel(), want) < 1e-11
    finally:
        S.selm_mac_destroy(h)


@pytest.mark.parametrize("dim,n,K", [(2, 16, 5), (3, 8, 3)])
@pytest.mark.parametrize("project", [0, 1])
def test_thermal(S, dim, n, K, project):
    cs = CompositeSELM(n, K, dim, mu=0.9, kT=1.3, project=bool(project))
    X = PARTS_2D if dim == 2 else PARTS_3D
    h = _handle(S, dim, n, K, kT=1.3, projection=project, proj_tol=1e-14, seed=3, instance=1)
    try:
        g = torch.zeros(X.shape, dtype=torch.float64, device="cuda")
        S.selm_mac_thermal(h, _dev(X), 2, g)
        ptr, cyc = S.selm_mac_chain(h)
        assert cyc == 2
        xi = torch.zeros(cs.g.n_faces, dtype=torch.float64, device="cuda")
        S.selm_mac_sample(h, 0, xi)
        want = cs.thermal_operator(X) @ _host(xi)
        assert maxrel(_host(g).ravel(), want) < 1e-12
        # and xi is the oracle's chain after two cycles
        cs.seed, cs.instance = 3, 1
        assert maxrel(_host(xi), cs.chain_cycles(2)) < 1e-12
    finally:
        S.selm_mac_destroy(h)


@pytest.mark.parametrize("dim,n,K,project", [(2, 16, 5, 1), (3, 8, 3, 0), (3, 8, 3, 1)])
def test_em_steps(S, dim, n, K, project):
    X0 = PARTS_2D if dim == 2 else PARTS_3D
    Fp = np.random.default_rng(7).standard_normal(X0.shape)
    cs = CompositeSELM(n, K, dim, mu=0.9, kT=0.8, project=bool(project), seed=11, instance=6, tol=1e-12)
    want = X0.copy()
    for _ in range(2):
        want, _ = cs.em_step(want, Fp, 1e-3, 2)
    h = _handle(S, dim, n, K, kT=0.8, projection=project, tol=1e-12, proj_tol=1e-14, seed=11, instance=6)
    try:
        X = _dev(X0)
        S.selm_mac_step(h, X, _dev(Fp), 1e-3, 2, 2)
        got = _host(X)
        assert maxrel(got - X0, want - X0) < 1e-10
    finally:
        S.selm_mac_destroy(h)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_cycle_spanning_many_tiles(S, prec):
    # a grid with ~200 K face unknowns: many 32-row slices per class and per
    # level, ragged class tails, two base classes of ~36 K rows swept one
    # lane per row, base level 2 swept in one block; one deterministic and
    # one stochastic cycle
    dim, n, K = 3, 32, 6
    F = _fac(dim, n, K, 1.0)
    fp32 = prec == "fp32"
    h = _handle(S, dim, n, K, mu=1.0, prec=S.SELM_FP32_REFINE64 if fp32 else S.SELM_FP64, seed=1, instance=1)
    try:
        rng = np.random.default_rng(8)
        z0, b = rng.standard_normal(F.g.n_faces), rng.standard_normal(F.g.n_faces)
        for sigma in (0.0, 1.0):
            want = z0.copy()
            F.fac_cycle(want, b, PhiloxNoise(1, 1, 3) if sigma else ExplicitNoise(), sigma)
            z = _dev(z0)
            S.selm_mac_fac_cycle(h, z, _dev(b), sigma, 3)
            got = _host(z)
            if fp32:
                assert rel(got - z0, want - z0) < 1e-5 and maxrel(got - z0, want - z0) < 1e-4
            else:
                assert rel(got - z0, want - z0) < 1e-12 and maxrel(got - z0, want - z0) < 1e-11
    finally:
        S.selm_mac_destroy(h)


def test_invalid_arguments(S):
    h = _handle(S, 2, 8, 2)
    try:
        with pytest.raises(S.SelmError):
            S.selm_mac_fac_cycle(h, None, None, 0.0, 0)
        assert S.selm_mac_colours(h, 99) == -1
    finally:
        S.selm_mac_destroy(h)
    with pytest.raises(S.SelmError) as info:
        S.selm_mac_create(S.make_mac_desc(2, 8, 9))
    assert info.value.status == S.SELM_EINVAL


def test_benchmark_size_properties(S):
    """The benchmark's staggered grid (64^3 base, 8 refined rows, 1.46 M faces,
    FP32 inner cycles), checked by properties that hold at any size: the
    projection's output is discretely divergence-free and a fixed point of
    the projection, and a FAC solve reaches its tolerance with A z = b (the
    operator applied by its own kernel)."""
    h = _handle(S, 3, 64, 8, mu=1.0, prec=S.SELM_FP32_REFINE64, projection=1, proj_tol=1e-12)
    try:
        nf, nc = S.selm_mac_faces(h), S.selm_mac_cells(h)
        assert nf == 1458176 and nc == 491520
        u = torch.randn(nf, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
        pu = torch.empty_like(u)
        S.selm_mac_project(h, u, pu)
        div_u, div_pu = torch.empty(nc, dtype=torch.float64, device="cuda"), torch.empty(nc, dtype=torch.float64,
                                                                                         device="cuda")
        S.selm_mac_divergence(h, u, div_u)
        S.selm_mac_divergence(h, pu, div_pu)
        assert div_pu.abs().max().item() < 1e-9 * div_u.abs().max().item()
        ppu = torch.empty_like(u)
        S.selm_mac_project(h, pu, ppu)
        assert (ppu - pu).abs().max().item() < 1e-9 * pu.abs().max().item()
        b = torch.randn(nf, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(2))
        z = torch.zeros_like(b)
        cycles, r = S.selm_mac_solve(h, z, b, 1e-10, 100)
        assert r <= 1e-10 and cycles < 60
        Az = torch.empty_like(z)
        S.selm_mac_apply(h, z, Az)
        assert ((Az - b).norm() / b.norm()).item() < 2e-10
    finally:
        S.selm_mac_destroy(h)
