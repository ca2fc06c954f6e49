"""GPU parity of the exact Stokes mobility and the Ito drift against the oracle.

The oracle (oracle/stokes.py, reading R28) solves the MAC saddle point by a
sparse direct solve; the library by conjugate gradients on the pressure
Schur complement with FAC inner solves.  Compared on the same seeded inputs:
the Stokes velocity, the mobility, the random-finite-difference directions
and drift, and whole Euler-Maruyama steps with both corrections.
"""

import numpy as np
import pytest
import torch

from oracle.stokes import StokesModel, StokesSolver, rfd_directions
from tests.gpu_util import maxrel, rel

pytestmark = pytest.mark.gpu

GRIDS = [(2, 16), (3, 8)]


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_2680_gb300 import selm as mod
    mod.lib()
    return mod


def _handle(S, dim, n, prec=0, mu=0.9, kT=1.2, seed=3, instance=2, tol=1e-12, max_particles=64):
    d = S.make_desc(dim=dim, n=n, mu=mu, kT=kT, precision=prec, seed=seed, instance=instance, tol=tol,
                    max_particles=max_particles, torch_allocator=False)
    return S.selm_mg_create(d)


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("dim,n", GRIDS)
@pytest.mark.parametrize("prec", [0, 1])
def test_stokes_solve(S, dim, n, prec):
    st = StokesSolver(n, dim, mu=0.9)
    f = np.random.default_rng(1).standard_normal(st.nv)
    want = st.solve(f)[0]
    h = _handle(S, dim, n, prec)
    try:
        u = torch.zeros(st.nv, dtype=torch.float64, device="cuda")
        it, res = S.selm_mg_stokes_solve(h, _dev(f), u, 1e-12)
        got = u.cpu().numpy()
        assert res <= 1e-12 and it < 200
        assert rel(got, want) < 1e-12 and maxrel(got, want) < 1e-12, (rel(got, want), it)
        assert np.abs(st.D @ got).max() < 1e-10 * np.abs(got).max()
    finally:
        S.selm_mg_destroy(h)


PARTS = {2: np.array([[0.31, 0.12], [0.77, 0.43], [0.5, 0.81]]),
         3: np.array([[0.31, 0.52, 0.14], [0.77, 0.1, 0.43], [0.45, 0.8, 0.79]])}


@pytest.mark.parametrize("dim,n", GRIDS)
def test_stokes_mobility(S, dim, n):
    X = PARTS[dim]
    Fp = np.random.default_rng(2).standard_normal(X.shape)
    m = StokesModel(n, dim, mu=0.9, kT=1.2)
    want = m.mobility_apply(X, Fp)
    h = _handle(S, dim, n)
    try:
        U = torch.zeros(X.shape, dtype=torch.float64, device="cuda")
        S.selm_mg_stokes_mobility(h, _dev(X), _dev(Fp), U)
        assert maxrel(U.cpu().numpy(), want) < 1e-12
    finally:
        S.selm_mg_destroy(h)


def test_rfd_directions_equal_the_oracle(S):
    h = _handle(S, 3, 8, seed=5, instance=2)
    try:
        W = torch.zeros((50, 3), dtype=torch.float64, device="cuda")
        S.selm_mg_rfd_directions(h, 50, 7, W)
        assert np.abs(W.cpu().numpy() - rfd_directions(5, 2, 7, 50, 3)).max() < 1e-14
    finally:
        S.selm_mg_destroy(h)


@pytest.mark.parametrize("dim,n", GRIDS)
def test_rfd_drift(S, dim, n):
    X = PARTS[dim]
    W = np.random.default_rng(3).standard_normal(X.shape)
    m = StokesModel(n, dim, mu=0.9, kT=1.2, delta=1e-3)
    want = m.rfd_drift(X, W)
    h = _handle(S, dim, n)
    try:
        d = torch.zeros(X.shape, dtype=torch.float64, device="cuda")
        S.selm_mg_rfd_drift(h, _dev(X), _dev(W), 1e-3, d)
        # a difference of two mobilities over delta = 1e-3: the solves' ~1e-13
        # relative accuracy becomes ~1e-10 of the drift
        assert maxrel(d.cpu().numpy(), want) < 1e-9
    finally:
        S.selm_mg_destroy(h)


@pytest.mark.parametrize("dim,n", GRIDS)
@pytest.mark.parametrize("delta", [0.0, 1e-3])
def test_stokes_steps(S, dim, n, delta):
    X0 = PARTS[dim]
    Fp = np.random.default_rng(4).standard_normal(X0.shape)
    m = StokesModel(n, dim, mu=0.9, kT=1.2, seed=3, instance=2, delta=delta if delta else 1e-3,
                    drift=delta > 0)
    want = X0.copy()
    for _ in range(2):
        want = m.em_step(want, Fp, 1e-3, 2)
    h = _handle(S, dim, n)
    try:
        X = _dev(X0)
        S.selm_mg_stokes_step(h, X, _dev(Fp), 1e-3, 2, 2, delta)
        got = X.cpu().numpy()
        assert maxrel(got - X0, want - X0) < 1e-10
    finally:
        S.selm_mg_destroy(h)


def test_stokes_mobility_at_the_benchmark_size(S):
    """128^3 FP32 channel: the Stokes velocity is divergence-free to the
    solve's accuracy and the mobility is symmetric (columns for two
    particles near the bottom wall)."""
    X = np.array([[0.31, 0.52, 0.06], [0.77, 0.12, 0.11]])
    h = _handle(S, 3, 128, prec=1, tol=1e-10, max_particles=8)
    try:
        M = np.zeros((6, 6))
        for col in range(6):
            F = np.zeros((2, 3))
            F[col // 3, col % 3] = 1.0
            U = torch.zeros((2, 3), dtype=torch.float64, device="cuda")
            S.selm_mg_stokes_mobility(h, _dev(X), _dev(F), U)
            M[:, col] = U.cpu().numpy().ravel()
        assert np.abs(M - M.T).max() < 1e-6 * np.abs(M).max()
        assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0
    finally:
        S.selm_mg_destroy(h)
