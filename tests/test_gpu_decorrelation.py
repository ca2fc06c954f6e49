"""GPU: lag correlations of the library's samplers equal the oracle's (Section 5).

The multigrid sampler iterates FAC cycles (``selm_mg_fac_cycle``), the
Gauss-Seidel sampler fine-grid red-black sweeps (``selm_mg_smooth`` at level
0); both start from w = A^-1 phi given by the library's solve.  The curves
rho(k) must equal the oracle's (oracle/decorrelation.py) to the precision of
the path: 1e-10 in FP64, 1e-5 with FP32 inner iterations.  At the benchmark's
128^3 size the wall mode's covariance image is checked against its closed
form and the curves against the properties that hold at any size.
"""

import numpy as np
import pytest
import torch

from oracle import decorrelation as OD
from oracle import grid
from tests.affine import flatten

pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1003_2680_gb300 import decorrelation as D
    from paper_1003_2680_gb300 import selm as S


@pytest.fixture(autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


PRECS = {"fp64": (0, 1e-10), "fp32": (1, 1e-5)}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,n,levels", [(2, 32, 4), (3, 16, 3)])
def test_lag_correlations_match_oracle(prec, dim, n, levels):
    p, tol = PRECS[prec]
    m = S.SelmMG(dim=dim, n=n, levels=levels, precision=p, mu=1.0, seed=2, instance=1)
    mg, gs = OD.mg_sampler(n, dim, levels=levels), OD.gs_sampler(n, dim)
    s = mg["system"]
    for phi_lib, phi_or in ((D.wall_mode(m.h, n), OD.wall_mode(s)), (D.point_probe(m.h), OD.point_probe(s))):
        assert np.array_equal(phi_lib, flatten(phi_or))      # same observable, same layout
        w_or = OD.covariance_image(mg, phi_or)
        wn = flatten(w_or)
        w = D.covariance_image(m.h, phi_lib, tol=1e-12)   # error <= cond(A) x 1e-12
        assert np.linalg.norm(w.cpu().numpy() - wn) / np.linalg.norm(wn) < 1e-9
        w = torch.tensor(wn, device="cuda")        # both curves from the same start
        r_mg = D.lag_correlations_mg(m.h, phi_lib, 4, w)
        assert np.abs(r_mg - OD.lag_correlations(mg, phi_or, 4, w_or)).max() < tol
        r_gs = D.lag_correlations_gs(m.h, phi_lib, 24, w)
        assert np.abs(r_gs - OD.lag_correlations(gs, phi_or, 24, w_or)).max() < tol
    m.close()


def test_bench_size_properties():
    # 128^3, FP32 inner iterations as in the benchmark
    n = 128
    m = S.SelmMG(dim=3, n=n, precision=1, seed=0, instance=0)
    phi = D.wall_mode(m.h, n)
    lam = (1.0 / n) * 4.0 * np.sin(np.pi / (2 * n)) ** 2   # mu h^(d-2) x DST-II eigenvalue
    w = D.covariance_image(m.h, phi)                        # to the solve's 1e-10
    assert np.abs(w.cpu().numpy() - phi / lam).max() < 1e-6 * np.abs(phi / lam).max()
    r_mg = D.lag_correlations_mg(m.h, phi, 3, w)
    assert D.lags_below(r_mg) == 1
    r_gs = D.lag_correlations_gs(m.h, phi, 30, w)
    assert np.all(np.diff(r_gs) < 0) and r_gs[-1] > 0.9      # slow mode, monotone decay
    probe = D.point_probe(m.h)
    r_p = D.lag_correlations_mg(m.h, probe, 3)
    assert D.lags_below(r_p) == 1
    m.close()


def test_layout_helpers_match_oracle_lattices():
    # the observable builders read the layout only; check them on a grid whose
    # component 0 lattice is the cell lattice across the walls
    for dim, n in [(2, 16), (3, 8)]:
        m = S.SelmMG(dim=dim, n=n, precision=0)
        s = grid.velocity_system(n, dim)
        assert np.array_equal(D.wall_mode(m.h, n), flatten(OD.wall_mode(s)))
        m.close()
