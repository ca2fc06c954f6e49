"""CPU: the staggered composite grid's host plan equals the oracle's operators.

The library builds every operator of the composite MAC grid on the host
(selm_mac_setup.cpp, no GPU involved): the velocity operator of reading R22,
divergence and gradient of reading R21 (Eq. equ_def_discr_div and the
coarse-face gradient), the pressure operator diag(vol) D G, the FAC
transfers and Galerkin base operators of reading R23 with their first-fit
colour classes, and the extension E of reading R24.  Each is compared with
the oracle's (oracle/composite_mac.py) entry by entry; the colour classes,
which fix the Gibbs visiting order and the noise addressing, must be equal.
"""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.composite_mac import CompositeMAC, CompositeMACFAC, CompositeSELM

CASES = [(2, 8, 2), (2, 8, 0), (2, 8, 8), (2, 16, 5), (3, 4, 1), (3, 8, 3), (3, 8, 0)]


@pytest.fixture(scope="module")
def S():
    from paper_1003_2680_gb300 import _build, selm
    _build.build()
    return selm


def _csr(t):
    nr, nc, ip, ix, d = t
    return sp.csr_matrix((d, ix, ip), shape=(nr, nc))


def _maxrel(a, b):
    return abs(a - b).max() / max(abs(b).max(), 1e-300)


@pytest.mark.parametrize("dim,n,K", CASES)
def test_operators_equal_the_oracle(S, dim, n, K):
    d = S.make_mac_desc(dim, n, K, mu=0.9)
    g = CompositeMAC(n, K, dim)
    F = CompositeMACFAC(g, mu=0.9)
    cs = CompositeSELM(n, K, dim, mu=0.9)
    want = {S.SELM_MAC_MAT_A: g.velocity_operator(0.9), S.SELM_MAC_MAT_D: g.D, S.SELM_MAC_MAT_G: g.G,
            S.SELM_MAC_MAT_S: sp.diags(g.vol) @ g.laplacian(), S.SELM_MAC_MAT_P: F.P, S.SELM_MAC_MAT_E: cs.E}
    for which, m in want.items():
        got = _csr(S.selm_mac_host_matrix(d, which))
        assert got.shape == m.shape
        assert _maxrel(got, m) < 1e-15, which
    for lev, m in enumerate(F.ops):
        assert _maxrel(_csr(S.selm_mac_host_matrix(d, S.SELM_MAC_MAT_OPS, lev)), m) < 1e-14
    for lev, m in enumerate(F.Pl):
        assert _maxrel(_csr(S.selm_mac_host_matrix(d, S.SELM_MAC_MAT_PL, lev)), m) == 0.0


@pytest.mark.parametrize("dim,n,K", CASES)
def test_colour_classes_equal_the_oracle(S, dim, n, K):
    d = S.make_mac_desc(dim, n, K)
    F = CompositeMACFAC(CompositeMAC(n, K, dim))
    for lev, classes in enumerate(F.colours):
        want = np.full(F.ops[lev].shape[0], -1)
        for c, idx in enumerate(classes):
            want[idx] = c
        assert np.array_equal(S.selm_mac_host_colours(d, lev), want)
    want = np.full(F.g.n_faces, -1)
    for c, idx in enumerate(F.patch_colours):
        want[idx] = c
    assert np.array_equal(S.selm_mac_host_colours(d, -1), want)


@pytest.mark.parametrize("bad", [dict(dim=4, n=8, K=2), dict(dim=3, n=6, K=1, levels=3), dict(dim=2, n=8, K=9),
                                 dict(dim=2, n=8, K=-1), dict(dim=3, n=8, K=2, precision=5)])
def test_invalid_descriptors_rejected(S, bad):
    d = S.make_mac_desc(**bad)
    with pytest.raises(S.SelmError) as info:
        S.selm_mac_host_matrix(d, S.SELM_MAC_MAT_A)
    assert info.value.status == S.SELM_EINVAL
