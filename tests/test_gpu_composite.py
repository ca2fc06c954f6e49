"""GPU parity of the composite-grid FAC (refined patch, Algorithms 1-2).

Every call goes through the C ABI (selm_comp_*) and is compared with the FP64
oracle (oracle/composite.py) on the same seeded inputs: 1e-12 relative for the
FP64 path, 1e-5 for FP32 inner cycles with FP64 refinement.
"""

import numpy as np
import pytest
import torch

import selm_inputs
from oracle import composite as OC, multigrid
from oracle.philox import PhiloxNoise

pytestmark = pytest.mark.gpu

# (dim, n, K): small grids span several tiles, the n = 32 grid runs the base
# levels from 2 in the cluster engine, n = 12 takes the scalar red-black path
# of the base grid and n = 10 the scalar patch sweep (2n not a multiple of 8)
GRIDS = [(2, 16, 2), (3, 8, 2), (3, 16, 3), (3, 32, 4), (2, 12, 2), (2, 10, 2)]


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_2680_gb300 import selm as mod
    mod.lib()
    return mod


def handle(S, dim, n, K, prec, ncomp=2, seed=5, instance=2, mu=1.3, **kw):
    p = S.SELM_FP64 if prec == "fp64" else S.SELM_FP32_REFINE64
    c = S.selm_comp_create(S.make_comp_desc(dim, n, K, ncomp=ncomp, mu=mu, precision=p, seed=seed,
                                            instance=instance, **kw))
    cg = OC.CompositeGrid(n, K, dim, mu=mu, ncomp=ncomp)
    return c, cg


def to_gpu(cg, zs):
    """Oracle per-component composite vectors -> the library's composite layout."""
    fines, bases = [], []
    for z in zs:
        f, b = cg.from_vec(z)
        fines.append(f.ravel())
        bases.append(b.ravel())
    return np.concatenate(fines + bases)


def from_gpu(cg, vec):
    nf, nb = cg.n_fine, int(np.prod(cg.base_shape))
    N0 = nf * cg.ncomp
    out = []
    for c in range(cg.ncomp):
        f = vec[c * nf:(c + 1) * nf].reshape(cg.fine_shape)
        b = vec[N0 + c * nb:N0 + (c + 1) * nb].reshape(cg.base_shape)
        out.append(cg.to_vec(f, b))
    return out


def rand_vecs(cg, seed, scale=1.0):
    rng = np.random.default_rng([seed, 77])
    return [scale * rng.standard_normal(cg.size) for _ in range(cg.ncomp)]


def rel(a, b):
    a = np.concatenate(a)
    b = np.concatenate(b)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def dev(x):
    return torch.tensor(x, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("dim,n,K", GRIDS)
def test_composite_residual(S, dim, n, K):
    c, cg = handle(S, dim, n, K, "fp64")
    z, b = rand_vecs(cg, 1), rand_vecs(cg, 2)
    zg = to_gpu(cg, z)
    zg_dirty = zg.copy()
    nf = cg.n_fine * cg.ncomp
    # covered base rows are not unknowns: garbage there must not matter
    for comp in range(cg.ncomp):
        (_, _, _), off, size = S.selm_comp_layout(c, 1, comp)
        covered = cg.K * cg.base_shape[1] * cg.base_shape[2]
        zg_dirty[off:off + covered] = 1e3
    r = torch.zeros(S.selm_comp_size(c), dtype=torch.float64, device="cuda")
    n2 = S.selm_comp_residual(c, dev(zg_dirty), dev(to_gpu(cg, b)), r)
    want = OC.residual(cg, z, b)
    got = from_gpu(cg, r.cpu().numpy())
    assert rel(got, want) < 1e-13
    assert abs(n2 - sum(float(x @ x) for x in want)) <= 1e-12 * n2
    S.selm_comp_destroy(c)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("noise", [0, 1])
@pytest.mark.parametrize("dim,n,K", GRIDS[:3] + GRIDS[5:])
def test_patch_sweeps(S, prec, noise, dim, n, K):
    c, cg = handle(S, dim, n, K, prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    q, r = rand_vecs(cg, 3), rand_vecs(cg, 4)
    if prec == "fp32":
        q = [x.astype(np.float32).astype(np.float64) for x in q]
        r = [x.astype(np.float32).astype(np.float64) for x in r]
    g_q, g_r = to_gpu(cg, q), to_gpu(cg, r)
    nf = cg.n_fine * cg.ncomp
    qp = torch.tensor(g_q[:nf], dtype=dt, device="cuda")
    qb = torch.tensor(g_q[nf:], dtype=dt, device="cuda")
    rp = torch.tensor(g_r[:nf], dtype=dt, device="cuda")
    S.selm_comp_patch_sweeps(c, qp, qb, rp, 2, 7, noise)
    nz = PhiloxNoise(5, 2, 7)
    want = []
    for comp in range(cg.ncomp):
        qq = q[comp].copy()
        rr = r[comp].copy()
        for s in range(2):
            cg.patch_sweep(qq, rr, comp, s, nz, float(noise))
        want.append(qq[:cg.n_fine])
    got = qp.double().cpu().numpy().reshape(cg.ncomp, cg.n_fine)
    assert rel(list(got), want) < (1e-12 if prec == "fp64" else 1e-5)
    S.selm_comp_destroy(c)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("noise", [0, 1])
@pytest.mark.parametrize("dim,n,K", GRIDS)
def test_fac_cycle(S, prec, noise, dim, n, K):
    c, cg = handle(S, dim, n, K, prec)
    z, b = rand_vecs(cg, 5), rand_vecs(cg, 6)
    zg = dev(to_gpu(cg, z))
    S.selm_comp_fac_cycle(c, zg, dev(to_gpu(cg, b)), 11, noise)
    want = [x.copy() for x in z]
    OC.fac_cycle(cg, want, b, PhiloxNoise(5, 2, 11), float(noise))
    got = from_gpu(cg, zg.cpu().numpy())
    # compare the change of z (the cycle's correction), the part the inner precision touches
    d_got = [g - z0 for g, z0 in zip(got, z)]
    d_want = [w - z0 for w, z0 in zip(want, z)]
    assert rel(d_got, d_want) < (1e-12 if prec == "fp64" else 1e-5)
    S.selm_comp_destroy(c)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,n,K", [(2, 16, 2), (3, 16, 3)])
def test_solve(S, prec, dim, n, K):
    c, cg = handle(S, dim, n, K, prec)
    b = rand_vecs(cg, 8)
    z = torch.zeros(S.selm_comp_size(c), dtype=torch.float64, device="cuda")
    cycles, res = S.selm_comp_solve(c, z, dev(to_gpu(cg, b)), 1e-10, 200)
    assert res <= 1e-10
    want, ocycles, _ = OC.solve(cg, b, tol=1e-10)
    if prec == "fp64":
        assert cycles == ocycles
    assert rel(from_gpu(cg, z.cpu().numpy()), want) < (1e-12 if prec == "fp64" else 1e-8)
    S.selm_comp_destroy(c)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,n,K", [(2, 16, 2), (3, 8, 2), (3, 16, 3)])
def test_chain(S, prec, dim, n, K):
    """Five stochastic cycles of the chain; with FP32 inner cycles the chain
    state is a double-float pair, compared at the FP32 tolerance."""
    c, cg = handle(S, dim, n, K, prec, seed=9, instance=4)
    S.selm_comp_set_cycle(c, 3)
    buf = torch.zeros(S.selm_comp_size(c), dtype=torch.float64, device="cuda")
    S.selm_comp_sample(c, 5, buf)
    assert S.selm_comp_chain(c) == 8
    want = [np.zeros(cg.size) for _ in range(cg.ncomp)]
    zero = [np.zeros(cg.size) for _ in range(cg.ncomp)]
    for k in range(3, 8):
        OC.fac_cycle(cg, want, zero, PhiloxNoise(9, 4, k), 1.0)
    assert rel(from_gpu(cg, buf.cpu().numpy()), want) < (1e-12 if prec == "fp64" else 1e-5)
    assert S.selm_comp_stats(c) == 5
    S.selm_comp_destroy(c)


@pytest.mark.slow
@pytest.mark.parametrize("n,K", [(128, 16), (256, 8)])
def test_fac_cycle_on_the_benchmark_base_paths(S, n, K):
    """One stochastic FP32 FAC cycle against the oracle on grids whose base
    hierarchy takes the launch paths of the benchmark's 256^3 grid: at n = 128
    the 64^3 level runs in cooperative launches and the levels below in the
    cluster engine; at n = 256 level 2 (128^3) takes one launch per colour
    pass, level 3 the cooperative launches and levels 4+ the engine, all with
    the z-dependent Galerkin bands of the covered rows.  Compared over the
    whole vector and element by element on the cycle's correction."""
    c, cg = handle(S, 3, n, K, "fp32", ncomp=1, seed=3, instance=1, mu=1.0)
    z, b = rand_vecs(cg, 15, scale=1e-2), rand_vecs(cg, 16)
    zg = dev(to_gpu(cg, z))
    S.selm_comp_fac_cycle(c, zg, dev(to_gpu(cg, b)), 4, 1)
    want = [x.copy() for x in z]
    OC.fac_cycle(cg, want, b, PhiloxNoise(3, 1, 4), 1.0)
    got = from_gpu(cg, zg.cpu().numpy())
    d_got = [g - z0 for g, z0 in zip(got, z)]
    d_want = [w - z0 for w, z0 in zip(want, z)]
    assert rel(d_got, d_want) < 1e-5
    err = np.abs(d_got[0] - d_want[0]).max() / np.abs(d_want[0]).max()
    assert err < 1e-5, err
    S.selm_comp_destroy(c)


def test_invalid_descriptors(S):
    for kw in [dict(dim=4, n=8, K=2), dict(dim=3, n=7, K=2), dict(dim=3, n=8, K=7), dict(dim=3, n=8, K=0)]:
        d = S.make_comp_desc(**kw)
        assert S.selm_comp_footprint(d) == 0
        with pytest.raises(S.SelmError):
            S.selm_comp_create(d)


# ---- the benchmark's size: 256^3 base, bottom 32 rows refined (512 x 512 x 64 patch),
# three components, FP32 inner cycles with FP64 refinement -----------------------------

BENCH = dict(dim=3, n=256, K=32, ncomp=3)


def _blocks(S, c, ncomp):
    """(part, (nz, ny, nx), offset) of every patch and base block of a composite vector."""
    out = []
    for comp in range(ncomp):
        for part in (0, 1):
            (nx, ny, nz), off, _ = S.selm_comp_layout(c, part, comp)
            out.append((part, (nz, ny, nx), off))
    return out


def test_bench_size_linear_field_closed_form(S):
    """c = z (cell-centre heights): r = -A z vanishes on every composite row but
    the top-wall base rows, where it is -mu H^(d-2) (the coarse-fine gradient
    rule is exact on linear fields); values placed in covered base rows must
    not reach any row, and covered rows of r are 0."""
    n, K, mu = BENCH["n"], BENCH["K"], 1.0
    H = 1.0 / n
    c = S.selm_comp_create(S.make_comp_desc(precision=S.SELM_FP32_REFINE64, mu=mu, seed=0, instance=0, **BENCH))
    z = torch.empty(S.selm_comp_size(c), dtype=torch.float64, device="cuda")
    for part, (nz, ny, nx), off in _blocks(S, c, BENCH["ncomp"]):
        k = torch.arange(nz, dtype=torch.float64, device="cuda")
        zk = (2 * k + 3) * H / 4 if part == 0 else torch.where(k < K, 7.0, (k + 1) * H)
        z[off:off + nz * ny * nx] = zk[:, None].expand(nz, ny * nx).reshape(-1)
    r = torch.empty_like(z)
    S.selm_comp_residual(c, z, None, r, want_norm=False)
    torch.cuda.synchronize()
    for part, (nz, ny, nx), off in _blocks(S, c, BENCH["ncomp"]):
        blk = r[off:off + nz * ny * nx].view(nz, ny, nx)
        if part == 0:
            assert blk.abs().max().item() < 1e-12 * H
        else:
            assert torch.count_nonzero(blk[:K]).item() == 0
            assert blk[K:nz - 1].abs().max().item() < 1e-12 * H
            assert (blk[nz - 1] + mu * H).abs().max().item() < 1e-12 * H
    S.selm_comp_destroy(c)


def _roll(S, c, vec, s):
    """Shift a composite vector by s base cells (2s patch cells) along x and y."""
    out = torch.empty_like(vec)
    for part, (nz, ny, nx), off in _blocks(S, c, BENCH["ncomp"]):
        t = s if part == 1 else 2 * s
        blk = vec[off:off + nz * ny * nx].view(nz, ny, nx)
        out[off:off + nz * ny * nx] = torch.roll(blk, shifts=(t, t), dims=(1, 2)).reshape(-1)
    return out


def test_bench_size_fac_cycle_is_translation_equivariant(S):
    """Along the periodic axes the composite grid is translation invariant, so
    one deterministic FAC cycle commutes with a shift that keeps every level's
    colouring (192 base cells: a multiple of 2 on each smoothed level down to
    the 8^3 one, and of 3).  Every kernel of the cycle runs at the
    benchmark's size and launch shapes; an index or stride slip breaks the
    identity at O(1).  Only the coarsest dense solve sees a permuted vector
    (rounding), so the corrections agree to the FP32 tolerance."""
    c = S.selm_comp_create(S.make_comp_desc(precision=S.SELM_FP32_REFINE64, seed=0, instance=0, **BENCH))
    N = S.selm_comp_size(c)
    g = torch.Generator(device="cuda")
    g.manual_seed(1234)
    z0 = torch.randn(N, dtype=torch.float64, device="cuda", generator=g)
    b = torch.randn(N, dtype=torch.float64, device="cuda", generator=g)
    for part, (nz, ny, nx), off in _blocks(S, c, BENCH["ncomp"]):
        if part == 1:   # covered base rows are not unknowns
            z0[off:off + BENCH["K"] * ny * nx] = 0.0
            b[off:off + BENCH["K"] * ny * nx] = 0.0
    z = z0.clone()
    S.selm_comp_fac_cycle(c, z, b, 0, 0)
    zs = _roll(S, c, z0, 192)
    S.selm_comp_fac_cycle(c, zs, _roll(S, c, b, 192), 0, 0)
    torch.cuda.synchronize()
    d = _roll(S, c, z - z0, 192)
    ds = zs - _roll(S, c, z0, 192)
    assert (torch.linalg.vector_norm(ds - d) / torch.linalg.vector_norm(d)).item() < 1e-5
    S.selm_comp_destroy(c)
