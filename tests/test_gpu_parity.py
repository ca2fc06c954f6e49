"""GPU parity: every hot-path step of the CUDA library against the FP64 oracle.

Same seeded inputs and the same Philox counters on both sides.  Tolerances
(relative 2-norm over the whole field): 1e-12 for the FP64 path, 1e-5 for the
FP32 path (FP32 smoothing and transfers; the oracle runs the same steps in
FP64 on the FP32-rounded inputs).  Bit-exact for the Philox words.
"""

import numpy as np
import pytest
import torch

import selm_inputs
from oracle import coupling, gibbs, grid, multigrid, philox, projection, selm as oselm
from tests.gpu_util import empty, from_dev, maxrel, rel, round_like, to_dev

pytestmark = pytest.mark.gpu

S = None


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global S
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_2680_gb300 import selm as mod
    mod.lib()
    S = mod


PRECS = {"fp64": (0, torch.float64, 1e-12), "fp32": (1, torch.float32, 1e-5)}

# (dim, n, levels): config-1 grid, a ragged 3-D grid and a 3-D power-of-two grid
GRIDS = [(2, 64, 6), (3, 24, 3), (3, 32, 4)]


def make(dim, n, levels, prec="fp64", **kw):
    p, dt, tol = PRECS[prec]
    m = S.SelmMG(dim=dim, n=n, levels=levels, precision=p, seed=kw.pop("seed", 11),
                 instance=kw.pop("instance", 3), **kw)
    osys = grid.velocity_system(n, dim, mu=kw.get("mu", 1.0), levels=levels)
    return m, osys, dt, tol


def test_philox_words_bit_exact():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    key = (0x01234567, 0x89ABCDEF)
    want = philox.philox4x32_10(ctr, key)
    c = torch.tensor(ctr.view(np.int32), device="cuda")
    out = torch.zeros_like(c)
    S.selm_philox4x32_10(c, key[0], key[1], out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), want)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,n,levels", GRIDS)
@pytest.mark.parametrize("noise", [0, 1])
def test_smooth_all_levels(prec, dim, n, levels, noise):
    m, osys, dt, tol = make(dim, n, levels, prec)
    for level in range(levels - 1):   # the coarsest level takes the exact step
        shapes = osys.shapes(level)
        v0 = round_like(selm_inputs.fields(shapes, seed=level), dt)
        b0 = round_like(selm_inputs.fields(shapes, seed=100 + level), dt)
        v = to_dev(m.h, v0, dt, level=level)
        b = to_dev(m.h, b0, dt, level=level)
        S.selm_mg_smooth(m.h, 0, level, v, b, sweep=1, cycle=7, noise=noise)
        want = gibbs.sweep(osys, level, [x.copy() for x in v0], b0, 1,
                           philox.PhiloxNoise(11, 3, 7), float(noise))
        assert rel(from_dev(m.h, v, level=level), want) < tol, (level, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,n,levels", GRIDS)
def test_residual_restrict_and_prolong(prec, dim, n, levels):
    m, osys, dt, tol = make(dim, n, levels, prec)
    for level in range(levels - 1):
        shapes = osys.shapes(level)
        v0 = round_like(selm_inputs.fields(shapes, seed=1), dt)
        b0 = round_like(selm_inputs.fields(shapes, seed=2), dt)
        bc = empty(m.h, dt, level=level + 1)
        S.selm_mg_residual_restrict(m.h, 0, level, to_dev(m.h, v0, dt, level=level),
                                    to_dev(m.h, b0, dt, level=level), bc)
        r = [bb - a for bb, a in zip(b0, osys.apply(level, v0))]
        assert rel(from_dev(m.h, bc, level=level + 1), osys.restrict(level, r)) < tol
        vc0 = round_like(selm_inputs.fields(osys.shapes(level + 1), seed=3), dt)
        v = to_dev(m.h, v0, dt, level=level)
        S.selm_mg_prolong_correct(m.h, 0, level, v, to_dev(m.h, vc0, dt, level=level + 1))
        want = [a + p for a, p in zip(v0, osys.prolong(level, vc0))]
        assert rel(from_dev(m.h, v, level=level), want) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,n,levels", GRIDS + [(2, 4, 1)])
@pytest.mark.parametrize("noise", [0, 1])
def test_coarsest_exact_step(prec, dim, n, levels, noise):
    m, osys, dt, tol = make(dim, n, levels, prec)
    lev = levels - 1
    b0 = round_like(selm_inputs.fields(osys.shapes(lev), seed=5), dt)
    v = empty(m.h, dt, level=lev)
    S.selm_mg_coarsest(m.h, 0, v, to_dev(m.h, b0, dt, level=lev), cycle=9, noise=noise)
    co = multigrid.Coarsest(osys)
    want = co.apply(osys, b0, philox.PhiloxNoise(11, 3, 9), float(noise))
    assert rel(from_dev(m.h, v, level=lev), want) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,n,levels", GRIDS)
def test_outer_residual_and_update(prec, dim, n, levels):
    m, osys, dt, tol = make(dim, n, levels, prec)
    shapes = osys.shapes(0)
    z0 = selm_inputs.fields(shapes, seed=7)
    b0 = selm_inputs.fields(shapes, seed=8)
    z = to_dev(m.h, z0, torch.float64)
    b = to_dev(m.h, b0, torch.float64)
    r = empty(m.h, dt)
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
    S.selm_mg_outer_residual(m.h, 0, z, b, r, nrm)
    want = [bb - a for bb, a in zip(b0, osys.apply(0, z0))]
    assert rel(from_dev(m.h, r), want) < (1e-12 if dt == torch.float64 else 1e-7)
    wn = sum(float(np.sum(x * x)) for x in want)
    assert abs(nrm.item() - wn) / wn < 1e-12
    d0 = round_like(selm_inputs.fields(shapes, seed=9), dt)
    S.selm_mg_outer_update(m.h, 0, z, to_dev(m.h, d0, dt))
    assert rel(from_dev(m.h, z), [a + d for a, d in zip(z0, d0)]) < 1e-15


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,n,levels", GRIDS)
@pytest.mark.parametrize("noise", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_fac_cycle(prec, dim, n, levels, noise, mode):
    m, osys, dt, tol = make(dim, n, levels, prec, coarse_mode=mode)
    if mode == 1 and dim == 3 and n == 24:
        pytest.skip("coarsest 6^3 level smoothed: valid, covered by the other grids")
    shapes = osys.shapes(0)
    z0 = selm_inputs.fields(shapes, seed=12)
    b0 = selm_inputs.fields(shapes, seed=13)
    z = to_dev(m.h, z0, torch.float64)
    S.selm_mg_fac_cycle(m.h, 0, z, to_dev(m.h, b0, torch.float64), cycle=21, noise=noise)
    want = [x.copy() for x in z0]
    multigrid.fac_cycle(osys, want, b0, philox.PhiloxNoise(11, 3, 21), float(noise),
                        coarse_mode="cholesky" if mode == 0 else "smooth")
    assert rel(from_dev(m.h, z), want) < tol


# grids whose first Galerkin level exceeds one CTA: the coarse engine runs
# z-slabs over a thread-block cluster with DSMEM halo exchange
ENGINE_GRIDS = [(3, 48, 4), (3, 64, 4), (2, 256, 7)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,n,levels", ENGINE_GRIDS + [(2, 64, 6), (3, 32, 4)])
@pytest.mark.parametrize("noise", [0, 1])
@pytest.mark.parametrize("engine", [1, 0])
def test_vcycle_engine_and_per_pass_paths(prec, dim, n, levels, noise, engine):
    m, osys, dt, tol = make(dim, n, levels, prec)
    S.selm_mg_set_option(m.h, S.SELM_OPT_COARSE_ENGINE, engine)
    l0, csize, smem = S.selm_mg_engine_info(m.h)
    assert l0 == 1 and csize >= 1 and smem > 0
    if (dim, n) in [(3, 48), (3, 64), (2, 256)]:
        assert csize > 1, "expected the cluster path on this grid"
    shapes = osys.shapes(0)
    v0 = round_like(selm_inputs.fields(shapes, seed=31), dt)
    b0 = round_like(selm_inputs.fields(shapes, seed=32), dt)
    v = to_dev(m.h, v0, dt)
    S.selm_mg_vcycle(m.h, 0, v, to_dev(m.h, b0, dt), cycle=41, noise=noise)
    want = [x.copy() for x in v0]
    multigrid.vcycle(osys, 0, want, b0, philox.PhiloxNoise(11, 3, 41), float(noise))
    assert rel(from_dev(m.h, v), want) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,n,levels", ENGINE_GRIDS)
@pytest.mark.parametrize("noise", [0, 1])
@pytest.mark.parametrize("coop", [1, 2, 0])
def test_vcycle_engine_from_level_2(prec, dim, n, levels, noise, coop):
    """Level 1 above the engine: one cooperative launch per half V-cycle with
    the colour passes in dataflow order (coop=1, FP32) or separated by grid
    barriers (coop=2), or one GPU-wide launch per colour pass (coop=0)."""
    m, osys, dt, tol = make(dim, n, levels, prec)
    S.selm_mg_set_option(m.h, S.SELM_OPT_ENGINE_LEVEL, 2)
    S.selm_mg_set_option(m.h, S.SELM_OPT_LEVEL_COOP, coop)
    l0, csize, smem = S.selm_mg_engine_info(m.h)
    assert l0 == 2 and csize >= 1 and smem > 0
    shapes = osys.shapes(0)
    v0 = round_like(selm_inputs.fields(shapes, seed=33), dt)
    b0 = round_like(selm_inputs.fields(shapes, seed=34), dt)
    v = to_dev(m.h, v0, dt)
    S.selm_mg_vcycle(m.h, 0, v, to_dev(m.h, b0, dt), cycle=43, noise=noise)
    want = [x.copy() for x in v0]
    multigrid.vcycle(osys, 0, want, b0, philox.PhiloxNoise(11, 3, 43), float(noise))
    assert rel(from_dev(m.h, v), want) < tol


@pytest.mark.parametrize("noise", [0, 1])
@pytest.mark.parametrize("coop", [1, 2])
def test_vcycle_128_cooperative_rows(noise, coop):
    """The 128^3 channel's V-cycle as the benchmark runs it (FP32 inner
    cycles, level 1 in cooperative launches, engine from level 2): colour
    passes in dataflow order (coop=1) or separated by grid barriers (coop=2)."""
    dim, n, levels = 3, 128, 6
    m, osys, dt, tol = make(dim, n, levels, "fp32")
    S.selm_mg_set_option(m.h, S.SELM_OPT_LEVEL_COOP, coop)
    assert S.selm_mg_engine_info(m.h)[0] == 2
    shapes = osys.shapes(0)
    v0 = round_like(selm_inputs.fields(shapes, seed=35), dt)
    b0 = round_like(selm_inputs.fields(shapes, seed=36), dt)
    v = to_dev(m.h, v0, dt)
    S.selm_mg_vcycle(m.h, 0, v, to_dev(m.h, b0, dt), cycle=47, noise=noise)
    want = [x.copy() for x in v0]
    multigrid.vcycle(osys, 0, want, b0, philox.PhiloxNoise(11, 3, 47), float(noise))
    got = from_dev(m.h, v)
    assert rel(got, want) < tol
    # element by element, per component: a wrong wall row or plane among the
    # 6.27 M unknowns would pass the field norm but not this
    for g, w in zip(got, want):
        assert maxrel(g, w) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("coop", [1, 2])
def test_fac_solve_with_cooperative_level(prec, coop):
    """Deterministic FAC solve with level 1 in cooperative launches: same
    cycle count (FP64) and solution as the oracle, no barrier timeout."""
    dim, n, levels = 3, 64, 4
    m, osys, dt, tol = make(dim, n, levels, prec)
    S.selm_mg_set_option(m.h, S.SELM_OPT_LEVEL_COOP, coop)
    S.selm_mg_set_option(m.h, S.SELM_OPT_ENGINE_LEVEL, 2)
    assert S.selm_mg_engine_info(m.h)[0] == 2
    b0 = selm_inputs.fields(osys.shapes(0), seed=15)
    z = empty(m.h, torch.float64)
    cycles, res = S.selm_mg_fac_solve(m.h, 0, z, to_dev(m.h, b0, torch.float64), 1e-10, 50)
    assert res <= 1e-10
    want, ocycles, _ = multigrid.solve(osys, b0, tol=1e-10)
    if prec == "fp64":
        assert cycles == ocycles
    assert rel(from_dev(m.h, z), want) < (1e-12 if prec == "fp64" else 1e-8)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,n,levels", GRIDS)
def test_fac_solve(prec, dim, n, levels):
    m, osys, dt, tol = make(dim, n, levels, prec)
    b0 = selm_inputs.fields(osys.shapes(0), seed=14)
    z = empty(m.h, torch.float64)
    cycles, res = S.selm_mg_fac_solve(m.h, 0, z, to_dev(m.h, b0, torch.float64), 1e-10, 50)
    assert res <= 1e-10 and 1 <= cycles <= 15
    want, ocycles, _ = multigrid.solve(osys, b0, tol=1e-10)
    if prec == "fp64":
        assert cycles == ocycles
    assert rel(from_dev(m.h, z), want) < (1e-12 if prec == "fp64" else 1e-8)


@pytest.mark.parametrize("dim,n", [(2, 64), (3, 32)])
@pytest.mark.parametrize("clear", [2.0, 0.0])
def test_spread_interp(dim, n, clear):
    m = S.SelmMG(dim=dim, n=n, levels=3)
    osys = grid.velocity_system(n, dim, levels=1)
    X0 = selm_inputs.particles(37, dim, n, seed=4, clearance_cells=clear)
    F0 = selm_inputs.forces(37, dim, seed=4)
    X = torch.tensor(X0, device="cuda")
    F = torch.tensor(F0, device="cuda")
    b = empty(m.h, torch.float64)
    S.selm_mg_spread(m.h, X, F, b)
    assert rel(from_dev(m.h, b), coupling.spread(osys, F0, X0)) < 1e-13
    u0 = selm_inputs.fields(osys.shapes(0), seed=5)
    U = torch.zeros_like(X)
    S.selm_mg_interp(m.h, X, to_dev(m.h, u0, torch.float64), U)
    assert rel(U.cpu().numpy(), coupling.interpolate(osys, u0, X0)) < 1e-13


def test_spread_interp_no_particles():
    m = S.SelmMG(dim=3, n=16, levels=2)
    X = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    b = empty(m.h, torch.float64) + 1.0
    S.selm_mg_spread(m.h, X, X, b)
    assert float(b.abs().max()) == 0.0
    S.selm_mg_interp(m.h, X, b, X)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,n,levels", [(2, 32, 4), (3, 16, 3)])
def test_projection(prec, dim, n, levels):
    p, dt, tol = PRECS[prec]
    m = S.SelmMG(dim=dim, n=n, levels=levels, precision=p, projection=1, proj_tol=1e-12)
    w0 = selm_inputs.fields(grid.velocity_system(n, dim, levels=1).shapes(0), seed=6)
    w = to_dev(m.h, w0, torch.float64)
    S.selm_mg_project(m.h, w)
    want = projection.Projector(n, dim, tol=1e-12, levels=levels).project(w0)
    # both sides run the same pressure FAC iteration and stop after the same
    # cycle: FP64 agrees to rounding; FP32 inner cycles within FP64 refinement
    # meet the same stopping rule
    assert rel(from_dev(m.h, w), want) < (1e-12 if prec == "fp64" else 1e-9)
    div = projection.divergence(from_dev(m.h, w), dim)
    assert np.abs(div).max() < 1e-9 * np.abs(projection.divergence(w0, dim)).max()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("project", [0, 1])
def test_mobility_solve(prec, project):
    p, dt, tol = PRECS[prec]
    n, dim = 32, 2
    m = S.SelmMG(dim=dim, n=n, levels=5, precision=p, projection=project, mu=1.3, tol=1e-11, proj_tol=1e-12)
    om = oselm.Model(n, dim, mu=1.3, levels=5, project=bool(project), tol=1e-11)
    X0 = selm_inputs.particles(16, dim, n, seed=9)
    F0 = selm_inputs.forces(16, dim, seed=9)
    X = torch.tensor(X0, device="cuda")
    U = torch.zeros_like(X)
    cycles, res = S.selm_mg_solve(m.h, X, torch.tensor(F0, device="cuda"), U)
    want, ocycles, _ = om.mobility_apply(X0, F0)
    assert res <= 1e-11
    if prec == "fp64":
        assert cycles == ocycles
    assert rel(U.cpu().numpy(), want) < (1e-12 if prec == "fp64" else 1e-7)


def test_config1_chain_1000_cycles_fp64():
    # 2-D 64x64, 6 levels, (2,2) sweeps, FP64, Philox seed 0: 1000 stochastic
    # cycles of the chain; the GPU state equals the oracle's to 1e-12.
    m = S.SelmMG(dim=2, n=64, levels=6, precision=0, seed=0, instance=0)
    om = oselm.Model(64, 2, levels=6, seed=0, instance=0)
    X0 = selm_inputs.particles(16, 2, 64, seed=0)
    X = torch.tensor(X0, device="cuda")
    g = torch.zeros_like(X)
    xi = empty(m.h, torch.float64)
    for _ in range(4):
        S.selm_mg_sample(m.h, X, 250, g, xi)
    om.chain_cycles(1000)
    assert S.selm_mg_chain(m.h)[1] == 1000
    assert rel(from_dev(m.h, xi), om.xi) < 1e-12
    want = np.sqrt(2.0) * coupling.interpolate(om.sys, om.xi, X0)
    assert rel(g.cpu().numpy(), want) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("project", [0, 1])
def test_em_steps(prec, project):
    p, dt_, tol = PRECS[prec]
    n, dim = 16, 3
    m = S.SelmMG(dim=dim, n=n, levels=3, precision=p, projection=project, kT=0.7, seed=5, instance=2,
                 proj_tol=1e-12)
    om = oselm.Model(n, dim, kT=0.7, levels=3, project=bool(project), seed=5, instance=2)
    X0 = selm_inputs.particles(24, dim, n, seed=3)
    F0 = selm_inputs.forces(24, dim, seed=3)
    X = torch.tensor(X0, device="cuda")
    S.selm_mg_step(m.h, X, torch.tensor(F0, device="cuda"), 1e-3, 3, 2)
    Xo = X0.copy()
    for _ in range(3):
        Xo, _ = om.em_step(Xo, F0, 1e-3, 2)
    assert rel(X.cpu().numpy() - X0, Xo - X0) < (1e-12 if prec == "fp64" else 1e-5)


def test_em_wrap_reflect():
    m = S.SelmMG(dim=3, n=16, levels=2)
    X0 = np.array([[0.95, 0.02, 0.03], [0.5, 0.5, 0.97]])
    V0 = np.array([[0.10, -0.05, -0.05], [0.0, 0.0, 0.06]])
    X = torch.tensor(X0, device="cuda")
    S.selm_mg_em_update(m.h, X, torch.tensor(V0, device="cuda"))
    want = oselm.Model(16, 3, levels=2).wrap_reflect(X0 + V0)
    assert np.allclose(X.cpu().numpy(), want, atol=1e-15)


@pytest.mark.slow
def test_full_size_128_cycle_fp32():
    # 3-D 128^3 channel in the benchmark's precision: one stochastic FAC cycle
    # on a random state, compared over the whole field.
    n, dim = 128, 3
    m = S.SelmMG(dim=dim, n=n, precision=1, seed=0, instance=0)
    osys = grid.velocity_system(n, dim)
    z0 = selm_inputs.fields(osys.shapes(0), seed=21, scale=1e-2)
    z = to_dev(m.h, z0, torch.float64)
    S.selm_mg_fac_cycle(m.h, 0, z, None, cycle=3, noise=1)
    zero = osys.zeros(0)
    want = [x.copy() for x in z0]
    multigrid.fac_cycle(osys, want, zero, philox.PhiloxNoise(0, 0, 3), 1.0)
    got = from_dev(m.h, z)
    assert rel(got, want) < 1e-5
    # element-wise on the cycle's correction, per component and per z plane
    for g, w, a in zip(got, want, z0):
        dg, dw = g - a, w - a
        assert maxrel(dg, dw) < 1e-5
        for k in (0, 1, dw.shape[0] // 2, dw.shape[0] - 2, dw.shape[0] - 1):
            assert maxrel(dg[k], dw[k]) < 1e-5, k


@pytest.mark.parametrize("dim,n,levels", [(3, 32, 4), (3, 128, 6)])
def test_graph_replay_matches_direct_launches(dim, n, levels):
    """Solve V-cycles replayed from captured CUDA graphs (the default) give the
    solve of direct launches bit for bit, with the same cycle count (128^3:
    the cooperative level and the engine inside the graph).  The kernel
    launch counter credits each replay with the kernels its graph holds, so
    both forms count the same launches."""
    outs = []
    for graphs in (1, 0):
        m, osys, dt, tol = make(dim, n, levels, "fp32")
        S.selm_mg_set_option(m.h, S.SELM_OPT_GRAPHS, graphs)
        b0 = to_dev(m.h, selm_inputs.fields(osys.shapes(0), seed=16), torch.float64)
        z = empty(m.h, torch.float64)
        torch.cuda.synchronize()
        l0 = S.selm_kernel_launches()
        cycles, res = S.selm_mg_fac_solve(m.h, 0, z, b0, 1e-10, 50)
        launches = S.selm_kernel_launches() - l0
        assert res <= 1e-10 and cycles >= 3   # a capture and replays took part
        outs.append((cycles, z.cpu().numpy(), launches))
    assert outs[0][0] == outs[1][0]
    assert np.array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2] and outs[0][2] > 3 * levels


@pytest.mark.parametrize("coop", [1, 2])
def test_timed_out_wait_is_reported_and_cleared(coop):
    """A cooperative level launch whose wait gives up (its timeout flag raised,
    as a wait that ran out of time raises it) returns; the solve reports
    SELM_ECUDA at its next norm read and clears the flag; the next solve runs
    normally.  No GPU fault, no wait of a second."""
    m, osys, dt, tol = make(3, 64, 4, "fp32")
    S.selm_mg_set_option(m.h, S.SELM_OPT_LEVEL_COOP, coop)
    S.selm_mg_set_option(m.h, S.SELM_OPT_ENGINE_LEVEL, 2)
    b0 = to_dev(m.h, selm_inputs.fields(osys.shapes(0), seed=17), torch.float64)
    z = empty(m.h, torch.float64)
    S.selm_mg_fail_waits(m.h, 0)
    with pytest.raises(S.SelmError) as err:
        S.selm_mg_fac_solve(m.h, 0, z, b0, 1e-10, 50)
    assert err.value.status == S.SELM_ECUDA and "timed out" in str(err.value)
    z.zero_()
    cycles, res = S.selm_mg_fac_solve(m.h, 0, z, b0, 1e-10, 50)
    assert res <= 1e-10 and cycles >= 1


def test_create_rejects_misaligned_workspace():
    """Allocator hooks must return 256-byte aligned memory (the kernels use
    vector accesses): a block 16 bytes off fails create with SELM_EINVAL and
    goes back to the free hook."""
    blocks, freed = {}, []

    def alloc(nbytes, ctx):
        base = torch.cuda.caching_allocator_alloc(int(nbytes) + 512)
        blocks[base + 16] = base
        return base + 16

    def free(ptr, ctx):
        freed.append(ptr)
        torch.cuda.caching_allocator_delete(blocks.pop(ptr))

    a_cb, f_cb = S.ALLOC_FN(alloc), S.FREE_FN(free)
    d = S.make_desc(dim=2, n=32, torch_allocator=False)
    d.alloc, d.free = a_cb, f_cb
    with pytest.raises(S.SelmError) as err:
        S.selm_mg_create(d)
    assert err.value.status == S.SELM_EINVAL
    assert len(freed) == 1 and not blocks


def _exact_projection(w0, n):
    """P~ w = w - D^T phi with (D D^T) phi = D w - mean, from the closed-form
    spectral inverse of the Neumann pressure operator (independent of both the
    library and the oracle's iterative solve)."""
    from tests import closed_forms as cf
    div = projection.divergence(w0, 3)
    phi = cf.spectral_solve(("P", "P", "N"), n, 1.0, div - div.mean())
    g = projection.divergence_transpose(phi, 3)
    return [a - b for a, b in zip(w0, g)]


@pytest.mark.parametrize("n", [16, 64, 128])
def test_projection_spectral_inner_solve(n):
    """FP32 inner cycles on the uniform channel: the projection's pressure
    refinement takes the spectral inner solve by default; P~w equals the exact
    projection (closed form) to the solve tolerance and the V-cycle path's
    result, and the field is divergence-free."""
    m = S.SelmMG(dim=3, n=n, precision=S.SELM_FP32_REFINE64, projection=1, proj_tol=1e-12)
    assert S.selm_mg_pressure_spectral(m.h) == 1
    w0 = selm_inputs.fields(grid.velocity_system(n, 3, levels=1).shapes(0), seed=26)
    w = to_dev(m.h, w0, torch.float64)
    iters = S.selm_mg_project(m.h, w)
    assert 1 <= iters <= 5
    got = from_dev(m.h, w)
    want = _exact_projection(w0, n)
    assert rel(got, want) < 1e-10
    div = projection.divergence(got, 3)
    assert np.abs(div).max() < 1e-10 * np.abs(projection.divergence(w0, 3)).max()
    S.selm_mg_set_option(m.h, S.SELM_OPT_PRESSURE_SPECTRAL, 0)
    assert S.selm_mg_pressure_spectral(m.h) == 0
    w2 = to_dev(m.h, w0, torch.float64)
    S.selm_mg_project(m.h, w2)
    assert rel(from_dev(m.h, w2), got) < 1e-9


def test_projection_spectral_unavailable_in_fp64():
    m = S.SelmMG(dim=3, n=16, precision=S.SELM_FP64, projection=1)
    assert S.selm_mg_pressure_spectral(m.h) == 0
    with pytest.raises(S.SelmError):
        S.selm_mg_set_option(m.h, S.SELM_OPT_PRESSURE_SPECTRAL, 1)
