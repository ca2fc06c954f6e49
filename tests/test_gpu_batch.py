"""GPU: the batched form equals each system advanced alone.

Several independent channel systems of uneven size, each with its own seed,
instance and kT, are advanced by selm_batch_step, in its persistent form (one
cooperative launch per FAC cycle of all systems) and in its per-system graph
form (one graph launch per phase with a branch per system).  Each system is
also advanced alone by selm_mg_step from the same state.  The stochastic chains see the same Philox counters, so the
thermal fields agree to rounding; the deterministic solves stop at the
batch's slowest system, which only tightens the tolerance.  Trajectories must
agree to well within the FP32-inner tolerance, before and after the
autotuner changes the engine's cluster size.
"""

import numpy as np
import pytest
import torch

import selm_inputs

pytestmark = pytest.mark.gpu

SYSTEMS = [  # (dim, n, particles, kT, seed)
    (3, 16, 24, 0.5, 1),
    (3, 32, 40, 1.3, 2),
    (3, 48, 33, 2.0, 3),
    (2, 64, 16, 0.9, 4),
]


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_2680_gb300 import selm as mod
    mod.lib()
    return mod


FORMS = ["persistent", "graphs"]


def _batch(S, descs, form):
    b = S.selm_batch_create(descs)
    if form == "persistent":
        assert S.selm_batch_info(b)["persistent"] == 1, "the batch should qualify for the persistent form"
    else:
        S.selm_batch_set_persistent(b, 0)
    return b


def _descs(S):
    return [S.make_desc(dim=d, n=n, kT=kT, precision=S.SELM_FP32_REFINE64, seed=seed, instance=7 + i,
                        max_particles=256)
            for i, (d, n, npart, kT, seed) in enumerate(SYSTEMS)]


def _inputs():
    Xs, Fs = [], []
    for d, n, npart, kT, seed in SYSTEMS:
        Xs.append(selm_inputs.particles(npart, d, n, seed=seed))
        Fs.append(selm_inputs.forces(npart, d, seed=seed))
    return Xs, Fs


def _alone(S, descs, Xs, Fs, nsteps):
    out = []
    for desc, X0, F0 in zip(descs, Xs, Fs):
        h = S.selm_mg_create(desc)
        X = torch.tensor(X0, device="cuda")
        S.selm_mg_step(h, X, torch.tensor(F0, device="cuda"), 1e-3, nsteps, 2)
        torch.cuda.synchronize()
        out.append(X.cpu().numpy())
        S.selm_mg_destroy(h)
    return out


@pytest.mark.parametrize("form", FORMS)
def test_batch_matches_systems_alone(S, form):
    descs = _descs(S)
    Xs, Fs = _inputs()
    b = _batch(S, descs, form)
    X = [torch.tensor(x, device="cuda") for x in Xs]
    F = [torch.tensor(f, device="cuda") for f in Fs]
    cycles = S.selm_batch_step(b, X, F, 1e-3, 1, 2)
    l0 = S.selm_kernel_launches()   # the second step replays the graphs the first captured
    cycles += S.selm_batch_step(b, X, F, 1e-3, 1, 2)
    torch.cuda.synchronize()
    # replays credit the kernels they hold
    assert S.selm_kernel_launches() - l0 > (4 if form == "persistent" else 4 * len(SYSTEMS))
    assert all(1 <= c <= 15 for c in cycles)
    want = _alone(S, descs, Xs, Fs, 2)
    for i, (x, w, x0) in enumerate(zip(X, want, Xs)):
        err = np.linalg.norm(x.cpu().numpy() - w) / np.linalg.norm(w - x0)
        assert err < 1e-5, (i, err)
    # the chains advanced by the same counters
    for i in range(len(SYSTEMS)):
        h = S.selm_batch_system(b, i)
        assert S.selm_mg_chain(h)[1] == 4
    S.selm_batch_destroy(b)


@pytest.mark.parametrize("form", FORMS)
def test_batch_autotune_keeps_results(S, form):
    descs = _descs(S)
    Xs, Fs = _inputs()
    b = _batch(S, descs, form)
    chosen = S.selm_batch_autotune(b)   # tunes both forms and keeps the faster one
    info = S.selm_batch_info(b)
    assert info["kc"] in (8, 16, 32) and info["blocks_per_sm"] in (1, 2)
    assert chosen in (4, 8, 16) and info["cluster"] == chosen
    S.selm_batch_set_persistent(b, 1 if form == "persistent" else 0)   # the form under test, tuned
    X = [torch.tensor(x, device="cuda") for x in Xs]
    F = [torch.tensor(f, device="cuda") for f in Fs]
    S.selm_batch_step(b, X, F, 1e-3, 2, 2)
    torch.cuda.synchronize()
    want = _alone(S, descs, Xs, Fs, 2)
    for i, (x, w, x0) in enumerate(zip(X, want, Xs)):
        err = np.linalg.norm(x.cpu().numpy() - w) / np.linalg.norm(w - x0)
        assert err < 1e-5, (i, err)
    S.selm_batch_destroy(b)


def test_batch_rejects_projection(S):
    d = S.make_desc(dim=3, n=16, projection=S.SELM_PROJ_MAC)
    with pytest.raises(S.SelmError):
        S.selm_batch_create([d])


@pytest.mark.parametrize("form", FORMS)
def test_batch_at_benchmark_shapes(S, form):
    """Systems of every edge the batched benchmark draws (32..128, FP32 inner
    cycles with FP64 refinement, 64..2048 particles), with the engine cluster
    size the autotuner picks, as the benchmark runs them: the batch equals each
    system advanced alone."""
    import selm_inputs
    edges = [128, 96, 64, 48, 32]
    nps = [2048, 700, 64, 300, 1000]
    descs = [S.make_desc(dim=3, n=e, kT=0.5 + 0.3 * i, precision=S.SELM_FP32_REFINE64, seed=i, instance=i,
                         max_particles=2048) for i, e in enumerate(edges)]
    Xs = [selm_inputs.particles(npart, 3, e, seed=i) for i, (npart, e) in enumerate(zip(nps, edges))]
    Fs = [selm_inputs.forces(npart, 3, seed=i) for i, npart in enumerate(nps)]
    b = _batch(S, descs, form)
    S.selm_batch_autotune(b)
    S.selm_batch_set_persistent(b, 1 if form == "persistent" else 0)
    X = [torch.tensor(x, device="cuda") for x in Xs]
    F = [torch.tensor(f, device="cuda") for f in Fs]
    S.selm_batch_step(b, X, F, 1e-3, 2, 2)
    torch.cuda.synchronize()
    S.selm_batch_destroy(b)
    for desc, x, X0, F0 in zip(descs, X, Xs, Fs):
        h = S.selm_mg_create(desc)
        Xa = torch.tensor(X0, device="cuda")
        S.selm_mg_step(h, Xa, torch.tensor(F0, device="cuda"), 1e-3, 2, 2)
        torch.cuda.synchronize()
        w = Xa.cpu().numpy()
        err = np.linalg.norm(x.cpu().numpy() - w) / np.linalg.norm(w - X0)
        assert err < 1e-5, (desc.n, err)
        S.selm_mg_destroy(h)


class _Raw:
    """A device buffer of the library seen as a torch tensor (no copy)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f8", "data": (ptr, False), "version": 3}


def _fp64_descs(S):
    return [S.make_desc(dim=d, n=n, kT=kT, precision=S.SELM_FP64, seed=seed, instance=7 + i, max_particles=256)
            for i, (d, n, npart, kT, seed) in enumerate(SYSTEMS)]


def _level_size(S, h):
    return S.selm_mg_layout(h, S.SELM_SYS_VELOCITY, 0, 0)[2]


@pytest.mark.parametrize("form", FORMS)
def test_batch_cycle_sample_equals_each_chain_alone(S, form):
    descs = _fp64_descs(S)
    b = _batch(S, descs, form)
    for _ in range(3):
        S.selm_batch_cycle(b, S.SELM_BATCH_SAMPLE)
    torch.cuda.synchronize()
    for i, desc in enumerate(descs):
        hb = S.selm_batch_system(b, i)
        assert S.selm_mg_chain(hb)[1] == 3
        xb = torch.as_tensor(_Raw(S.selm_mg_chain(hb)[0], _level_size(S, hb)), device="cuda").clone()
        h = S.selm_mg_create(desc)
        X = torch.zeros((0, desc.dim), dtype=torch.float64, device="cuda")
        xa = torch.zeros_like(xb)
        S.selm_mg_sample(h, X, 3, torch.zeros_like(X), xa)
        torch.cuda.synchronize()
        assert (torch.linalg.vector_norm(xb - xa) / torch.linalg.vector_norm(xa)).item() < 1e-12
        S.selm_mg_destroy(h)
    with pytest.raises(S.SelmError):
        S.selm_batch_cycle(b, 7)
    S.selm_batch_destroy(b)


@pytest.mark.parametrize("form", FORMS)
def test_batch_cycle_solve_is_one_fac_cycle(S, form):
    # after a step, each system's solve iterate u (perturbed here) goes through
    # one deterministic FAC cycle with the step's right-hand side Gamma^T F
    from oracle import coupling, grid, multigrid
    from oracle.philox import ExplicitNoise
    from tests.gpu_util import from_dev
    descs = _fp64_descs(S)
    Xs, Fs = _inputs()
    b = _batch(S, descs, form)
    X = [torch.tensor(x, device="cuda") for x in Xs]
    F = [torch.tensor(f, device="cuda") for f in Fs]
    S.selm_batch_step(b, X, F, 1e-3, 1, 1)
    torch.cuda.synchronize()
    rng = np.random.default_rng(9)
    starts = []
    for i in range(len(descs)):
        hb = S.selm_batch_system(b, i)
        u = torch.as_tensor(_Raw(S.selm_mg_velocity(hb), _level_size(S, hb)), device="cuda")
        u += torch.tensor(rng.standard_normal(u.numel()), device="cuda")
        starts.append(u.clone())
    torch.cuda.synchronize()
    S.selm_batch_cycle(b, S.SELM_BATCH_SOLVE)
    torch.cuda.synchronize()
    for i, ((d, n, npart, kT, seed), u0) in enumerate(zip(SYSTEMS, starts)):
        hb = S.selm_batch_system(b, i)
        u1 = torch.as_tensor(_Raw(S.selm_mg_velocity(hb), _level_size(S, hb)), device="cuda").clone()
        osys = grid.velocity_system(n, d, mu=1.0)
        rhs = coupling.spread(osys, Fs[i], Xs[i])
        z0 = from_dev(hb, u0)
        want = multigrid.fac_cycle(osys, [x.copy() for x in z0], rhs, ExplicitNoise(), 0.0)
        got = from_dev(hb, u1)
        dg = np.concatenate([(g - z).ravel() for g, z in zip(got, z0)])
        dw = np.concatenate([(w - z).ravel() for w, z in zip(want, z0)])
        assert np.linalg.norm(dg - dw) / np.linalg.norm(dw) < 1e-12, i
    S.selm_batch_destroy(b)
