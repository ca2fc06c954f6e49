"""GPU: the served form gives each request the same result alone and in the mix.

Requests of uneven sizes (2-D and 3-D channels, own seeds, kT, particle
counts and step counts) are served twice: one at a time (one slot), and all
submitted at once to a server with several slots and a device budget that
admits only part of them together, so later requests are admitted as memory
frees up while others run.  Every request's final positions must agree
between the two runs; the budget and the slot count must never be exceeded,
and more than one request must have been on the device at once.
"""

import numpy as np
import pytest
import torch

import selm_inputs

pytestmark = pytest.mark.gpu

REQUESTS = [  # (dim, n, particles, nsteps, kT, seed)
    (3, 16, 20, 3, 0.7, 11),
    (2, 64, 16, 2, 1.0, 12),
    (3, 24, 40, 4, 1.6, 13),
    (3, 32, 30, 2, 0.5, 14),
    (2, 128, 50, 3, 2.0, 15),
    (3, 16, 8, 1, 1.2, 16),
]


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1003_2680_gb300 import selm as mod
    mod.lib()
    return mod


def _desc(S, dim, n, kT, seed):
    return S.make_desc(dim=dim, n=n, kT=kT, precision=S.SELM_FP32_REFINE64, seed=seed, instance=seed,
                       torch_allocator=False)


def _serve(S, budget, slots, requests=REQUESTS):
    srv = S.selm_server_create(budget, slots)
    Xs, Fs = [], []
    for i, (dim, n, npart, nsteps, kT, seed) in enumerate(requests):
        X = np.ascontiguousarray(selm_inputs.particles(npart, dim, n, seed=seed))
        F = np.ascontiguousarray(selm_inputs.forces(npart, dim, seed=seed))
        Xs.append(X)
        Fs.append(F)
        S.selm_server_submit(srv, _desc(S, dim, n, kT, seed), X, F, 1e-3, nsteps, 2, user=i + 1)
    S.selm_server_drain(srv)
    results = S.selm_server_poll(srv)
    stats = S.selm_server_stats(srv)
    S.selm_server_destroy(srv)
    return Xs, results, stats


def test_each_request_same_alone_and_in_the_mix(S):
    sizes = [S.selm_mg_footprint(_desc(S, d, n, kT, seed)) for d, n, _, _, kT, seed in REQUESTS]
    X_alone, res_alone, st_alone = _serve(S, budget=max(sizes) + (1 << 20), slots=1)
    budget = sum(sorted(sizes)[-3:]) + (1 << 20)       # admits about three at once
    X_mix, res_mix, st_mix = _serve(S, budget=budget, slots=4)
    assert len(res_alone) == len(res_mix) == len(REQUESTS)
    assert all(r["status"] == 0 for r in res_alone + res_mix)
    assert st_alone["peak_slots"] == 1
    assert 2 <= st_mix["peak_slots"] <= 4
    assert st_mix["peak_bytes"] <= budget
    X0 = [selm_inputs.particles(npart, d, n, seed=seed) for d, n, npart, _, _, seed in REQUESTS]
    for i, (a, m, x0) in enumerate(zip(X_alone, X_mix, X0)):
        assert not np.array_equal(a, x0)            # the particles moved
        err = np.linalg.norm(m - a) / np.linalg.norm(a - x0)
        assert err < 1e-9, (i, err)
    # the served clock orders submit <= admit <= done
    for r in res_mix:
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]


def test_request_larger_than_pool_is_refused(S):
    srv = S.selm_server_create(1 << 20, 1)
    X = np.zeros((4, 3))
    with pytest.raises(S.SelmError) as info:
        S.selm_server_submit(srv, _desc(S, 3, 64, 1.0, 0), X, X, 1e-3, 1, 2)
    assert info.value.status == S.SELM_EBUSY
    S.selm_server_destroy(srv)


BENCH_REQUESTS = [  # the served benchmark's extremes: 2-D edges to 1024, 3-D to 192, 16..4096 particles
    (2, 1024, 4096, 2, 1.0, 21),
    (3, 192, 16, 1, 1.0, 22),
    (2, 256, 700, 3, 1.0, 23),
    (3, 32, 2500, 2, 1.0, 24),
    (3, 128, 300, 1, 1.0, 25),
]


def test_benchmark_shapes_same_alone_and_in_the_mix(S):
    """The served benchmark's configuration (12 slots, 32 GB pool) on requests
    of its largest and smallest shapes: every request ends where it ends when
    served alone."""
    X_alone, res_alone, _ = _serve(S, budget=32 << 30, slots=1, requests=BENCH_REQUESTS)
    X_mix, res_mix, st_mix = _serve(S, budget=32 << 30, slots=12, requests=BENCH_REQUESTS)
    assert all(r["status"] == 0 for r in res_alone + res_mix)
    assert st_mix["peak_slots"] >= 2
    X0 = [selm_inputs.particles(npart, d, n, seed=seed) for d, n, npart, _, _, seed in BENCH_REQUESTS]
    for i, (a, m, x0) in enumerate(zip(X_alone, X_mix, X0)):
        assert not np.array_equal(a, x0)
        err = np.linalg.norm(m - a) / np.linalg.norm(a - x0)
        assert err < 1e-9, (i, err)


def test_served_results_equal_the_oracle(S):
    """Two FP64 requests served side by side (two slots, both on the device at
    once) end where the oracle's Euler-Maruyama steps (Algorithm 4) put them."""
    from oracle import selm as oselm
    reqs = [(3, 16, 20, 3, 0.7, 31, 3), (2, 32, 12, 2, 1.4, 32, 4)]   # dim, n, np, steps, kT, seed, levels
    srv = S.selm_server_create(1 << 30, 2)
    Xs = []
    for i, (dim, n, npart, nsteps, kT, seed, levels) in enumerate(reqs):
        X = np.ascontiguousarray(selm_inputs.particles(npart, dim, n, seed=seed))
        F = np.ascontiguousarray(selm_inputs.forces(npart, dim, seed=seed))
        Xs.append(X)
        d = S.make_desc(dim=dim, n=n, kT=kT, levels=levels, precision=S.SELM_FP64, seed=seed, instance=seed,
                        torch_allocator=False)
        S.selm_server_submit(srv, d, X, F, 1e-3, nsteps, 2, user=i + 1)
    S.selm_server_drain(srv)
    results = S.selm_server_poll(srv)
    stats = S.selm_server_stats(srv)
    S.selm_server_destroy(srv)
    assert len(results) == 2 and all(r["status"] == 0 for r in results)
    assert stats["peak_slots"] == 2
    for (dim, n, npart, nsteps, kT, seed, levels), X in zip(reqs, Xs):
        X0 = selm_inputs.particles(npart, dim, n, seed=seed)
        F0 = selm_inputs.forces(npart, dim, seed=seed)
        om = oselm.Model(n, dim, kT=kT, levels=levels, seed=seed, instance=seed)
        Xo = X0.copy()
        for _ in range(nsteps):
            Xo, _ = om.em_step(Xo, F0, 1e-3, 2)
        err = np.linalg.norm(X - Xo) / np.linalg.norm(Xo - X0)
        assert err < 1e-12, (dim, n, err)


def _serve_batched(S, budget, slots, persistent, requests=REQUESTS, dts=None):
    srv = S.selm_server_create_batched(budget, slots, persistent)
    Xs = []
    for i, (dim, n, npart, nsteps, kT, seed) in enumerate(requests):
        X = np.ascontiguousarray(selm_inputs.particles(npart, dim, n, seed=seed))
        F = np.ascontiguousarray(selm_inputs.forces(npart, dim, seed=seed))
        Xs.append((X, F))
        dt = 1e-3 if dts is None else dts[i]
        S.selm_server_submit(srv, _desc(S, dim, n, kT, seed), X, F, dt, nsteps, 2, user=i + 1)
    S.selm_server_drain(srv)
    results = S.selm_server_poll(srv)
    stats = S.selm_server_stats(srv)
    bstats = S.selm_server_batch_stats(srv)
    S.selm_server_destroy(srv)
    return [x for x, _ in Xs], results, stats, bstats


# Requests of one and two steps: short enough for an element-wise comparison
# with their runs alone (a rounding-level difference grows about 15x per step
# at these resolutions, reading R27), uneven enough that members retire and
# join between ticks.
BATCH_REQUESTS = [  # (dim, n, particles, nsteps, kT, seed)
    (3, 16, 20, 1, 0.7, 41),
    (2, 64, 16, 2, 1.0, 42),
    (3, 24, 40, 1, 1.6, 43),
    (3, 32, 30, 2, 0.5, 44),
    (2, 128, 50, 1, 2.0, 45),
    (3, 16, 8, 1, 1.2, 46),
    (2, 64, 24, 2, 0.9, 47),
]


@pytest.mark.parametrize("persistent", [True, False])
def test_continuous_batching_same_as_alone(S, persistent):
    """Requests served by continuous batching (one batched step of every
    admitted request per tick, members retired and admitted between ticks)
    end where they end when served alone.  The batched step differs from the
    one alone only by the extra FAC cycles a batched solve gives the systems
    that converge first and by the FP32 summation order of the batched
    kernels: within 1e-5 of the displacement after one step, and within one
    step's growth of that (reading R27) after two."""
    reqs = BATCH_REQUESTS
    sizes = [S.selm_mg_footprint(_desc(S, d, n, kT, seed)) for d, n, _, _, kT, seed in reqs]
    X_alone, res_alone, _ = _serve(S, budget=max(sizes) + (1 << 20), slots=1, requests=reqs)
    budget = sum(sorted(sizes)[-3:]) + (1 << 20)
    X_b, res_b, st_b, bst = _serve_batched(S, budget, 4, persistent, requests=reqs)
    assert len(res_b) == len(reqs) and all(r["status"] == 0 for r in res_b)
    assert 2 <= st_b["peak_slots"] <= 4 and st_b["peak_bytes"] <= budget
    # more than one membership: members retire at different ticks
    assert bst["rebuilds"] >= 2 and bst["steps"] >= 2
    X0 = [selm_inputs.particles(npart, d, n, seed=seed) for d, n, npart, _, _, seed in reqs]
    for i, (a, m, x0, r) in enumerate(zip(X_alone, X_b, X0, reqs)):
        assert not np.array_equal(m, x0)
        err = np.linalg.norm(m - a) / np.linalg.norm(a - x0)
        assert err < (1e-5 if r[3] == 1 else 3e-4), (i, err)
    for r in res_b:
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]


def test_continuous_batching_groups_by_step_parameters(S):
    """A request whose dt differs from the running batch's waits for the
    batch to drain and then runs in a batch of its own; every result still
    equals its run alone."""
    reqs = [r[:3] + (1,) + r[4:] for r in BATCH_REQUESTS[:4]]     # one step each
    dts = [1e-3, 2e-3, 1e-3, 2e-3]
    X_b, res_b, _, bst = _serve_batched(S, 1 << 30, 4, True, requests=reqs, dts=dts)
    assert all(r["status"] == 0 for r in res_b)
    for (dim, n, npart, nsteps, kT, seed), x, dt in zip(reqs, X_b, dts):
        X0 = selm_inputs.particles(npart, dim, n, seed=seed)
        F0 = selm_inputs.forces(npart, dim, seed=seed)
        h = S.selm_mg_create(_desc(S, dim, n, kT, seed))
        X = torch.tensor(X0, device="cuda")
        S.selm_mg_step(h, X, torch.tensor(F0, device="cuda"), dt, nsteps, 2)
        torch.cuda.synchronize()
        want = X.cpu().numpy()
        S.selm_mg_destroy(h)
        assert np.linalg.norm(x - want) / np.linalg.norm(want - X0) < 1e-5


def test_continuous_batching_rejects_projection(S):
    srv = S.selm_server_create_batched(1 << 28, 2, True)
    X = np.zeros((4, 3))
    d = S.make_desc(dim=3, n=16, projection=S.SELM_PROJ_MAC, torch_allocator=False)
    with pytest.raises(S.SelmError) as info:
        S.selm_server_submit(srv, d, X, X, 1e-3, 1, 2)
    assert info.value.status == S.SELM_EINVAL
    S.selm_server_destroy(srv)
