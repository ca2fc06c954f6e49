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
