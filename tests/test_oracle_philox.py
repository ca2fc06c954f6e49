"""Pins for the oracle's counter-based normals (oracle/philox.py)."""

import os

import numpy as np

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        vals = [int(t, 16) for t in line.split()]
        rows.append((vals[0:4], vals[4:6], vals[6:10]))
    return rows


def test_philox_known_answers():
    for ctr, key, out in _kat():
        got = philox.philox4x32_10(np.array(ctr, dtype=np.uint32), key)
        assert [int(x) for x in got] == out


def test_philox_vectorised_equals_scalar():
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2 ** 32, size=(64, 4), dtype=np.uint64).astype(np.uint32)
    key = (0x12345678, 0x9ABCDEF0)
    batch = philox.philox4x32_10(ctr, key)
    for i in range(64):
        assert np.array_equal(batch[i], philox.philox4x32_10(ctr[i], key))


def test_box_muller_moments():
    # 4e5 normals from one stream: mean 0, variance 1, kurtosis 3 (textbook N(0,1))
    n = philox.normals_for_ranks(philox.make_key(7, 3), philox.pack_ctr1(0, 0, 0, 0, 0), 5,
                                 400_000)
    assert abs(n.mean()) < 5 / np.sqrt(n.size)
    assert abs(n.var() - 1.0) < 5 * np.sqrt(2.0 / n.size)
    kurt = np.mean(n ** 4) / np.mean(n ** 2) ** 2
    assert abs(kurt - 3.0) < 0.05
    # the two members of a Box-Muller pair are uncorrelated
    blocks = n[: (n.size // 4) * 4].reshape(-1, 4)
    assert abs(np.corrcoef(blocks[:, 0], blocks[:, 1])[0, 1]) < 0.02


def test_rank_to_lane_mapping():
    key = philox.make_key(0, 0)
    c1 = philox.pack_ctr1(2, 1, 3, 1, 0)
    n = philox.normals_for_ranks(key, c1, 9, 10)
    for rank in range(10):
        ctr = np.array([rank >> 2, c1, 9, 0], dtype=np.uint32)
        blk = philox.words_to_normals(philox.philox4x32_10(ctr, key))
        assert n[rank] == blk[rank & 3]


def test_streams_distinct():
    key = philox.make_key(0, 0)
    a = philox.normals_for_ranks(key, philox.pack_ctr1(0, 0, 0, 0, 0), 0, 16)
    b = philox.normals_for_ranks(key, philox.pack_ctr1(0, 0, 1, 0, 0), 0, 16)
    c = philox.normals_for_ranks(key, philox.pack_ctr1(0, 0, 0, 0, 0), 1, 16)
    d = philox.normals_for_ranks(philox.make_key(0, 1), philox.pack_ctr1(0, 0, 0, 0, 0), 0, 16)
    for x in (b, c, d):
        assert not np.allclose(a, x)
