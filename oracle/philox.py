"""Counter-based Gaussian noise for the stochastic smoother (oracle side).

The stochastic Gauss-Seidel iteration (Section 3.1, Eq. equ_def_Q_GS) needs
one standard normal n_i per updated site.  The paper does not say how they are
drawn; the method only needs them independent N(0,1).  To let a GPU and this
CPU code draw the *same* variates, both sides implement the Philox4x32-10
counter-based generator from its published definition (Salmon, Moraes, Dror,
Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11) and the Box-Muller
transform (Box & Muller, Ann. Math. Stat. 1958).  This file is the oracle's own
implementation; the CUDA library has an independent one.

Stream layout (a convention of this project, stated once here and in the C
header):

* key   = (lo32(seed) ^ hi32(instance),  hi32(seed) ^ lo32(instance))
* ctr0  = group index = (rank of the site within its colour class) >> 2
* ctr1  = level | comp << 4 | (colour & 15) << 8 | sweep << 12 | kind << 20
          | (colour >> 4) << 24
          (kind 0 = smoother sweep, kind 1 = exact coarsest-level sample,
          kind 2 = sweep of a refined patch, whose sites are addressed by
          a counter index of their own instead of a class rank; colours
          beyond 15, which only the general sparse levels of the staggered
          composite grid have, continue in the top byte, so every stream of
          a colour below 16 keeps its counter)
* ctr2, ctr3 = lo32(cycle), hi32(cycle)   (cycle = chain step counter)

One Philox call yields four 32-bit words w0..w3 -> uniforms
u_k = (w_k + 1/2) 2^-32 -> two Box-Muller pairs
(n0, n1) = sqrt(-2 ln u0) (cos 2 pi u1, sin 2 pi u1),
(n2, n3) = sqrt(-2 ln u2) (cos 2 pi u3, sin 2 pi u3);
lane (rank & 3) of the group takes n_lane.
"""

import numpy as np

# Philox4x32 round multipliers and Weyl key increments (Salmon et al. 2011).
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK32 = 0xFFFFFFFF

KIND_SWEEP = 0
KIND_COARSEST = 1
KIND_PATCH = 2


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds.

    ctr : uint32 array of shape (..., 4)
    key : pair of ints (k0, k1), each < 2**32
    returns uint32 array of shape (..., 4)
    """
    ctr = np.asarray(ctr, dtype=np.uint32)
    c0, c1, c2, c3 = (ctr[..., i].astype(np.uint64) for i in range(4))
    k0 = int(key[0]) & _MASK32
    k1 = int(key[1]) & _MASK32
    m0 = np.uint64(PHILOX_M0)
    m1 = np.uint64(PHILOX_M1)
    mask = np.uint64(_MASK32)
    sh = np.uint64(32)
    for rnd in range(10):
        if rnd > 0:  # the key is bumped between rounds
            k0 = (k0 + PHILOX_W0) & _MASK32
            k1 = (k1 + PHILOX_W1) & _MASK32
        p0 = c0 * m0  # 32 x 32 -> 64 bit products, exact in uint64
        p1 = c2 * m1
        hi0, lo0 = p0 >> sh, p0 & mask
        hi1, lo1 = p1 >> sh, p1 & mask
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1,
                          hi0 ^ c3 ^ np.uint64(k1), lo0)
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def make_key(seed, instance=0):
    seed = int(seed) & ((1 << 64) - 1)
    instance = int(instance) & ((1 << 64) - 1)
    k0 = (seed & _MASK32) ^ (instance >> 32)
    k1 = (seed >> 32) ^ (instance & _MASK32)
    return (k0, k1)


def pack_ctr1(level, comp, colour, sweep, kind):
    assert 0 <= level < 16 and 0 <= comp < 16 and 0 <= colour < 4096
    assert 0 <= sweep < 256 and 0 <= kind < 16
    return (level | (comp << 4) | ((colour & 15) << 8) | (sweep << 12) | (kind << 20)
            | ((colour >> 4) << 24))


def words_to_normals(words):
    """Box-Muller on one Philox output block: (..., 4) uint32 -> (..., 4) float64."""
    u = (words.astype(np.float64) + 0.5) * 2.0 ** -32
    r01 = np.sqrt(-2.0 * np.log(u[..., 0]))
    r23 = np.sqrt(-2.0 * np.log(u[..., 2]))
    t1 = 2.0 * np.pi * u[..., 1]
    t3 = 2.0 * np.pi * u[..., 3]
    return np.stack([r01 * np.cos(t1), r01 * np.sin(t1),
                     r23 * np.cos(t3), r23 * np.sin(t3)], axis=-1)


def normals_for_ranks(key, ctr1, cycle, nsites):
    """Normals for ranks 0..nsites-1 of one colour class (one counter stream)."""
    ngroups = (nsites + 3) // 4
    ctr = np.zeros((ngroups, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(ngroups, dtype=np.uint64).astype(np.uint32)
    ctr[:, 1] = ctr1
    ctr[:, 2] = int(cycle) & _MASK32
    ctr[:, 3] = (int(cycle) >> 32) & _MASK32
    n = words_to_normals(philox4x32_10(ctr, key))
    return n.reshape(-1)[:nsites]


def normals_for_indices(key, ctr1, cycle, idx):
    """Normals for sites addressed by linear index: group idx >> 2, lane idx & 3."""
    idx = np.asarray(idx, dtype=np.int64)
    if idx.size == 0:
        return np.zeros(0)
    ctr = np.zeros((idx.size, 4), dtype=np.uint32)
    ctr[:, 0] = (idx >> 2).astype(np.uint64).astype(np.uint32)
    ctr[:, 1] = ctr1
    ctr[:, 2] = int(cycle) & _MASK32
    ctr[:, 3] = (int(cycle) >> 32) & _MASK32
    n = words_to_normals(philox4x32_10(ctr, key))
    return n[np.arange(idx.size), idx & 3]


class PhiloxNoise:
    """Noise source for one stochastic cycle of one chain.

    ``sweep(level, comp, colour, sweep, nsites)`` returns the normals of the
    sites of one colour class in rank order; ``coarsest(level, comp, n)`` the
    normals of the exact coarsest-level sample.
    """

    def __init__(self, seed, instance, cycle):
        self.key = make_key(seed, instance)
        self.cycle = int(cycle)

    def sweep(self, level, comp, colour, sweep, nsites):
        c1 = pack_ctr1(level, comp, colour, sweep, KIND_SWEEP)
        return normals_for_ranks(self.key, c1, self.cycle, nsites)

    def coarsest(self, level, comp, n):
        c1 = pack_ctr1(level, comp, 0, 0, KIND_COARSEST)
        return normals_for_ranks(self.key, c1, self.cycle, n)

    def patch(self, comp, pass_id, sweep, idx):
        """Normals of refined-patch sites (counter indices idx) in one pass."""
        c1 = pack_ctr1(0, comp, pass_id, sweep, KIND_PATCH)
        return normals_for_indices(self.key, c1, self.cycle, idx)


class ExplicitNoise:
    """Noise source that hands out consecutive entries of a given vector.

    Used by the pins to treat the cycle as an affine map of its noise
    (probing with unit vectors).  ``count`` records how many were consumed.
    """

    def __init__(self, vec=None):
        self.vec = None if vec is None else np.asarray(vec, dtype=np.float64)
        self.count = 0

    def _take(self, n):
        if self.vec is None:
            out = np.zeros(n)
        else:
            out = self.vec[self.count:self.count + n]
            assert out.shape[0] == n, "noise vector too short"
        self.count += n
        return out

    def sweep(self, level, comp, colour, sweep, nsites):
        return self._take(nsites)

    def coarsest(self, level, comp, n):
        return self._take(n)

    def patch(self, comp, pass_id, sweep, idx):
        return self._take(len(idx))
