"""Writes the exact covariance block of the composite sampler's probe sites.

The stochastic composite FAC cycle keeps xi ~ N(0, A^-1) invariant (Section 3,
Eqs. equ_G_special_form and equ_g_gen_xi; invariance of the Galerkin
hierarchy in Section 3.2), so the covariance of xi at a set of probe sites is
the block of A^-1 on those sites.  This script computes that block with the
oracle's deterministic composite FAC solve (oracle/composite.py, Algorithms 1
and 2) and nothing else, and stores it as text next to itself.

Probe block (the 256^3 channel with the bottom 32 base rows refined): 64
unknowns of one component straddling the coarse-fine interface -- x and y
indices 126..129 in each level's own indexing; in z the two fine layers just
below the interface (m = 2K-2, 2K-1) and the two uncovered base rows just above
it (j = K+1, K+2, array rows K, K+1).  Order: layer, then y, then x.

The composite grid is invariant under shifts by whole base cells along x and
y (two fine cells), so A^-1 e_j for a probe site j that is such a shift of
another probe site is that site's column shifted: one solve per fine-cell
parity class (x, y even or odd) and layer, and one per base row -- ten solves.

Usage: python tests/golden/make_composite_probe_cov.py [n K] [--procs P]
(default 256 32; each solve takes tens of minutes of one core at that size).
"""

import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))


def probe_sites(n, K):
    """[(part, z, y, x)] of the 64 probe unknowns: part 0 = fine (layer m), 1 = base (array row)."""
    out = []
    for part, z in ((0, 2 * K - 2), (0, 2 * K - 1), (1, K), (1, K + 1)):
        for y in range(126 * n // 256, 126 * n // 256 + 4):
            for x in range(126 * n // 256, 126 * n // 256 + 4):
                out.append((part, z, y, x))
    return out


def representative(site):
    """The solve whose shifted column gives this site's column, and the shift (base cells)."""
    part, z, y, x = site
    if part == 0:
        return (0, z, y & 1, x & 1), (y >> 1, x >> 1)
    return (1, z, 0, 0), (y, x)


def _solve_one(args):
    n, K, site, tol = args
    sys.path.insert(0, ROOT)
    from oracle import composite as OC
    t0 = time.time()
    cg = OC.CompositeGrid(n, K, 3, mu=1.0, ncomp=1)
    part, z, y, x = site
    e = np.zeros(cg.size)
    idx = cg.fine_index(z, y, x) if part == 0 else cg.base_index(z, y, x)
    e[idx] = 1.0
    sol, cycles, rel = OC.solve(cg, [e], tol=tol)
    fine, base = cg.from_vec(sol[0])
    print(f"site {site}: {cycles} cycles, residual {rel:.1e}, {time.time() - t0:.0f} s", flush=True)
    return site, fine, base


def block(n, K, procs=1, tol=1e-9):
    sites = probe_sites(n, K)
    reps = sorted({representative(s)[0] for s in sites})
    args = [(n, K, r, tol) for r in reps]
    if procs > 1:
        with mp.get_context("spawn").Pool(procs) as pool:
            cols = dict((r, (f, b)) for r, f, b in pool.map(_solve_one, args))
    else:
        cols = dict((r, (f, b)) for r, f, b in map(_solve_one, args))
    C = np.zeros((len(sites), len(sites)))
    for j, sj in enumerate(sites):
        rep, (sy, sx) = representative(sj)
        f, b = cols[rep]
        f = np.roll(f, (2 * sy, 2 * sx), axis=(1, 2))
        b = np.roll(b, (sy, sx), axis=(1, 2))
        for i, (part, z, y, x) in enumerate(sites):
            C[i, j] = f[z, y, x] if part == 0 else b[z, y, x]
    return C


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("n", nargs="?", type=int, default=256)
    ap.add_argument("K", nargs="?", type=int, default=32)
    ap.add_argument("--procs", type=int, default=1)
    a = ap.parse_args()
    C = block(a.n, a.K, a.procs)
    asym = np.abs(C - C.T).max() / np.abs(C).max()
    path = os.path.join(HERE, f"composite_probe_cov_n{a.n}_K{a.K}.txt")
    hdr = (f"A^-1 on the 64 probe unknowns of the composite channel n={a.n}, K={a.K}, mu=1 "
           f"(one component; Section 3 invariance: the stochastic composite FAC samples N(0, A^-1)).\n"
           f"Written by tests/golden/make_composite_probe_cov.py from the oracle's composite FAC solve "
           f"(tol 1e-9); order: layer (fine m=2K-2, 2K-1; base rows K, K+1), y, x; "
           f"x, y = {126 * a.n // 256}..{126 * a.n // 256 + 3}.  max|C - C^T|/max|C| = {asym:.1e}")
    np.savetxt(path, C, fmt="%.12e", header=hdr)
    print("wrote", path, "asymmetry", asym)


if __name__ == "__main__":
    main()
