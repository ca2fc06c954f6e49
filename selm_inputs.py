"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

Holds no arithmetic of the method: only the recipes that draw particle
positions, forces and right-hand-side fields from numpy's PCG64 generator.
The workloads are channel flows on the unit box (periodic in x and y, walls at
z = 0 and z = 1); particles keep a clearance of a few cells from the walls.
"""

import numpy as np


def particles(npart, dim, n, seed, clearance_cells=2.0):
    """Positions (npart, dim): uniform in the periodic directions, uniform in
    [c h, 1 - c h] along the wall axis (last column), h = 1 / n."""
    rng = np.random.default_rng([int(seed), 101])
    X = rng.uniform(0.0, 1.0, size=(npart, dim))
    c = clearance_cells / n
    X[:, -1] = rng.uniform(c, 1.0 - c, size=npart)
    return X


def forces(npart, dim, seed):
    """Forces (npart, dim) with independent N(0, 1) entries."""
    rng = np.random.default_rng([int(seed), 202])
    return rng.standard_normal((npart, dim))


def fields(shapes, seed, scale=1.0):
    """List of N(0, scale^2) arrays with the given shapes."""
    rng = np.random.default_rng([int(seed), 303])
    return [scale * rng.standard_normal(s) for s in shapes]


def velocity_shapes(n, dim, level=0):
    """Array shapes (nz, ny, nx) of the MAC velocity components at a level.

    Components are the face-normal velocities; the wall-normal one has one
    fewer node along z (its wall nodes carry the no-slip value).
    """
    m = n >> level
    if dim == 3:
        return [(m, m, m), (m, m, m), (m - 1, m, m)]
    return [(m, 1, m), (m - 1, 1, m)]


def batched_edges(nsys, seed, choices=(32, 48, 64, 96, 128)):
    """Grid edges of a batch of independent channel systems."""
    rng = np.random.default_rng([int(seed), 404])
    return [int(x) for x in rng.choice(np.asarray(choices), size=nsys)]
