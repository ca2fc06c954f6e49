"""Lag correlations of the library's two stochastic samplers (Section 5).

Section 5 judges a sampler by how strongly its variates stay correlated after
a given number of iterations, and contrasts the multigrid sampler (O(1)
iterations) with stochastic Gauss-Seidel (correlated after many).  For a
sampler z' = M z + N b + B n with invariant law N(0, A^-1) (b = 0) and a
linear observable phi, the lag-k covariance follows Section 3.1's recurrence
C^(0,k) = M^k C^(0,0) with C^(0,0) = A^-1, so the lag-k correlation is

    rho(k) = phi^T M^k A^-1 phi / phi^T A^-1 phi,

obtained without sampling: w = A^-1 phi by the deterministic FAC solve, then
k noiseless iterations from w, each followed by the inner product with phi.

* Multigrid sampler: one iteration is one FAC cycle (Algorithm 1, V-cycle of
  Algorithm 3) on the FP64 state, ``selm_mg_fac_cycle``.
* Gauss-Seidel sampler: one iteration is one red-black sweep of the fine grid
  (Section 3.1) on the inner-precision state, ``selm_mg_smooth`` at level 0.

Every iteration runs in the library's kernels; the host only reads the state
back and forms the inner product in float64.
"""

import math

import numpy as np
import torch

from . import selm as S


def _components(h):
    out = []
    for c in range(S.selm_mg_ncomp(h, S.SELM_SYS_VELOCITY)):
        (nx, ny, nz), off, size = S.selm_mg_layout(h, S.SELM_SYS_VELOCITY, 0, c)
        out.append(((nz, ny, nx), off, size))
    return out


def wall_mode(h, n):
    """Host float64 field: component 0 = sin(pi z) at its nodes (uniform along the
    periodic axes), other components 0.  Component 0 sits on the cell lattice
    across the walls (n nodes at (k + 1/2)/n) or the vertex lattice (n - 1
    interior nodes at (k + 1)/n)."""
    comps = _components(h)
    phi = np.zeros(comps[0][2])
    (nz, ny, nx), off, _ = comps[0]
    if nz == n:
        z = (np.arange(nz) + 0.5) / n
    elif nz == n - 1:
        z = (np.arange(nz) + 1.0) / n
    else:
        raise ValueError("component 0 is not on a wall-normal lattice of the grid")
    phi[off:off + nz * ny * nx] = np.repeat(np.sin(math.pi * z), ny * nx)
    return phi


def point_probe(h):
    """Host float64 field: unit value at the centre node of component 0."""
    comps = _components(h)
    phi = np.zeros(comps[0][2])
    (nz, ny, nx), off, _ = comps[0]
    phi[off + ((nz // 2) * ny + ny // 2) * nx + nx // 2] = 1.0
    return phi


def covariance_image(h, phi, tol=1e-10, max_cycles=100):
    """w = A^-1 phi on the device (FP64), by the library's FAC solve.  The
    default tolerance is the solve's: for a smooth phi on a large grid the FP64
    residual b - Aw itself rounds at ~1e-16 |A||w| / |b| (about 2e-12 for the
    wall mode at 128^3), so much tighter tolerances are not reachable."""
    b = torch.tensor(phi, dtype=torch.float64, device="cuda")
    w = torch.zeros_like(b)
    cycles, res = S.selm_mg_fac_solve(h, S.SELM_SYS_VELOCITY, w, b, tol, max_cycles)
    if not res <= tol:
        raise RuntimeError(f"covariance image: residual {res:g} above {tol:g}")
    return w


class _Reader:
    """Reads a device field back into pinned memory and forms phi . z in float64."""

    def __init__(self, phi, dtype):
        self.phi = phi
        self.host = torch.empty(phi.size, dtype=dtype, pin_memory=True)

    def dot(self, z):
        self.host.copy_(z)
        return float(np.dot(self.phi, self.host.numpy().astype(np.float64, copy=False)))


def lag_correlations_mg(h, phi, K, w=None):
    """rho(0..K) of the multigrid sampler (noiseless FAC cycles with b = 0)."""
    w = covariance_image(h, phi) if w is None else w
    z = w.clone()
    zero = torch.zeros_like(z)
    rd = _Reader(phi, torch.float64)
    var = rd.dot(z)
    rho = [1.0]
    for k in range(K):
        S.selm_mg_fac_cycle(h, S.SELM_SYS_VELOCITY, z, zero, k, 0)
        rho.append(rd.dot(z) / var)
    return np.array(rho)


def lag_correlations_gs(h, phi, K, w=None):
    """rho(0..K) of the Gauss-Seidel sampler (noiseless fine-grid sweeps with b = 0),
    iterated in the handle's inner precision."""
    w = covariance_image(h, phi) if w is None else w
    dt = torch.float32 if S.selm_mg_inner_bytes(h) == 4 else torch.float64
    v = w.to(dt)
    zero = torch.zeros_like(v)
    rd = _Reader(phi, dt)
    var = rd.dot(v)
    rho = [1.0]
    for k in range(K):
        S.selm_mg_smooth(h, S.SELM_SYS_VELOCITY, 0, v, zero, 0, k, 0)
        rho.append(rd.dot(v) / var)
    return np.array(rho)


def integrated_time(rho):
    """1 + 2 sum_{k>=1} rho(k) over the computed lags (a lower bound when the
    curve is still positive at its last lag)."""
    return 1.0 + 2.0 * float(np.sum(rho[1:]))


def lags_below(rho, threshold=0.05):
    """First lag k with |rho(j)| < threshold for every computed j >= k, else None."""
    above = np.nonzero(np.abs(rho) >= threshold)[0]
    k = int(above[-1]) + 1 if above.size else 0
    return k if k < len(rho) else None
