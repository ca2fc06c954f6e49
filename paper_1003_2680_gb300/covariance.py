"""Sample covariance of the library's thermal chains on a probe block (Section 3).

The stochastic multigrid cycle keeps xi ~ N(0, A^-1) invariant (Eqs.
equ_G_special_form and equ_g_gen_xi; the Galerkin coarse levels of Section 3.2
keep the invariance exact), so the covariance of the chain state on a block
of sites must approach the block of A^-1 on those sites.  This module draws
the chain's samples through the C ABI (``selm_mg_sample``,
``selm_comp_sample``) and estimates that block.

The grids are translation invariant along their periodic axes (x and y; on
the composite grid by whole base cells), so every translate of the block is
another sample of the same covariance.  A probe block is described by
"channels": 2-D fields over the periodic plane that translate together (a
z row of a component; on the composite grid each fine layer splits into its
four x-y parity sub-lattices so that every channel lives on the base cells).
Per sample the cross-correlations of all channel pairs over every shift come
from FFTs of the channels on the device,

    R_ab(d) = 1/(NY NX) * sum_p xi_a(p) xi_b(p + d),

and a probe site (channel a, position p) pairs with (b, q) through
R_ab(q - p).  The mean is the known value 0 (no subtraction).  Samples are
split into batches; the spread of the batch estimates gives standard errors
(batch means), which also cover the correlation between consecutive samples.

Every cycle of the chain runs in the library's kernels; the host and torch
only read the state back and form these averages (analysis, not the method).
"""

import numpy as np
import torch

from . import selm as S


class TranslateCovariance:
    """Batch-means estimate of the covariance of probe sites over all translates.

    channels: number of 2-D channels per sample, shape (NY, NX) each.
    sites: list of (channel, y, x) probe sites (positions on the channel grid).
    """

    def __init__(self, nchannels, shape, sites, device="cuda"):
        self.nch = nchannels
        self.NY, self.NX = shape
        self.sites = list(sites)
        self.device = device
        self.batches = []          # one block estimate per finished batch
        self._reset()

    def _reset(self):
        self.acc = torch.zeros((self.nch, self.nch, self.NY, self.NX), dtype=torch.complex128,
                               device=self.device)
        self.count = 0

    def add(self, channels):
        """channels: float64 tensor (nch, NY, NX) of one sample."""
        F = torch.fft.fft2(channels.to(torch.float64))
        # sum_p a(p) b(p + d)  <->  conj(F_a) F_b
        self.acc += torch.conj(F)[:, None] * F[None, :]
        self.count += 1

    def end_batch(self):
        if self.count == 0:
            return
        R = torch.fft.ifft2(self.acc).real / (self.NY * self.NX * self.count)
        R = R.cpu().numpy()
        ns = len(self.sites)
        C = np.empty((ns, ns))
        for i, (a, yi, xi) in enumerate(self.sites):
            for j, (b, yj, xj) in enumerate(self.sites):
                C[i, j] = R[a, b, (yj - yi) % self.NY, (xj - xi) % self.NX]
        self.batches.append((C, self.count))
        self._reset()

    def result(self):
        """(mean block, standard error of each entry, number of samples)."""
        Cs = np.array([c for c, _ in self.batches])
        n = sum(k for _, k in self.batches)
        mean = Cs.mean(axis=0)
        se = Cs.std(axis=0, ddof=1) / np.sqrt(len(Cs)) if len(Cs) > 1 else np.full_like(mean, np.nan)
        return mean, se, n


def compare(est, se, exact):
    """Accuracy figures of estimated blocks against the exact ones.

    est, se, exact: one block each, or lists of blocks (e.g. one per
    component) taken together.  rel_frobenius = ||est - exact||_F /
    ||exact||_F; se = the standard error of that figure's noise floor,
    sqrt(sum se_ij^2) / ||exact||_F; max_rel_diag = the largest relative error
    of a diagonal entry; n_eff = the effective number of independent samples
    seen by a diagonal entry, 2 C_ii^2 / se_ii^2 (the variance of a Gaussian
    second moment), averaged over the diagonals."""
    if not isinstance(est, (list, tuple)):
        est, se, exact = [est], [se], [exact]
    nrm = np.sqrt(sum(float(np.sum(e ** 2)) for e in exact))
    err = np.sqrt(sum(float(np.sum((a - e) ** 2)) for a, e in zip(est, exact)))
    se_f = np.sqrt(sum(float(np.sum(s ** 2)) for s in se))
    d = np.concatenate([np.diag(e) for e in exact])
    de = np.concatenate([np.diag(a) for a in est])
    sd = np.concatenate([np.diag(s) for s in se])
    return {
        "rel_frobenius": float(err / nrm),
        "se": float(se_f / nrm),
        "max_rel_diag": float(np.max(np.abs(de - d) / np.abs(d))),
        "n_eff": float(np.mean(2.0 * d ** 2 / np.maximum(sd ** 2, 1e-300))),
    }


# ---- the uniform channel: a block of z rows of each velocity component ------

def uniform_block(h, rows, nsamples, nbatches=10, cycles_per_sample=1, burn_in=10, comps=None):
    """Covariance of the velocity chain xi of handle h on the 4 x 4 x len(rows)
    block x, y in {0..3} (every translate), z in `rows`, per component.

    Returns {comp: (mean block, se, samples)}; sites ordered row, y, x."""
    ncomp = S.selm_mg_ncomp(h, S.SELM_SYS_VELOCITY)
    comps = list(range(ncomp)) if comps is None else comps
    lay = []
    total = 0
    for c in range(ncomp):
        (nx, ny, nz), off, size = S.selm_mg_layout(h, S.SELM_SYS_VELOCITY, 0, c)
        lay.append(((nz, ny, nx), off))
        total = size
    xi = torch.zeros(total, dtype=torch.float64, device="cuda")
    dim = 3 if lay[0][0][1] > 1 else 2
    X = torch.zeros((0, dim), dtype=torch.float64, device="cuda")
    g = torch.zeros((0, dim), dtype=torch.float64, device="cuda")
    S.selm_mg_sample(h, X, burn_in, g, xi)
    ests = {}
    for c in comps:
        (nz, ny, nx), _ = lay[c]
        sites = [(r, y, x) for r in range(len(rows)) for y in range(min(4, ny)) for x in range(4)]
        ests[c] = TranslateCovariance(len(rows), (ny, nx), sites)
    per = max(1, nsamples // nbatches)
    for k in range(per * nbatches):
        S.selm_mg_sample(h, X, cycles_per_sample, g, xi)
        for c in comps:
            (nz, ny, nx), off = lay[c]
            f = xi[off:off + nz * ny * nx].view(nz, ny, nx)
            ests[c].add(f[list(rows)])
        if (k + 1) % per == 0:
            for c in comps:
                ests[c].end_batch()
    return {c: ests[c].result() for c in comps}


# ---- the composite grid: the probe block across the coarse-fine interface ----

def composite_probe_sites(n, K):
    """Channels and sites of the composite probe block (one component).

    The block: x, y indices 126..129 (scaled by n/256) in each level's own
    indexing; in z the fine layers m = 2K-2, 2K-1 just below the interface and
    the uncovered base rows K, K+1 just above it; order layer, y, x.
    Channels 0..7: fine layer (2K-2, 2K-1) x parity (py, px) on the base-cell
    grid; channels 8, 9: base rows K, K+1."""
    x0 = 126 * n // 256
    sites = []
    for layer in range(2):
        for y in range(x0, x0 + 4):
            for x in range(x0, x0 + 4):
                sites.append((layer * 4 + (y & 1) * 2 + (x & 1), y >> 1, x >> 1))
    for row in range(2):
        for y in range(x0, x0 + 4):
            for x in range(x0, x0 + 4):
                sites.append((8 + row, y, x))
    return sites


def composite_block(c, n, K, ncomp, nsamples, nbatches=10, cycles_per_sample=2, burn_in=10):
    """Covariance of the composite chain (selm_comp_sample) of a handle with
    `ncomp` components on the probe block, pooled over the components
    (independent chains of the same operator; each component's field counts
    as one sample).  Returns (mean block, se, samples)."""
    sites = composite_probe_sites(n, K)
    est = TranslateCovariance(10, (n, n), sites)
    xi = torch.zeros(S.selm_comp_size(c), dtype=torch.float64, device="cuda")
    S.selm_comp_sample(c, burn_in, xi)
    per = max(1, nsamples // nbatches)
    for k in range(per * nbatches):
        S.selm_comp_sample(c, cycles_per_sample, xi)
        for comp in range(ncomp):
            (fx, fy, fz), foff, _ = S.selm_comp_layout(c, 0, comp)
            (bx, by, bz), boff, _ = S.selm_comp_layout(c, 1, comp)
            fine = xi[foff:foff + fz * fy * fx].view(fz, fy, fx)
            base = xi[boff:boff + bz * by * bx].view(bz, by, bx)
            ch = []
            for m in (2 * K - 2, 2 * K - 1):
                lay = fine[m]
                for py in range(2):
                    for px in range(2):
                        ch.append(lay[py::2, px::2])
            ch.append(base[K])
            ch.append(base[K + 1])
            est.add(torch.stack(ch))
        if (k + 1) % per == 0:
            est.end_batch()
    return est.result()
