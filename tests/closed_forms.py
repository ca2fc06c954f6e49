"""Closed forms used to pin the oracle (independent of oracle/ code).

* 1-D eigenvalues of the second-difference matrices of each lattice type.
* An exact spectral solver for the uniform-grid operator: on the unit box the
  operator is a Kronecker sum of 1-D second differences whose eigenvectors are
  Fourier modes (periodic axes), DST-I (wall-normal vertex lattice), DST-II
  (cell lattice, Dirichlet walls) or DCT-II (cell lattice, Neumann walls).
* Linear interpolation built from node *positions* (hat functions), to check
  the index-based prolongation of the oracle.
"""

import numpy as np
import scipy.fft as sfft


def eigenvalues_1d(kind, n):
    if kind == "P":
        m = np.arange(n)
        return 2.0 - 2.0 * np.cos(2.0 * np.pi * m / n)
    if kind == "V":
        m = np.arange(1, n)
        return 2.0 - 2.0 * np.cos(np.pi * m / n)
    if kind == "C":
        m = np.arange(1, n + 1)
        return 2.0 - 2.0 * np.cos(np.pi * m / n)
    if kind == "N":
        m = np.arange(n)
        return 2.0 - 2.0 * np.cos(np.pi * m / n)
    if kind == "O":
        return np.zeros(1)
    raise ValueError(kind)


def _fwd(x, kind, axis):
    if kind == "P":
        return sfft.fft(x, axis=axis, norm="ortho")
    if kind == "V":
        return sfft.dst(x, type=1, axis=axis, norm="ortho")
    if kind == "C":
        return sfft.dst(x, type=2, axis=axis, norm="ortho")
    if kind == "N":
        return sfft.dct(x, type=2, axis=axis, norm="ortho")
    return x


def _inv(x, kind, axis):
    if kind == "P":
        return sfft.ifft(x, axis=axis, norm="ortho")
    if kind == "V":
        return sfft.idst(x, type=1, axis=axis, norm="ortho")
    if kind == "C":
        return sfft.idst(x, type=2, axis=axis, norm="ortho")
    if kind == "N":
        return sfft.idct(x, type=2, axis=axis, norm="ortho")
    return x


def spectral_solve(kinds, n, scale, b):
    """x = A^-1 b for A = scale * (Kx (+) Ky (+) Kz) on arrays of shape (nz, ny, nx).

    For a singular (all-'P'/'N') operator the zero mode is dropped (minimum
    norm solution).
    """
    lam = [eigenvalues_1d(k, n if k != "O" else 1) for k in kinds]
    t = b.astype(np.complex128) if "P" in kinds else b.astype(np.float64)
    for a in range(3):
        t = _fwd(t, kinds[a], 2 - a)
    L = (lam[2][:, None, None] + lam[1][None, :, None] + lam[0][None, None, :]) * scale
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(L > 1e-13, t / np.where(L > 1e-13, L, 1.0), 0.0)
    for a in range(3):
        t = _inv(t, kinds[a], 2 - a)
    return np.real(t)


def hat_prolongation(kind, nc):
    """Linear interpolation matrix (fine x coarse) from node positions.

    Coarse and fine unknowns sit at the positions of their lattice type; the
    interpolant is the piecewise-linear function through the coarse values
    and, at a wall, through 0 (Dirichlet) or with zero slope (Neumann);
    periodic axes wrap.  The fine lattice has 2 nc cells on the unit interval.
    """
    nf = 2 * nc
    H, h = 1.0 / nc, 1.0 / nf
    if kind == "P":
        xc = np.arange(nc) * H
        xf = np.arange(nf) * h
        P = np.zeros((nf, nc))
        for image in (-1.0, 0.0, 1.0):          # hats of the periodic images
            d = np.abs(xf[:, None] - xc[None, :] - image)
            P += np.maximum(0.0, 1.0 - d / H)
        return P
    if kind == "V":
        xc = np.arange(1, nc) * H
        xf = np.arange(1, nf) * h
        return np.maximum(0.0, 1.0 - np.abs(xf[:, None] - xc[None, :]) / H)
    xc = (np.arange(nc) + 0.5) * H
    xf = (np.arange(nf) + 0.5) * h
    P = np.zeros((nf, nc))
    for f, x in enumerate(xf):
        if x < xc[0]:
            if kind == "C":       # between the wall value 0 at x = 0 and c_0
                P[f, 0] = x / xc[0]
            else:                 # Neumann: constant continuation
                P[f, 0] = 1.0
        elif x > xc[-1]:
            if kind == "C":
                P[f, nc - 1] = (1.0 - x) / (1.0 - xc[-1])
            else:
                P[f, nc - 1] = 1.0
        else:
            J = int(np.searchsorted(xc, x) - 1)
            J = min(max(J, 0), nc - 2)
            t = (x - xc[J]) / H
            P[f, J] += 1.0 - t
            P[f, J + 1] += t
    return P


def stencil_apply_3d(kinds, scale, v):
    """Top-level operator from the explicit 7-point formula with ghost rules.

    (Av)_i = scale * sum over axes of (2 v_i - v_left - v_right), where a
    missing neighbour beyond a wall is 0 ('V'), -v_i ('C') or +v_i ('N'),
    and periodic axes wrap.  Arrays have shape (nz, ny, nx).
    """
    out = np.zeros_like(v)
    for a, kind in enumerate(kinds):
        if kind == "O":
            continue
        ax = 2 - a
        if kind == "P":
            left = np.roll(v, 1, axis=ax)
            right = np.roll(v, -1, axis=ax)
        else:
            pad_val = {"V": 0.0, "C": -1.0, "N": 1.0}[kind]
            vm = np.moveaxis(v, ax, 0)
            left = np.empty_like(vm)
            right = np.empty_like(vm)
            left[1:] = vm[:-1]
            right[:-1] = vm[1:]
            left[0] = pad_val * vm[0]
            right[-1] = pad_val * vm[-1]
            left = np.moveaxis(left, 0, ax)
            right = np.moveaxis(right, 0, ax)
        out += 2.0 * v - left - right
    return scale * out
