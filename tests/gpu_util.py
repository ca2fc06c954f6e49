"""Helpers for the GPU parity tests: move oracle fields (lists of (nz, ny, nx)
arrays) to and from the library's flat device layout."""

import numpy as np
import torch

from paper_1003_2680_gb300 import selm as S


def comps(h, system=S.SELM_SYS_VELOCITY, level=0):
    n = S.selm_mg_ncomp(h, system)
    out = []
    size = 0
    for c in range(n):
        (nx, ny, nz), off, size = S.selm_mg_layout(h, system, level, c)
        out.append(((nz, ny, nx), off))
    return out, size


def to_dev(h, fields, dtype, system=S.SELM_SYS_VELOCITY, level=0):
    lay, size = comps(h, system, level)
    flat = np.zeros(size)
    for (shape, off), f in zip(lay, fields):
        assert tuple(f.shape) == tuple(shape), (f.shape, shape)
        flat[off:off + f.size] = f.ravel()
    return torch.tensor(flat, dtype=dtype, device="cuda")


def from_dev(h, t, system=S.SELM_SYS_VELOCITY, level=0):
    lay, size = comps(h, system, level)
    flat = t.detach().double().cpu().numpy()
    assert flat.size == size
    return [flat[off:off + int(np.prod(shape))].reshape(shape).copy() for shape, off in lay]


def rel(a, b):
    a = np.concatenate([x.ravel() for x in a]) if isinstance(a, list) else np.asarray(a).ravel()
    b = np.concatenate([x.ravel() for x in b]) if isinstance(b, list) else np.asarray(b).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def maxrel(a, b):
    """max |a - b| / max |b|: an element-wise bound that a field-norm
    comparison cannot give (one bad row among millions of good ones)."""
    a = np.concatenate([x.ravel() for x in a]) if isinstance(a, list) else np.asarray(a).ravel()
    b = np.concatenate([x.ravel() for x in b]) if isinstance(b, list) else np.asarray(b).ravel()
    mb = np.abs(b).max() if b.size else 0.0
    return np.abs(a - b).max() / (mb if mb > 0 else 1.0)


def round_like(fields, dtype):
    if dtype == torch.float32:
        return [f.astype(np.float32).astype(np.float64) for f in fields]
    return [f.copy() for f in fields]


def empty(h, dtype, system=S.SELM_SYS_VELOCITY, level=0):
    _, size = comps(h, system, level)
    return torch.zeros(size, dtype=dtype, device="cuda")
