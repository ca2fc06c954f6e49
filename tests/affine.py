"""Helpers: treat an oracle step as an affine map of its inputs and noise."""

import numpy as np

from oracle.philox import ExplicitNoise


def flatten(fields):
    return np.concatenate([f.ravel() for f in fields])


def unflatten(vec, shapes):
    out, o = [], 0
    for sh in shapes:
        n = int(np.prod(sh))
        out.append(vec[o:o + n].reshape(sh).copy())
        o += n
    return out


def count_noise(step, shapes):
    """Number of noise variates one call of step(z, b, noise) consumes."""
    probe = ExplicitNoise(None)
    zero = [np.zeros(s) for s in shapes]
    step(unflatten(np.zeros(sum(int(np.prod(s)) for s in shapes)), shapes), zero, probe)
    return probe.count


def extract(step, shapes, shapes_b=None):
    """Return (M, N, B, c) with step(z, b, n) = M z + N b + B n + c.

    step(z_fields, b_fields, noise) must return the new z (list of arrays).
    """
    shapes_b = shapes if shapes_b is None else shapes_b
    nz = sum(int(np.prod(s)) for s in shapes)
    nb = sum(int(np.prod(s)) for s in shapes_b)
    nn = count_noise(step, shapes)

    def run(z, b, n):
        noise = ExplicitNoise(n)
        out = flatten(step(unflatten(z, shapes), unflatten(b, shapes_b), noise))
        assert noise.count == nn
        return out

    c = run(np.zeros(nz), np.zeros(nb), np.zeros(nn))
    M = np.zeros((nz, nz))
    for i in range(nz):
        e = np.zeros(nz)
        e[i] = 1.0
        M[:, i] = run(e, np.zeros(nb), np.zeros(nn)) - c
    N = np.zeros((nz, nb))
    for i in range(nb):
        e = np.zeros(nb)
        e[i] = 1.0
        N[:, i] = run(np.zeros(nz), e, np.zeros(nn)) - c
    B = np.zeros((nz, nn))
    for i in range(nn):
        e = np.zeros(nn)
        e[i] = 1.0
        B[:, i] = run(np.zeros(nz), np.zeros(nb), e) - c
    return M, N, B, c


def block_diag(mats):
    n = sum(m.shape[0] for m in mats)
    out = np.zeros((n, n))
    o = 0
    for m in mats:
        k = m.shape[0]
        out[o:o + k, o:o + k] = m
        o += k
    return out
