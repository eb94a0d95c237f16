"""Test helpers: convert between the oracle's full complex sphere and the engine's
Gamma real packing (x[0] = c(0), x[1+2k] = sqrt2 Re c(G_k), x[2+2k] = sqrt2 Im c(G_k))."""
import math

import numpy as np


def sphere_lookup(model):
    return {tuple(m): i for i, m in enumerate(model.m.tolist())}


def full_from_packed(model, miller, x):
    """x: (nvec, npw) packed -> (npw_full, nvec) complex full-sphere coefficients."""
    x = np.atleast_2d(x)
    lut = sphere_lookup(model)
    c = np.zeros((model.npw, x.shape[0]), dtype=np.complex128)
    c[lut[(0, 0, 0)], :] = x[:, 0]
    r2 = 1.0 / math.sqrt(2.0)
    for k, m in enumerate(miller[1:].tolist()):
        v = (x[:, 1 + 2 * k] + 1j * x[:, 2 + 2 * k]) * r2
        c[lut[tuple(m)], :] = v
        c[lut[tuple(-np.array(m))], :] = np.conj(v)
    return c


def packed_from_full(model, miller, c):
    """(npw_full, nvec) complex -> (nvec, npw) packed (uses c(G) of the half sphere)."""
    lut = sphere_lookup(model)
    nvec = c.shape[1]
    x = np.zeros((nvec, 1 + 2 * (len(miller) - 1)))
    x[:, 0] = c[lut[(0, 0, 0)], :].real
    s2 = math.sqrt(2.0)
    for k, m in enumerate(miller[1:].tolist()):
        v = c[lut[tuple(m)], :]
        x[:, 1 + 2 * k] = s2 * v.real
        x[:, 2 + 2 * k] = s2 * v.imag
    return x
