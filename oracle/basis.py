"""Plane-wave basis at the Gamma point (oracle; test infrastructure only).

The paper's DFT level is a plane-wave pseudopotential code (Sec. II D) whose
inputs are the supercell, the atoms and the plane-wave cutoff.  The basis is
every reciprocal-lattice vector G = m1 b1 + m2 b2 + m3 b3 with |G|^2/2 <= Ecut,
kept as the FULL sphere with complex coefficients (no Gamma half-sphere trick).
"""
import math

import numpy as np


def reciprocal(cell):
    """Rows b_j with a_i . b_j = 2 pi delta_ij."""
    cell = np.asarray(cell, dtype=np.float64)
    return 2.0 * math.pi * np.linalg.inv(cell).T


def volume(cell):
    return abs(float(np.linalg.det(np.asarray(cell, dtype=np.float64))))


def sphere(cell, ecut):
    """Miller indices m (n,3), G vectors (n,3) and |G|^2 of the Ecut sphere.

    |m_i| = |a_i . G| / 2 pi <= |a_i| sqrt(2 Ecut) / 2 pi, so enumerating that
    box and filtering by |G|^2/2 <= Ecut is exhaustive.  Order: |G|^2, then m.
    """
    cell = np.asarray(cell, dtype=np.float64)
    B = reciprocal(cell)
    mx = np.floor(np.linalg.norm(cell, axis=1) * math.sqrt(2.0 * ecut) / (2.0 * math.pi)).astype(int) + 1
    r = [np.arange(-k, k + 1) for k in mx]
    m = np.stack(np.meshgrid(*r, indexing="ij"), axis=-1).reshape(-1, 3)
    G = m @ B
    g2 = np.einsum("ij,ij->i", G, G)
    keep = 0.5 * g2 <= ecut
    m, G, g2 = m[keep], G[keep], g2[keep]
    order = np.lexsort((m[:, 2], m[:, 1], m[:, 0], np.round(g2, 10)))
    return m[order], G[order], g2[order]


def box_miller(grid):
    """Miller index of every FFT-box point, wrapped to [-N/2, N/2), shape grid + (3,)."""
    axes = [np.fft.fftfreq(n, d=1.0 / n).round().astype(int) for n in grid]
    return np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1)


def box_G(cell, grid):
    """G vectors of the whole FFT box (grid + (3,)) and a mask that is False on the
    Nyquist planes m_i = -N_i/2 (even N_i), where a real function has no partner
    +N_i/2; fields defined by a formula in G are zeroed there so that they stay real."""
    m = box_miller(grid)
    G = m @ reciprocal(cell)
    sym = np.ones(tuple(grid), dtype=bool)
    for ax, n in enumerate(grid):
        if n % 2 == 0:
            sym &= m[..., ax] != -(n // 2)
    return m, G, sym


def grid_index(m, grid):
    """Flat-free tuple index of Miller indices m (n,3) into an array of shape grid."""
    return tuple((m[:, i] % grid[i]) for i in range(3))
