"""Ewald sum of point ion charges in a neutralising background (oracle; test infrastructure).

The paper's DFT step reports the total energy and forces of each structure
(Sec. II A, Sec. II D); the ion-ion term of a plane-wave total energy is the
Ewald sum (P. P. Ewald, Ann. Phys. 64, 253 (1921)):
    E = 1/2 sum'_{I,J,L} Z_I Z_J erfc(eta |R_IJ + L|)/|R_IJ + L|
      + (2 pi/Omega) sum_{G != 0} |S(G)|^2 exp(-G^2/(4 eta^2))/G^2
      - (eta/sqrt(pi)) sum_I Z_I^2 - pi (sum_I Z_I)^2 / (2 Omega eta^2),
    S(G) = sum_I Z_I exp(iG.R_I).  The result does not depend on eta.
"""
import math

import numpy as np
from scipy.special import erfc

from .basis import reciprocal, volume


def ewald(cell, z, pos, eta=None, tol=1e-16):
    """Return (E, F) with F_I = -dE/dR_I, shape (n,3).  Plain loops over images."""
    cell = np.asarray(cell, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    pos = np.asarray(pos, dtype=np.float64)
    n = len(z)
    omega = volume(cell)
    if eta is None:
        eta = math.sqrt(math.pi) / omega ** (1.0 / 3.0)
    # real-space: erfc(eta r) < tol beyond r_max; reciprocal: exp(-G^2/4eta^2) < tol beyond g_max
    x = 1.0
    while erfc(x) > tol:
        x += 0.05
    r_max = x / eta
    g_max = 2.0 * eta * math.sqrt(-math.log(tol))
    B = reciprocal(cell)
    # image ranges from the plane spacings
    nr = [int(math.ceil(r_max * np.linalg.norm(B[i]) / (2 * math.pi))) + 1 for i in range(3)]
    ng = [int(math.ceil(g_max * np.linalg.norm(cell[i]) / (2 * math.pi))) + 1 for i in range(3)]

    L = np.stack(np.meshgrid(*[np.arange(-k, k + 1) for k in nr], indexing="ij"), -1).reshape(-1, 3) @ cell
    e_real = 0.0
    f = np.zeros((n, 3))
    for i in range(n):
        for j in range(n):
            d = pos[i] - pos[j] + L                       # R_I - R_J + L
            r = np.linalg.norm(d, axis=1)
            ok = (r > 1e-12) & (r < r_max)
            r, d = r[ok], d[ok]
            e_real += 0.5 * z[i] * z[j] * np.sum(erfc(eta * r) / r)
            # -d/dR_I of erfc(eta r)/r, both (i,j) and (j,i) orderings counted via the loop
            fac = erfc(eta * r) / r ** 2 + 2.0 * eta / math.sqrt(math.pi) * np.exp(-(eta * r) ** 2) / r
            f[i] += z[i] * z[j] * np.sum((fac / r)[:, None] * d, axis=0)

    m = np.stack(np.meshgrid(*[np.arange(-k, k + 1) for k in ng], indexing="ij"), -1).reshape(-1, 3)
    G = m @ B
    g2 = np.einsum("ij,ij->i", G, G)
    ok = (g2 > 1e-12) & (g2 < g_max ** 2)
    G, g2 = G[ok], g2[ok]
    phase = np.exp(1j * (pos @ G.T))                      # (n, nG) exp(iG.R_I)
    S = z @ phase
    w = np.exp(-g2 / (4.0 * eta * eta)) / g2
    e_recip = 2.0 * math.pi / omega * float(np.sum(np.abs(S) ** 2 * w))
    # F_I = (4 pi Z_I / Omega) sum_G w(G) G Im[exp(iG.R_I) S(G)^*]
    im = np.imag(phase * np.conj(S)[None, :])             # (n, nG)
    f += 4.0 * math.pi / omega * z[:, None] * ((im * w[None, :]) @ G)

    e_self = -eta / math.sqrt(math.pi) * float(np.sum(z * z))
    e_bg = -math.pi * float(np.sum(z)) ** 2 / (2.0 * omega * eta * eta)
    return e_real + e_recip + e_self + e_bg, f
