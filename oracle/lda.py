"""LDA exchange-correlation, unpolarised (oracle; test infrastructure).

The paper's searches use PBE (Sec. III); the workloads here fix LDA.  Exchange is
Slater's: eps_x = -(3/4)(3 rho/pi)^{1/3}, v_x = 4/3 eps_x.  Correlation is the
Perdew-Zunger 1981 fit to Ceperley-Alder (Phys. Rev. B 23, 5048, Appendix C):
    r_s >= 1: eps_c = gamma / (1 + beta1 sqrt(r_s) + beta2 r_s)
    r_s <  1: eps_c = A ln r_s + B + C r_s ln r_s + D r_s
with v_c = eps_c - (r_s/3) d eps_c / d r_s.  Points with rho <= 1e-30 give 0.
"""
import math

import numpy as np

PZ_GAMMA, PZ_BETA1, PZ_BETA2 = -0.1423, 1.0529, 0.3334
PZ_A, PZ_B, PZ_C, PZ_D = 0.0311, -0.048, 0.0020, -0.0116
RHO_MIN = 1e-30


def rs_of_rho(rho):
    return (3.0 / (4.0 * math.pi * rho)) ** (1.0 / 3.0)


def exchange(rho):
    """(eps_x, v_x) for rho > 0."""
    ex = -0.75 * (3.0 * rho / math.pi) ** (1.0 / 3.0)
    return ex, 4.0 / 3.0 * ex


def correlation(rs):
    """(eps_c, v_c) as functions of r_s (array)."""
    rs = np.asarray(rs, dtype=np.float64)
    ec = np.empty_like(rs)
    vc = np.empty_like(rs)
    hi = rs >= 1.0
    s = np.sqrt(rs[hi])
    den = 1.0 + PZ_BETA1 * s + PZ_BETA2 * rs[hi]
    ec[hi] = PZ_GAMMA / den
    vc[hi] = ec[hi] * (1.0 + 7.0 / 6.0 * PZ_BETA1 * s + 4.0 / 3.0 * PZ_BETA2 * rs[hi]) / den
    lo = ~hi
    r = rs[lo]
    lr = np.log(r)
    ec[lo] = PZ_A * lr + PZ_B + PZ_C * r * lr + PZ_D * r
    vc[lo] = PZ_A * lr + (PZ_B - PZ_A / 3.0) + 2.0 / 3.0 * PZ_C * r * lr + (2.0 * PZ_D - PZ_C) / 3.0 * r
    return ec, vc


def lda(rho):
    """(eps_xc, v_xc) on an array of densities; rho is clipped with max(rho, 0)."""
    rho = np.maximum(np.asarray(rho, dtype=np.float64), 0.0)
    exc = np.zeros_like(rho)
    vxc = np.zeros_like(rho)
    ok = rho > RHO_MIN
    ex, vx = exchange(rho[ok])
    ec, vc = correlation(rs_of_rho(rho[ok]))
    exc[ok] = ex + ec
    vxc[ok] = vx + vc
    return exc, vxc
