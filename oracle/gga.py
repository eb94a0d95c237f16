"""PBE generalized-gradient exchange-correlation, unpolarised (oracle; test infrastructure).

The paper's searches use PBE (Sec. III); the workloads fix LDA, and this is the GGA variant.
Energy per volume e(rho, sigma) = rho eps_xc, sigma = |grad rho|^2:

Exchange (Perdew, Burke & Ernzerhof, PRL 77, 3865 (1996), Eq. 14):
    e_x = rho eps_x^unif(rho) F_x(s),  eps_x^unif = -(3/4) (3 rho / pi)^{1/3},
    F_x = 1 + kappa - kappa / (1 + mu s^2 / kappa),  s^2 = sigma / (4 k_F^2 rho^2),
    k_F = (3 pi^2 rho)^{1/3},  kappa = 0.804,  mu = beta pi^2 / 3.
Correlation (same paper, Eqs. 3, 7, 8; spin-unpolarised, phi = 1):
    e_c = rho (eps_c^unif(r_s) + H),  H = gamma ln(1 + (beta/gamma) t^2 (1 + A t^2) / (1 + A t^2 + A^2 t^4)),
    A = (beta/gamma) / (exp(-eps_c^unif / gamma) - 1),  t^2 = sigma / (4 k_s^2 rho^2),
    k_s = sqrt(4 k_F / pi),  gamma = (1 - ln 2) / pi^2,  beta = 0.06672455060314922.
eps_c^unif is Perdew & Wang's fit (PRB 45, 13244 (1992), Eq. 10 with Table I, zeta = 0):
    G(r_s) = -2 A0 (1 + a1 r_s) ln(1 + 1 / (2 A0 (b1 r_s^{1/2} + b2 r_s + b3 r_s^{3/2} + b4 r_s^2))).

The potential is the functional derivative
    v_xc = de/drho - div(2 de/dsigma grad rho),
with the gradient and the divergence taken in G space on the FFT box (Nyquist planes zero).
The two partial derivatives of e come from the complex-step rule (Squire & Trapp, SIAM Rev.
40, 110 (1998)): df/dx = Im f(x + i h) / h, exact to rounding for a function analytic in x,
which e is (no absolute values: sigma enters squared).  Points with rho <= RHO_CUT give 0
(the reduced gradients of near-empty regions carry no weight).
"""
import math

import numpy as np

KAPPA = 0.804
BETA = 0.06672455060314922
MU = BETA * math.pi ** 2 / 3.0
GAMMA = (1.0 - math.log(2.0)) / math.pi ** 2
PW_A, PW_A1 = 0.031091, 0.21370
PW_B1, PW_B2, PW_B3, PW_B4 = 7.5957, 3.5876, 1.6382, 0.49294
RHO_CUT = 1e-10


def pw92(rs):
    """Perdew-Wang 1992 correlation energy per electron of the uniform gas (zeta = 0)."""
    s = np.sqrt(rs)
    den = 2.0 * PW_A * (PW_B1 * s + PW_B2 * rs + PW_B3 * rs * s + PW_B4 * rs * rs)
    return -2.0 * PW_A * (1.0 + PW_A1 * rs) * np.log(1.0 + 1.0 / den)


def fx(s2):
    """PBE exchange enhancement factor as a function of s^2."""
    return 1.0 + KAPPA - KAPPA / (1.0 + MU * s2 / KAPPA)


def h_pbe(ec, t2):
    """PBE gradient correction to the correlation energy per electron (phi = 1)."""
    a = (BETA / GAMMA) / (np.exp(-ec / GAMMA) - 1.0)
    at2 = a * t2
    return GAMMA * np.log(1.0 + (BETA / GAMMA) * t2 * (1.0 + at2) / (1.0 + at2 + at2 * at2))


def energy_density(rho, sigma):
    """e(rho, sigma) = rho eps_xc for rho > 0 (arrays; complex arguments allowed)."""
    kf = (3.0 * math.pi ** 2 * rho) ** (1.0 / 3.0)
    ex_unif = -0.75 * (3.0 * rho / math.pi) ** (1.0 / 3.0)
    s2 = sigma / (4.0 * kf * kf * rho * rho)
    rs = (3.0 / (4.0 * math.pi * rho)) ** (1.0 / 3.0)
    ec = pw92(rs)
    ks2 = 4.0 * kf / math.pi
    t2 = sigma / (4.0 * ks2 * rho * rho)
    return rho * (ex_unif * fx(s2) + ec + h_pbe(ec, t2))


def pbe_point(rho, sigma):
    """(e, de/drho, de/dsigma) on arrays; 0 where rho <= RHO_CUT."""
    rho = np.asarray(rho, dtype=np.float64)
    sigma = np.maximum(np.asarray(sigma, dtype=np.float64), 0.0)
    e = np.zeros_like(rho)
    dr = np.zeros_like(rho)
    ds = np.zeros_like(rho)
    ok = rho > RHO_CUT
    r, g = rho[ok], sigma[ok]
    e[ok] = energy_density(r, g)
    hr = 1e-20 * r
    dr[ok] = energy_density(r + 1j * hr, g + 0j).imag / hr
    hs = 1e-20 * np.maximum(g, r ** (8.0 / 3.0))
    ds[ok] = energy_density(r + 0j, g + 1j * hs).imag / hs
    return e, dr, ds


def gradient(model, rho_r):
    """grad rho on the FFT box: (3, N1, N2, N3), from i G rho(G) (Nyquist planes zero)."""
    rg = model.to_recip(rho_r) * model.sym
    return np.stack([model.to_real(1j * model.bG[..., a] * rg).real for a in range(3)])


def divergence(model, h):
    """div h for a real vector field h (3, N1, N2, N3) on the FFT box."""
    acc = np.zeros(model.grid, dtype=np.complex128)
    for a in range(3):
        acc += 1j * model.bG[..., a] * model.to_recip(h[a]) * model.sym
    return model.to_real(acc).real


def pbe(model, rho_r):
    """(E_xc, v_xc(r)) of PBE on the FFT box, rho clipped at 0."""
    rho = np.maximum(np.asarray(rho_r, dtype=np.float64), 0.0)
    g = gradient(model, rho_r)
    sigma = np.einsum("a...,a...->...", g, g)
    e, dr, ds = pbe_point(rho, sigma)
    v = dr - divergence(model, 2.0 * ds[None] * g)
    return model.omega / model.N * float(np.sum(e)), v
