"""Synthetic analytic pseudopotential in reciprocal space (oracle; test infrastructure).

The paper uses real norm-conserving / ultrasoft PBE potentials (Sec. II D), which
are not available; the stand-in per species s is
    v_s(r) = -Z erf(r/rc)/r + A exp(-r^2/sigma^2)      (local)
    D |beta><beta|, beta(r) = N exp(-r^2/(2 rp^2)), <beta|beta> = 1   (KB s-projector)
    + D_p sum_m |beta_m><beta_m|, beta_m(r) = N_p x_m exp(-r^2/(2 rp_p^2))   (optional p channel,
      species keys d_p, rp_p; absent or d_p = 0: none).
Fourier convention: f(G) = (1/Omega) int f(r) exp(-iG.r) d^3r for the local
part; <G|beta> with |G> = Omega^{-1/2} exp(iG.r) for the projector.
"""
import math

import numpy as np

PI32 = math.pi ** 1.5


def vloc_g(sp, g2, omega):
    """v_s(G) for |G|^2 = g2 (any shape).  At G = 0 the -4 pi Z / G^2 divergence is
    dropped and the finite 'alpha' term (1/Omega) int (v_s(r) + Z/r) d^3r =
    (pi Z rc^2 + A pi^{3/2} sigma^3)/Omega is used; it pairs with the neutralising
    background of the Ewald sum and the G = 0 Hartree term set to zero."""
    g2 = np.asarray(g2, dtype=np.float64)
    Z, rc, A, sg = sp["z_val"], sp["rc"], sp["a_sr"], sp["sigma_sr"]
    out = np.empty_like(g2)
    nz = g2 > 1e-14
    out[nz] = (-4.0 * math.pi * Z * np.exp(-g2[nz] * rc * rc / 4.0) / g2[nz]
               + A * PI32 * sg ** 3 * np.exp(-g2[nz] * sg * sg / 4.0)) / omega
    out[~nz] = (math.pi * Z * rc * rc + A * PI32 * sg ** 3) / omega
    return out


def vloc_alpha(sp, omega):
    return (math.pi * sp["z_val"] * sp["rc"] ** 2 + sp["a_sr"] * PI32 * sp["sigma_sr"] ** 3) / omega


def beta_g(sp, g2, omega):
    """<G|beta> for a projector centred at the origin: Omega^{-1/2} N (2pi)^{3/2} rp^3 exp(-G^2 rp^2/2)."""
    rp = sp["rp"]
    norm = 1.0 / math.sqrt(PI32 * rp ** 3)
    return norm * (2.0 * math.pi) ** 1.5 * rp ** 3 * np.exp(-np.asarray(g2) * rp * rp / 2.0) / math.sqrt(omega)


def atomic_density_g(sp, g2, omega):
    """Initial-guess neutral Gaussian charge of Z electrons per atom: (Z/Omega) exp(-G^2 rc^2/4)."""
    return sp["z_val"] * np.exp(-np.asarray(g2) * sp["rc"] ** 2 / 4.0) / omega


def beta_p_g(sp, G, omega):
    """<G|beta_m>, m = x, y, z, for the p-channel projector at the origin, shape (3,) + G.shape[:-1].

    beta_m(r) = N_p x_m exp(-r^2/(2 s^2)) with s = rp_p and N_p = (pi^{3/2} s^5 / 2)^{-1/2}
    (so <beta_m|beta_m> = 1: the integral of x^2 exp(-r^2/s^2) is pi^{3/2} s^5 / 2).  Its
    transform is i d/dG_m of the Gaussian's, (2 pi)^{3/2} s^3 exp(-G^2 s^2/2):
    <G|beta_m> = Omega^{-1/2} N_p (-i G_m s^2) (2 pi)^{3/2} s^3 exp(-G^2 s^2 / 2)."""
    s_ = sp["rp_p"]
    norm = 1.0 / math.sqrt(PI32 * s_ ** 5 / 2.0)
    G = np.asarray(G, dtype=np.float64)
    g2 = np.einsum("...i,...i->...", G, G)
    radial = norm * (2.0 * math.pi) ** 1.5 * s_ ** 3 * s_ * s_ * np.exp(-g2 * s_ * s_ / 2.0) / math.sqrt(omega)
    return np.stack([-1j * G[..., m] * radial for m in range(3)])
