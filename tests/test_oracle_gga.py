"""Pins of the oracle's PBE exchange-correlation (oracle/gga.py) against the published forms.

Perdew, Burke & Ernzerhof, PRL 77, 3865 (1996) (exchange Eq. 14; correlation Eqs. 3, 7, 8 at
zeta = 0) on Perdew & Wang's uniform-gas correlation, PRB 45, 13244 (1992) (Eq. 10, Table I).
"""
import math

import numpy as np
import pytest

import workloads
from oracle import dft, gga, lda

# PW92 eps_c(r_s), zeta = 0, evaluated by hand at 30 digits from the published constants
# (A = 0.031091, alpha1 = 0.21370, beta1..4 = 7.5957, 3.5876, 1.6382, 0.49294):
#   den = 2 A (beta1 r_s^1/2 + beta2 r_s + beta3 r_s^3/2 + beta4 r_s^2),
#   eps_c = -2 A (1 + alpha1 r_s) ln(1 + 1/den)
PW92_TABLE = [(0.5, 0.489198052704, -0.076619029223376), (1.0, 0.82791850808, -0.059773864184404),
              (2.0, 1.52485382132, -0.044759590030786), (5.0, 4.07675354655, -0.028216261068974),
              (10.0, 10.0109379276, -0.018572297743848)]
# F_x(s^2) = 1 + kappa - kappa / (1 + mu s^2 / kappa), kappa = 0.804, mu = beta pi^2 / 3 =
# 0.2195149727645171 (beta = 0.06672455060314922)
FX_TABLE = [(0.25, 1.0513722220691), (1.0, 1.1724352284031), (4.0, 1.4196997717879)]
# H(r_s = 2, t^2): gamma = (1 - ln 2)/pi^2 = 0.0310906908696549, A = (beta/gamma) /
# (exp(-eps_c/gamma) - 1) = 0.6666640533331 at eps_c(2) above
H_TABLE = [(0.5, 0.021402710277943), (2.0, 0.038376839619631)]


@pytest.mark.parametrize("rs,den,ec_ref", PW92_TABLE)
def test_pw92_at_tabulated_rs(rs, den, ec_ref):
    assert abs(gga.pw92(rs) - ec_ref) < 1e-13
    # the same uniform gas as Perdew-Zunger's fit to the Ceperley-Alder data: the two fits
    # agree to < 6e-4 Ha (a wrong coefficient in either moves it by more)
    ec_pz, _ = lda.correlation(np.array([rs]))
    assert abs(gga.pw92(rs) - ec_pz[0]) < 6e-4


@pytest.mark.parametrize("s2,fx_ref", FX_TABLE)
def test_exchange_enhancement(s2, fx_ref):
    assert abs(gga.fx(s2) - fx_ref) < 1e-13
    assert gga.fx(0.0) == 1.0
    # gradient expansion for small s: F_x = 1 + mu s^2 + O(s^4); Lieb-Oxford limit 1 + kappa
    assert abs((gga.fx(1e-6) - 1.0) / 1e-6 - gga.MU) < 1e-6
    assert abs(gga.fx(1e12) - 1.804) < 1e-9


@pytest.mark.parametrize("t2,h_ref", H_TABLE)
def test_correlation_gradient_term(t2, h_ref):
    ec = gga.pw92(2.0)
    assert abs(gga.h_pbe(ec, t2) - h_ref) < 1e-13
    # small t: H = beta t^2 (the gradient expansion); large t: H -> -eps_c (correlation
    # vanishes for rapidly varying densities)
    assert abs(gga.h_pbe(ec, 1e-8) / (gga.BETA * 1e-8) - 1.0) < 1e-6
    assert abs(gga.h_pbe(ec, 1e10) + ec) < 1e-8


def test_uniform_limit_is_slater_plus_pw92():
    for rs in (0.5, 1.0, 3.0, 8.0):
        rho = 3.0 / (4.0 * math.pi * rs ** 3)
        e, dr, ds = gga.pbe_point(np.array([rho]), np.array([0.0]))
        assert abs(e[0] / rho - (-0.4581652932831429 / rs + gga.pw92(rs))) < 1e-13
        # de/drho at sigma = 0: the LDA potential of Slater + PW92 (central difference)
        h = rho * 1e-5
        f = lambda r: r * (-0.75 * (3 * r / math.pi) ** (1 / 3) + gga.pw92((3 / (4 * math.pi * r)) ** (1 / 3)))
        assert abs(dr[0] - (f(rho + h) - f(rho - h)) / (2 * h)) < 1e-8


def test_complex_step_derivatives_match_differences():
    rho = np.array([0.003, 0.05, 0.4, 2.0])
    sigma = np.array([1e-6, 0.01, 0.3, 5.0])
    e, dr, ds = gga.pbe_point(rho, sigma)
    for k in range(len(rho)):
        hr, hs = 1e-6 * rho[k], 1e-6 * sigma[k]
        fr = (gga.energy_density(rho[k] + hr, sigma[k]) - gga.energy_density(rho[k] - hr, sigma[k])) / (2 * hr)
        fs = (gga.energy_density(rho[k], sigma[k] + hs) - gga.energy_density(rho[k], sigma[k] - hs)) / (2 * hs)
        assert abs(dr[k] - fr) < 1e-7 * max(1.0, abs(fr))
        assert abs(ds[k] - fs) < 1e-6 * max(1e-3, abs(fs))
    # below the density cut every output is zero
    e0, d0, s0 = gga.pbe_point(np.array([1e-12]), np.array([1.0]))
    assert e0[0] == 0.0 and d0[0] == 0.0 and s0[0] == 0.0


def _smooth_density(model, seed=3):
    rng = np.random.default_rng(seed)
    rho = np.zeros(model.grid)
    pts = rng.uniform(size=(4, 3)) @ model.cell
    r = np.stack(np.meshgrid(*[np.arange(n) / n for n in model.grid], indexing="ij"), -1) @ model.cell
    for p in pts:
        d = r - p
        f = np.linalg.solve(model.cell.T, d.reshape(-1, 3).T).T
        d = (f - np.round(f)) @ model.cell
        rho += 0.08 * np.exp(-np.sum(d * d, axis=1) / 3.0).reshape(model.grid)
    return rho + 1e-3


def test_potential_is_the_functional_derivative():
    """E_xc[rho + h delta] - E_xc[rho - h delta] = 2 h (Omega/N) sum v_xc delta + O(h^3): pins
    the divergence term (its sign and the factor 2 of d sigma / d grad rho) and the gradient's
    G-space convention on a cubic and a skewed cell."""
    for st in (workloads.tiny(nat=2, ecut=3.0, seed=7), workloads.honeycomb24()):
        model = dft.Model(dataclass_with_xc(st))
        rho = _smooth_density(model)
        rng = np.random.default_rng(5)
        delta = model.to_real(model.to_recip(rng.normal(size=model.grid)) * (model.bg2 < 2.0) * model.sym).real
        e0, v = gga.pbe(model, rho)
        h = 1e-5
        ep, _ = gga.pbe(model, rho + h * delta)
        em, _ = gga.pbe(model, rho - h * delta)
        lhs = (ep - em) / (2 * h)
        rhs = model.omega / model.N * float(np.sum(v * delta))
        scale = model.omega / model.N * float(np.sum(np.abs(v * delta)))
        assert abs(lhs - rhs) < 1e-7 * scale, (lhs, rhs, scale)


def dataclass_with_xc(st, xc="pbe"):
    import dataclasses
    return dataclasses.replace(st, xc=xc)


def test_exchange_scales_linearly_under_uniform_scaling():
    """rho_l(r) = l^3 rho(l r): PBE exchange (s is scale invariant) gives E_x[rho_l] = l E_x[rho]
    exactly, here on the FFT box of the cell shrunk by l with the same grid values times l^3."""
    st = dataclass_with_xc(workloads.tiny(nat=2, ecut=3.0, seed=7))
    lam = 1.37

    def e_x(model, rho):
        g = gga.gradient(model, rho)
        sigma = np.einsum("a...,a...->...", g, g)
        kf = (3 * math.pi ** 2 * rho) ** (1 / 3)
        s2 = sigma / (4 * kf * kf * rho * rho)
        return model.omega / model.N * float(np.sum(rho * -0.75 * (3 * rho / math.pi) ** (1 / 3) * gga.fx(s2)))

    m1 = dft.Model(st)
    rho = _smooth_density(m1)
    import dataclasses
    m2 = dft.Model(dataclasses.replace(st, cell=st.cell / lam))
    assert abs(e_x(m2, lam ** 3 * rho) - lam * e_x(m1, rho)) < 1e-12 * abs(e_x(m1, rho))


def test_pbe_scf_forces_are_energy_derivatives():
    """The oracle's PBE SCF: Hellmann-Feynman forces against central differences of the free
    energy (h = 1e-3 bohr), which holds only if v_xc is the derivative of E_xc."""
    import oracle
    st = dataclass_with_xc(workloads.tiny(nat=2, ecut=3.0, seed=7, kT=0.01))
    r = oracle.scf(st, tol_e=1e-12, tol_rho=1e-10)
    h = 1e-3
    for (I, a) in [(0, 0), (1, 2)]:
        p = st.pos.copy()
        p[I, a] += h
        ep = oracle.scf(st.with_positions(p), tol_e=1e-12, tol_rho=1e-10).free_energy
        p[I, a] -= 2 * h
        em = oracle.scf(st.with_positions(p), tol_e=1e-12, tol_rho=1e-10).free_energy
        assert abs(-(ep - em) / (2 * h) - r.forces[I, a]) < 2e-5, (I, a)
    # PBE differs from LDA (the variant is not a no-op)
    r_lda = oracle.scf(dataclass_with_xc(st, "lda"), tol_e=1e-12, tol_rho=1e-10)
    assert abs(r.free_energy - r_lda.free_energy) > 1e-3
