"""Plain FP64 plane-wave Kohn-Sham DFT at the Gamma point (oracle; test infrastructure).

What the paper's bottom level computes (Sec. II A, Sec. II D): "the energy and
atomic force of each structure ... calculated self-consistently".  One SCF step
(Sec. II D, paragraph after Algorithm 1) starts from rho_in, solves the Kohn-Sham
equation H psi_i = eps_i psi_i (Algorithm 1's problem), builds rho_out from the
occupied states and mixes rho_out with rho_in.  The paper gives no Hamiltonian,
so the oracle writes out the textbook momentum-space total energy (Ihm, Zunger &
Cohen, J. Phys. C 12, 4409 (1979)):

    E = sum_n f_n <psi_n| -1/2 nabla^2 + V_NL |psi_n>
      + Omega sum_G V_ion(G) rho(G)^*          (alpha term at G = 0)
      + (Omega/2) sum_{G!=0} 4 pi |rho(G)|^2 / G^2
      + (Omega/N) sum_r rho(r) eps_xc(rho(r))   (LDA on the FFT grid; PBE: gga.py)
      + E_Ewald,          F = E - kT S  (Mermin free energy, reported)

Conventions: psi(r) = Omega^{-1/2} sum_G c(G) exp(iG.r), sum |c|^2 = 1, over the
FULL complex Ecut sphere.  A field f on the FFT box: f(G) = (1/N) sum_r f(r)
exp(-iG.r).  The eigenproblem is solved exactly: dense H + LAPACK for small
bases, LOBPCG on the FFT-applied H (residual-checked) otherwise.  This is a
different formulation from the CUDA path (real Gamma half-sphere, all-band CG of
Algorithm 1); both reach the same self-consistent fixed point.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.linalg
import scipy.sparse.linalg
from scipy.special import expit

from . import basis
from .ewald import ewald
from . import gga
from .lda import lda
from .pseudo import atomic_density_g, beta_g, beta_p_g, vloc_g


# ---------------------------------------------------------------------------
# Structure-independent tables
# ---------------------------------------------------------------------------
class Model:
    """Basis, FFT box and per-species reciprocal-space tables for one cell."""

    def __init__(self, st):
        self.st = st
        self.cell = np.asarray(st.cell, dtype=np.float64)
        self.omega = basis.volume(self.cell)
        self.grid = tuple(int(x) for x in st.fft)
        self.N = int(np.prod(self.grid))
        self.m, self.G, self.g2 = basis.sphere(self.cell, st.ecut)
        self.npw = len(self.g2)
        self.idx = basis.grid_index(self.m, self.grid)
        mmax = np.max(np.abs(self.m), axis=0)
        if any(n < 4 * k + 1 for n, k in zip(self.grid, mmax)):
            raise ValueError(f"FFT grid {self.grid} aliases for m_max {mmax}")
        self.bm, self.bG, self.sym = basis.box_G(self.cell, self.grid)
        self.bg2 = np.einsum("...i,...i->...", self.bG, self.bG)
        self.species = list(st.species)
        self.spec = np.asarray(st.species_of_atom, dtype=int)
        self.vloc_box = [vloc_g(sp, self.bg2, self.omega) * self.sym for sp in self.species]
        self.beta_sph = [beta_g(sp, self.g2, self.omega) for sp in self.species]
        # p channel (species with d_p != 0): three projectors per atom after its s projector
        self.betap_sph = [beta_p_g(sp, self.G, self.omega) if sp.get("d_p", 0.0) != 0.0 else None
                          for sp in self.species]
        self.z = np.array([self.species[s]["z_val"] for s in self.spec])
        # per projector (atom-major: s, then p_x, p_y, p_z where present): strength and atom
        d, atom = [], []
        for I, s in enumerate(self.spec):
            d.append(self.species[s]["d_nl"])
            atom.append(I)
            if self.betap_sph[s] is not None:
                d += [self.species[s]["d_p"]] * 3
                atom += [I] * 3
        self.d = np.array(d)
        self.proj_atom = np.array(atom, dtype=int)
        self.nel = float(np.sum(self.z))

    # FFT-box transforms with the f(G) = (1/N) sum_r convention
    def to_recip(self, fr):
        return np.fft.fftn(fr, axes=(-3, -2, -1)) / self.N

    def to_real(self, fg):
        return np.fft.ifftn(fg, axes=(-3, -2, -1)) * self.N

    def wave_real(self, C):
        """psi_n(r) on the grid for coefficient columns C (npw, nb) -> (nb, N1, N2, N3)."""
        nb = C.shape[1]
        g = np.zeros((nb,) + self.grid, dtype=np.complex128)
        g[(slice(None),) + self.idx] = C.T
        return np.fft.ifftn(g, axes=(1, 2, 3)) * (self.N / math.sqrt(self.omega))


# ---------------------------------------------------------------------------
# Structure-dependent terms
# ---------------------------------------------------------------------------
def ionic_potential_g(model, pos):
    """V_ion(G) = sum_I v_s(G) exp(-iG.R_I) on the FFT box (zero on Nyquist planes)."""
    v = np.zeros(model.grid, dtype=np.complex128)
    for I, s in enumerate(model.spec):
        v += model.vloc_box[s] * np.exp(-1j * (model.bG @ pos[I]))
    return v


def projectors(model, pos):
    """beta_k(G) exp(-iG.R_I(k)) on the sphere for every projector k (atom-major: the s
    projector of atom I, then its p_x, p_y, p_z where its species has a p channel), shape
    (nproj, npw)."""
    rows = []
    for I, s in enumerate(model.spec):
        ph = np.exp(-1j * (model.G @ pos[I]))
        rows.append(model.beta_sph[s] * ph)
        if model.betap_sph[s] is not None:
            rows += [model.betap_sph[s][m] * ph for m in range(3)]
    return np.array(rows)


def initial_density(model, pos):
    """Sum of neutral atomic Gaussians, band-limited to |G|^2/2 <= 4 Ecut (real space)."""
    rg = np.zeros(model.grid, dtype=np.complex128)
    lim = (0.5 * model.bg2 <= 4.0 * model.st.ecut) & model.sym
    for I, s in enumerate(model.spec):
        rg += atomic_density_g(model.species[s], model.bg2, model.omega) * np.exp(-1j * (model.bG @ pos[I]))
    return model.to_real(rg * lim).real


# ---------------------------------------------------------------------------
# Hamiltonian
# ---------------------------------------------------------------------------
def apply_h(model, veff_r, beta, C):
    """H C for coefficient columns C (npw, nb): kinetic + local (via FFT) + KB nonlocal."""
    C = np.asarray(C, dtype=np.complex128)
    out = 0.5 * model.g2[:, None] * C
    nb = C.shape[1]
    g = np.zeros((nb,) + model.grid, dtype=np.complex128)
    g[(slice(None),) + model.idx] = C.T
    psi = np.fft.ifftn(g, axes=(1, 2, 3)) * model.N
    back = np.fft.fftn(psi * veff_r[None], axes=(1, 2, 3)) / model.N
    out += back[(slice(None),) + model.idx].T
    P = beta.conj() @ C
    out += beta.T @ (model.d[:, None] * P)
    return out


def dense_h(model, veff_r, beta):
    """The full npw x npw matrix H(G,G') = |G|^2/2 delta + V_eff(G-G') + sum_I D beta_I(G) beta_I(G')^*."""
    vg = model.to_recip(veff_r)
    dm = model.m[:, None, :] - model.m[None, :, :]
    H = vg[dm[..., 0] % model.grid[0], dm[..., 1] % model.grid[1], dm[..., 2] % model.grid[2]]
    H = H + np.diag(0.5 * model.g2)
    H = H + (beta.T * model.d[None, :]) @ beta.conj()
    return H


# ---------------------------------------------------------------------------
# Density, Hartree, exchange-correlation
# ---------------------------------------------------------------------------
def density(model, C, f):
    """rho(r) = sum_n f_n |psi_n(r)|^2."""
    psi = model.wave_real(C)
    return np.einsum("n,nxyz->xyz", f, np.abs(psi) ** 2)


def hartree(model, rho_r):
    """(E_H, V_H(r)): V_H(G) = 4 pi rho(G)/G^2 for G != 0, 0 at G = 0."""
    rg = model.to_recip(rho_r) * model.sym
    nz = model.bg2 > 1e-14
    vg = np.zeros_like(rg)
    vg[nz] = 4.0 * math.pi * rg[nz] / model.bg2[nz]
    e = 0.5 * model.omega * float(np.sum((np.conj(rg) * vg).real))
    return e, model.to_real(vg).real


def xc(model, rho_r):
    """(E_xc, v_xc(r)) = ((Omega/N) sum_r rho eps_xc, d(rho eps)/d rho) with rho clipped at 0
    (LDA), or PBE's energy and functional derivative (gga.pbe) for a structure with xc = "pbe"."""
    if getattr(model.st, "xc", "lda") == "pbe":
        return gga.pbe(model, rho_r)
    exc, vxc = lda(rho_r)
    return model.omega / model.N * float(np.sum(np.maximum(rho_r, 0.0) * exc)), vxc


def local_energy(model, vion_g, rho_r):
    return model.omega * float(np.sum((vion_g * np.conj(model.to_recip(rho_r))).real))


# ---------------------------------------------------------------------------
# Occupations (Fermi-Dirac, Mermin entropy)
# ---------------------------------------------------------------------------
def occupations(eps, nel, kT):
    """(f, mu, S): integer occupations (2 per band) for kT = 0, else Fermi-Dirac with mu by
    bisection so that sum f = N_el; S = -2 sum [x ln x + (1-x) ln(1-x)], x = f/2."""
    eps = np.asarray(eps, dtype=np.float64)
    nb = len(eps)
    if kT <= 0.0:
        nocc = int(round(nel / 2.0))
        if abs(nocc * 2.0 - nel) > 1e-12 or nocc > nb:
            raise ValueError("integer occupations need an even electron count and enough bands")
        f = np.zeros(nb)
        f[:nocc] = 2.0
        mu = 0.5 * (eps[nocc - 1] + eps[nocc]) if nocc < nb else eps[-1]
        return f, mu, 0.0
    if nel > 2.0 * nb:
        raise ValueError("not enough bands")
    lo, hi = eps.min() - 40.0 * kT - 1.0, eps.max() + 40.0 * kT + 1.0

    def count(mu):
        return float(np.sum(2.0 * expit(-(eps - mu) / kT)))

    for _ in range(200):
        mu = 0.5 * (lo + hi)
        if count(mu) < nel:
            lo = mu
        else:
            hi = mu
        if hi - lo < 1e-15:
            break
    mu = 0.5 * (lo + hi)
    x = expit(-(eps - mu) / kT)
    f = 2.0 * x
    with np.errstate(divide="ignore", invalid="ignore"):
        s = np.where(x > 0, x * np.log(x), 0.0) + np.where(x < 1, (1 - x) * np.log1p(-x), 0.0)
    return f, mu, -2.0 * float(np.sum(s))


# ---------------------------------------------------------------------------
# Eigen-solvers (exact lowest nb eigenpairs; not Algorithm 1)
# ---------------------------------------------------------------------------
def solve_dense(model, veff_r, beta, nb):
    H = dense_h(model, veff_r, beta)
    w, v = scipy.linalg.eigh(H, subset_by_index=[0, nb - 1])
    return w, v


def solve_lobpcg(model, veff_r, beta, nb, C0=None, tol=1e-9, seed=0):
    extra = 4
    k = nb + extra
    op = scipy.sparse.linalg.LinearOperator((model.npw, model.npw), dtype=np.complex128,
                                            matvec=lambda x: apply_h(model, veff_r, beta, x.reshape(-1, 1))[:, 0],
                                            matmat=lambda X: apply_h(model, veff_r, beta, X))
    pre = 1.0 / (0.5 * model.g2 + 1.0)
    M = scipy.sparse.linalg.LinearOperator((model.npw, model.npw), dtype=np.complex128,
                                           matvec=lambda x: pre * x.ravel(), matmat=lambda X: pre[:, None] * X)
    if C0 is None or C0.shape[1] < k:
        rng = np.random.default_rng(seed)
        X = (rng.normal(size=(model.npw, k)) + 1j * rng.normal(size=(model.npw, k))) / (1.0 + model.g2[:, None])
        if C0 is not None:
            X[:, :C0.shape[1]] = C0
    else:
        X = C0[:, :k].copy()
    for _ in range(20):
        w, X = scipy.sparse.linalg.lobpcg(op, X, M=M, largest=False, tol=tol, maxiter=400)
        order = np.argsort(w)
        w, X = w[order], X[:, order]
        R = apply_h(model, veff_r, beta, X[:, :nb]) - X[:, :nb] * w[None, :nb]
        if np.max(np.linalg.norm(R, axis=0)) < 10 * tol:
            break
    return w[:nb], X[:, :nb], X


# ---------------------------------------------------------------------------
# SCF
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Result:
    free_energy: float          # F = E - kT S, Ha (the reported energy)
    energy: float               # E, Ha
    terms: dict
    forces: np.ndarray          # (n,3) Ha/bohr, -dF/dR
    eig: np.ndarray
    occ: np.ndarray
    mu: float
    rho: np.ndarray             # rho_out on the FFT grid
    rho_in: np.ndarray
    coeffs: np.ndarray          # (npw, nb) complex, full sphere
    n_iter: int
    resid: float
    history: list


def _kerker(model, R, q0):
    if q0 <= 0.0:
        return R
    rg = model.to_recip(R)
    rg *= model.bg2 / (model.bg2 + q0 * q0)
    return model.to_real(rg).real


def energy_terms(model, st, C, f, kT, S, beta, vion_g, rho_out, e_ew):
    """Every term of the total energy with the wavefunctions C and the density rho_out."""
    e_kin = float(np.sum(f * np.sum(0.5 * model.g2[:, None] * np.abs(C) ** 2, axis=0)))
    P = beta.conj() @ C
    e_nl = float(np.sum(f[None, :] * model.d[:, None] * np.abs(P) ** 2))
    e_loc = local_energy(model, vion_g, rho_out)
    e_h, _ = hartree(model, rho_out)
    e_xc, _ = xc(model, rho_out)
    e = e_kin + e_nl + e_loc + e_h + e_xc + e_ew
    ts = kT * S
    return dict(kinetic=e_kin, nonlocal_=e_nl, local=e_loc, hartree=e_h, xc=e_xc, ewald=e_ew,
                minus_ts=-ts, total=e - ts)


def forces(model, pos, C, f, beta, rho_out, f_ew):
    """Hellmann-Feynman forces F_I = -dF/dR_I (local + nonlocal + Ewald)."""
    n = len(model.spec)
    rg = model.to_recip(rho_out)
    out = np.array(f_ew, dtype=np.float64, copy=True)
    for I, s in enumerate(model.spec):
        ph = np.exp(-1j * (model.bG @ pos[I]))
        w = model.vloc_box[s] * ph * np.conj(rg)                       # d/dR adds (-iG)
        dE = model.omega * np.real(np.einsum("xyz,xyzc->c", -1j * w, model.bG))
        out[I] -= dE
    P = beta.conj() @ C                                                # (nproj, nb)
    for k, I in enumerate(model.proj_atom):
        for a in range(3):
            dP = (1j * model.G[:, a] * beta[k].conj()) @ C                # (nb,)
            dE = float(np.sum(f * model.d[k] * 2.0 * np.real(np.conj(P[k]) * dP)))
            out[I, a] -= dE
    return out


def scf(st, pos=None, tol_e=1e-8, tol_rho=1e-7, max_iter=200, mix=0.5, q0=0.8, hist=8,
        dense_max=3000, rho0=None, eta=None, verbose=False, model=None):
    """Self-consistent ground state and its energy and forces (Sec. II D).

    Stops when |F_k - F_{k-1}| < tol_e (Ha) and (Omega/N) sum |rho_out - rho_in| / N_el < tol_rho.
    Mixing: Pulay (DIIS) on the residual rho_out - rho_in with a Kerker-damped step.
    """
    if tuple(getattr(st, "kgrid", (1, 1, 1))) != (1, 1, 1):
        raise ValueError("a k-point mesh: oracle.kpoints.scf")
    model = Model(st) if model is None else model
    pos = np.asarray(st.pos if pos is None else pos, dtype=np.float64).reshape(-1, 3)
    nb = int(st.nbands)
    kT = float(st.kT)
    vion_g = ionic_potential_g(model, pos)
    vion_r = model.to_real(vion_g).real
    beta = projectors(model, pos)
    e_ew, f_ew = ewald(model.cell, model.z, pos, eta=eta)
    rho_in = initial_density(model, pos) if rho0 is None else np.array(rho0, dtype=np.float64)
    dv = model.omega / model.N
    hist_rho, hist_res = [], []
    F_prev = None
    Xfull = None
    history = []
    for it in range(1, max_iter + 1):
        _, vh = hartree(model, rho_in)
        _, vx = xc(model, rho_in)
        veff = vion_r + vh + vx
        if model.npw <= dense_max:
            eps, C = solve_dense(model, veff, beta, nb)
        else:
            eps, C, Xfull = solve_lobpcg(model, veff, beta, nb, C0=Xfull)
        f, mu, S = occupations(eps, model.nel, kT)
        rho_out = density(model, C, f)
        terms = energy_terms(model, st, C, f, kT, S, beta, vion_g, rho_out, e_ew)
        F = terms["total"]
        R = rho_out - rho_in
        resid = dv * float(np.sum(np.abs(R))) / model.nel
        history.append((F, resid))
        if verbose:
            print(f"scf {it:3d} F={F:.12f} dF={F - (F_prev or 0):.3e} resid={resid:.3e}")
        if F_prev is not None and abs(F - F_prev) < tol_e and resid < tol_rho:
            break
        F_prev = F
        hist_rho.append(rho_in)
        hist_res.append(R)
        hist_rho, hist_res = hist_rho[-hist:], hist_res[-hist:]
        m = len(hist_res)
        A = np.empty((m + 1, m + 1))
        for i in range(m):
            for j in range(m):
                A[i, j] = float(np.sum(hist_res[i] * hist_res[j]))
        A[m, :m] = A[:m, m] = 1.0
        A[m, m] = 0.0
        rhs = np.zeros(m + 1)
        rhs[m] = 1.0
        alpha = np.linalg.lstsq(A, rhs, rcond=None)[0][:m]
        rho_opt = sum(a * r for a, r in zip(alpha, hist_rho))
        res_opt = sum(a * r for a, r in zip(alpha, hist_res))
        rho_in = rho_opt + mix * _kerker(model, res_opt, q0)
    fo = forces(model, pos, C, f, beta, rho_out, f_ew)
    return Result(free_energy=F, energy=F + kT * S, terms=terms, forces=fo, eig=eps, occ=f, mu=mu,
                  rho=rho_out, rho_in=rho_in, coeffs=C, n_iter=it, resid=resid, history=history)


def evaluate(st, **kw):
    """(F, forces) of one structure: the energy+force evaluation of Sec. II A / II D."""
    r = scf(st, **kw)
    return r.free_energy, r.forces
