"""Brillouin-zone sampling by Bloch wavevectors k (oracle; test infrastructure only).

The paper lets its local relaxations use a rough k-point sampling grid (Sec. II C,
the paragraph on the cost of the relaxations) while its clusters are computed at one
point; this module is the textbook k-point form of the same energy (Ihm, Zunger & Cohen,
J. Phys. C 12, 4409 (1979), Eq. 13 summed over the k mesh):

    psi_nk(r) = Omega^{-1/2} sum_G c_nk(G) exp(i(k+G).r),  sum_G |c_nk(G)|^2 = 1,
    basis |k+G|^2/2 <= Ecut at each k (complex coefficients, no Gamma symmetry),
    H_k(G,G') = |k+G|^2/2 delta + V_eff(G-G') + sum_j D_j beta_j(k+G) beta_j(k+G')^*,
    beta_j(k+G) = <k+G|beta_j> at the atom: the origin-centred transform times exp(-i(k+G).R),
    rho(r) = sum_k w_k sum_n f_nk |psi_nk(r)|^2,
    one Fermi level over every (n, k) with weights w_k: sum_k w_k sum_n f_nk = N_el,
    E = sum_k w_k sum_n f_nk <psi_nk| T + V_NL |psi_nk> + (the density terms of dft.py),
    F = E - kT S with S = -2 sum_k w_k sum_n [x ln x + (1 - x) ln(1 - x)], x = f/2.

The mesh is Monkhorst-Pack's, Gamma-centred: k = sum_i (t_i / n_i) b_i, t_i = 0 .. n_i - 1,
w_k = 1 / (n_1 n_2 n_3).  Each H_k is diagonalised densely; everything else (V_eff, the
mixing, Ewald) is shared with the Gamma oracle in dft.py.  Independent of the CUDA path,
which reaches the same energy through the Gamma point of the n_1 x n_2 x n_3 supercell.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg
from scipy.special import expit

from . import basis, dft
from .ewald import ewald
from .pseudo import beta_g, beta_p_g


def mesh(cell, kgrid):
    """Cartesian k (nk, 3) and weights (nk,) of the Gamma-centred n1 x n2 x n3 mesh."""
    B = basis.reciprocal(cell)
    t = np.stack(np.meshgrid(*[np.arange(n) for n in kgrid], indexing="ij"), -1).reshape(-1, 3)
    frac = t / np.asarray(kgrid, dtype=np.float64)
    return frac @ B, np.full(len(t), 1.0 / len(t))


def sphere_k(cell, ecut, k):
    """Miller indices m and the vectors k+G of the basis |k+G|^2/2 <= Ecut, and |k+G|^2.

    |m_i| = |a_i . G| / 2 pi <= |a_i| (sqrt(2 Ecut) + |k|) / 2 pi bounds the box."""
    cell = np.asarray(cell, dtype=np.float64)
    B = basis.reciprocal(cell)
    kn = float(np.linalg.norm(k))
    mx = np.floor(np.linalg.norm(cell, axis=1) * (math.sqrt(2.0 * ecut) + kn) / (2.0 * math.pi)).astype(int) + 1
    r = [np.arange(-x, x + 1) for x in mx]
    m = np.stack(np.meshgrid(*r, indexing="ij"), axis=-1).reshape(-1, 3)
    kG = np.asarray(k, dtype=np.float64)[None, :] + m @ B
    g2 = np.einsum("ij,ij->i", kG, kG)
    keep = 0.5 * g2 <= ecut
    m, kG, g2 = m[keep], kG[keep], g2[keep]
    order = np.lexsort((m[:, 2], m[:, 1], m[:, 0], np.round(g2, 10)))
    return m[order], kG[order], g2[order]


class KBasis:
    """Basis of one k: Miller indices, k+G, |k+G|^2 and grid positions."""

    def __init__(self, model, k):
        self.k = np.asarray(k, dtype=np.float64)
        self.m, self.kG, self.g2 = sphere_k(model.cell, model.st.ecut, self.k)
        self.npw = len(self.g2)
        self.idx = basis.grid_index(self.m, model.grid)
        # alias-free: the density and V_eff psi reach Miller differences up to twice the
        # basis' extent per axis (4 m_max + 1 for a sphere centred at the origin)
        span = np.max(self.m, axis=0) - np.min(self.m, axis=0)
        if any(n < 2 * x + 1 for n, x in zip(model.grid, span)):
            raise ValueError(f"FFT grid {model.grid} aliases for the basis extent {span} at k = {self.k}")


def projectors(model, kb, pos):
    """beta_j(k+G) exp(-i(k+G).R_I(j)) for every projector j (the atom-major order of
    dft.projectors), shape (nproj, npw_k)."""
    rows = []
    for I, s in enumerate(model.spec):
        sp = model.species[s]
        ph = np.exp(-1j * (kb.kG @ pos[I]))
        rows.append(beta_g(sp, kb.g2, model.omega) * ph)
        if sp.get("d_p", 0.0) != 0.0:
            bp = beta_p_g(sp, kb.kG, model.omega)
            rows += [bp[m] * ph for m in range(3)]
    return np.array(rows).reshape(-1, kb.npw)


def dense_h(model, kb, veff_r, beta):
    """H_k(G,G') = |k+G|^2/2 delta + V_eff(G-G') + sum_j D_j beta_j(k+G) beta_j(k+G')^*."""
    vg = model.to_recip(veff_r)
    dm = kb.m[:, None, :] - kb.m[None, :, :]
    H = vg[dm[..., 0] % model.grid[0], dm[..., 1] % model.grid[1], dm[..., 2] % model.grid[2]]
    H = H + np.diag(0.5 * kb.g2)
    if len(beta):
        H = H + (beta.T * model.d[None, :]) @ beta.conj()
    return H


def occupations(eps, w, nel, kT):
    """(f, mu, S) over every (n, k): eps (nk, nb), weights w (nk,).

    kT > 0: Fermi-Dirac, mu by bisection so that sum_k w_k sum_n f_nk = N_el.  kT = 0:
    f = 2 on the N_el/2 / w lowest states of the mesh (each state carries weight w; the mesh
    must then be uniform and N_el / (2 w) an integer), 0 elsewhere."""
    eps = np.asarray(eps, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    if kT <= 0.0:
        if not np.allclose(w, w[0]):
            raise ValueError("integer occupations need a uniform mesh")
        nstate = nel / (2.0 * w[0])
        nocc = int(round(nstate))
        if abs(nocc - nstate) > 1e-9 or nocc > eps.size:
            raise ValueError("integer occupations need N_el/(2w) integral and enough bands")
        order = np.argsort(eps, axis=None, kind="stable")
        f = np.zeros(eps.size)
        f[order[:nocc]] = 2.0
        flat = eps.ravel()[order]
        mu = 0.5 * (flat[nocc - 1] + flat[nocc]) if nocc < eps.size else flat[-1]
        return f.reshape(eps.shape), mu, 0.0
    if nel > 2.0 * float(np.sum(w)) * eps.shape[1] + 1e-12:
        raise ValueError("not enough bands")
    lo, hi = eps.min() - 40.0 * kT - 1.0, eps.max() + 40.0 * kT + 1.0

    def count(mu):
        return float(np.sum(w[:, None] * 2.0 * expit(-(eps - mu) / kT)))

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
    with np.errstate(divide="ignore", invalid="ignore"):
        s = np.where(x > 0, x * np.log(x), 0.0) + np.where(x < 1, (1 - x) * np.log1p(-x), 0.0)
    return 2.0 * x, mu, -2.0 * float(np.sum(w[:, None] * s))


def density(model, kbs, w, C, f):
    """rho(r) = sum_k w_k sum_n f_nk |psi_nk(r)|^2 (|exp(ik.r)| = 1 drops out)."""
    rho = np.zeros(model.grid)
    for kb, wk, Ck, fk in zip(kbs, w, C, f):
        g = np.zeros((Ck.shape[1],) + model.grid, dtype=np.complex128)
        g[(slice(None),) + kb.idx] = Ck.T
        psi = np.fft.ifftn(g, axes=(1, 2, 3)) * (model.N / math.sqrt(model.omega))
        rho += wk * np.einsum("n,nxyz->xyz", fk, np.abs(psi) ** 2)
    return rho


def band_terms(model, kbs, w, C, f, betas):
    """(E_kin, E_nl) = sum_k w_k sum_n f_nk <psi_nk| -1/2 nabla^2 | V_NL |psi_nk>."""
    e_kin = e_nl = 0.0
    for kb, wk, Ck, fk, bk in zip(kbs, w, C, f, betas):
        e_kin += wk * float(np.sum(fk * np.sum(0.5 * kb.g2[:, None] * np.abs(Ck) ** 2, axis=0)))
        P = bk.conj() @ Ck
        e_nl += wk * float(np.sum(fk[None, :] * model.d[:, None] * np.abs(P) ** 2))
    return e_kin, e_nl


def forces(model, pos, kbs, w, C, f, betas, rho_out, f_ew):
    """F_I = -dF/dR_I: local (the density's, as in dft.forces), Ewald, and the nonlocal part
    summed over the mesh with d [beta_j(k+G) exp(-i(k+G).R)] / dR = -i (k+G) (...)."""
    rg = model.to_recip(rho_out)
    out = np.array(f_ew, dtype=np.float64, copy=True)
    for I, s in enumerate(model.spec):
        wv = model.vloc_box[s] * np.exp(-1j * (model.bG @ pos[I])) * np.conj(rg)   # d/dR adds (-iG)
        out[I] -= model.omega * np.real(np.einsum("xyz,xyzc->c", -1j * wv, model.bG))
    for kb, wk, Ck, fk, bk in zip(kbs, w, C, f, betas):
        P = bk.conj() @ Ck
        for j, I in enumerate(model.proj_atom):
            for a in range(3):
                dP = (1j * kb.kG[:, a] * bk[j].conj()) @ Ck
                out[I, a] -= wk * float(np.sum(fk * model.d[j] * 2.0 * np.real(np.conj(P[j]) * dP)))
    return out


def scf(st, pos=None, kgrid=None, tol_e=1e-8, tol_rho=1e-7, max_iter=200, mix=0.5, q0=0.8, hist=8,
        verbose=False):
    """Self-consistent ground state on the k mesh (st.kgrid unless kgrid is given): the SCF
    cycle of dft.scf (Pulay on rho_out - rho_in with a Kerker-damped step, the same stopping
    rule) with the Kohn-Sham problem solved at every k.  nbands bands per k."""
    kgrid = tuple(int(x) for x in (kgrid if kgrid is not None else getattr(st, "kgrid", (1, 1, 1))))
    model = dft.Model(st)
    pos = np.asarray(st.pos if pos is None else pos, dtype=np.float64).reshape(-1, 3)
    nb = int(st.nbands)
    kT = float(st.kT)
    K, w = mesh(model.cell, kgrid)
    kbs = [KBasis(model, k) for k in K]
    betas = [projectors(model, kb, pos) for kb in kbs]
    vion_g = dft.ionic_potential_g(model, pos)
    vion_r = model.to_real(vion_g).real
    e_ew, f_ew = ewald(model.cell, model.z, pos)
    rho_in = dft.initial_density(model, pos)
    dv = model.omega / model.N
    hist_rho, hist_res = [], []
    F_prev = None
    history = []
    for it in range(1, max_iter + 1):
        _, vh = dft.hartree(model, rho_in)
        _, vx = dft.xc(model, rho_in)
        veff = vion_r + vh + vx
        eps, C = [], []
        for kb, bk in zip(kbs, betas):
            wk_, vk_ = scipy.linalg.eigh(dense_h(model, kb, veff, bk), subset_by_index=[0, nb - 1])
            eps.append(wk_)
            C.append(vk_)
        eps = np.array(eps)
        f, mu, S = occupations(eps, w, model.nel, kT)
        rho_out = density(model, kbs, w, C, f)
        e_kin, e_nl = band_terms(model, kbs, w, C, f, betas)
        e_loc = dft.local_energy(model, vion_g, rho_out)
        e_h, _ = dft.hartree(model, rho_out)
        e_xc, _ = dft.xc(model, rho_out)
        F = e_kin + e_nl + e_loc + e_h + e_xc + e_ew - kT * S
        terms = dict(kinetic=e_kin, nonlocal_=e_nl, local=e_loc, hartree=e_h, xc=e_xc, ewald=e_ew,
                     minus_ts=-kT * S, total=F)
        R = rho_out - rho_in
        resid = dv * float(np.sum(np.abs(R))) / model.nel
        history.append((F, resid))
        if verbose:
            print(f"scf_k {it:3d} F={F:.12f} resid={resid:.3e}")
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
        rho_in = rho_opt + mix * dft._kerker(model, res_opt, q0)
    fo = forces(model, pos, kbs, w, C, f, betas, rho_out, f_ew)
    return dft.Result(free_energy=F, energy=F + kT * S, terms=terms, forces=fo, eig=eps, occ=f, mu=mu,
                      rho=rho_out, rho_in=rho_in, coeffs=C, n_iter=it, resid=resid, history=history)
