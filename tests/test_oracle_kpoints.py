"""Pins of the oracle's k-point form (oracle/kpoints.py): free-electron bands, Bloch
periodicity and time reversal of the spectrum, the zone-folding identity against the Gamma
oracle on the supercell, the Gamma mesh against dft.scf, and forces against finite
differences of the k-point free energy."""
import dataclasses

import numpy as np
import pytest

import workloads
from oracle import basis, dft, kpoints


def _tiny(**kw):
    # (a 12^3 box: the spheres of the mesh points are off-centre and reach further than
    # the Gamma sphere's 9^3)
    st = workloads.tiny(nat=2, ecut=3.0, seed=7, kT=0.01, nbands=9)
    return dataclasses.replace(st, **dict(dict(fft=(12, 12, 12)), **kw))


def test_free_electron_bands():
    """V_eff = 0 and no projectors: H_k is diagonal and its spectrum is sorted |k+G|^2/2,
    here compared with a brute-force enumeration of |k + m.B|^2/2 over a wide box."""
    st = _tiny()
    model = dft.Model(st)
    B = basis.reciprocal(model.cell)
    k = np.array([0.31, -0.12, 0.2]) @ B
    kb = kpoints.KBasis(model, k)
    H = kpoints.dense_h(model, kb, np.zeros(model.grid), np.zeros((0, kb.npw)))
    w = np.linalg.eigvalsh(H)
    r = np.arange(-8, 9)
    m = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    e = 0.5 * np.sum((k + m @ B) ** 2, axis=1)
    e = np.sort(e[e <= st.ecut])
    assert len(e) == kb.npw
    assert np.abs(w - e).max() < 1e-12


def _spectrum(model, k, veff, pos, nb=12):
    kb = kpoints.KBasis(model, k)
    H = kpoints.dense_h(model, kb, veff, kpoints.projectors(model, kb, pos))
    assert np.abs(H - H.conj().T).max() < 1e-13
    return np.linalg.eigvalsh(H)[:nb]


def test_bloch_periodicity_and_time_reversal():
    """eps_n(k + b_1) = eps_n(k) (the basis shifts by one reciprocal vector) and
    eps_n(-k) = eps_n(k) (a real potential); a k dropped from the kinetic energy, the
    projector phase or the sphere breaks the first, a sign error in the p channel's
    -i(k+G) factor or the phase breaks the second."""
    st = _tiny(species=[dict(workloads.SPECIES_Z4_P)])
    model = dft.Model(st)
    rng = np.random.default_rng(1)
    veff = model.to_real(model.to_recip(rng.normal(size=model.grid)) * (model.bg2 < 3.0) * model.sym).real
    B = basis.reciprocal(model.cell)
    k = np.array([0.23, 0.17, -0.31]) @ B
    e0 = _spectrum(model, k, veff, st.pos)
    assert np.abs(_spectrum(model, k + B[0], veff, st.pos) - e0).max() < 1e-11
    assert np.abs(_spectrum(model, -k, veff, st.pos) - e0).max() < 1e-11
    # the spectrum does depend on k
    assert np.abs(_spectrum(model, 0.5 * k, veff, st.pos) - e0).max() > 1e-3


def test_gamma_mesh_is_the_gamma_oracle():
    st = _tiny()
    r = kpoints.scf(st, kgrid=(1, 1, 1), tol_e=1e-11, tol_rho=1e-9)
    g = dft.scf(st, tol_e=1e-11, tol_rho=1e-9)
    assert abs(r.free_energy - g.free_energy) < 1e-9
    assert np.abs(r.forces - g.forces).max() < 1e-7
    assert np.abs(r.eig[0] - g.eig).max() < 1e-8


@pytest.mark.parametrize("kgrid,pchan", [((2, 1, 1), True), ((1, 2, 2), False)])
def test_zone_folding_identity(kgrid, pchan):
    """The n1 x n2 x n3 Gamma-centred mesh on a cell equals the Gamma point of the
    n1 x n2 x n3 supercell (same basis: the supercell's G are the cell's k + G): free energy
    per cell, the forces on the cell's atoms (each translate carries the same force) and the
    occupied band energies (the supercell's spectrum is the union of the eps_n(k)).  A
    kinetic energy of |G|^2 instead of |k+G|^2, p projectors along G instead of k+G, or
    unequal k weights in the density each move F by more than 0.1 Ha here."""
    st = _tiny(species=[dict(workloads.SPECIES_Z4_P if pchan else workloads.SPECIES_Z4)])
    nk = int(np.prod(kgrid))
    rk = kpoints.scf(st, kgrid=kgrid, tol_e=1e-11, tol_rho=1e-9)
    sup = workloads.supercell(st, kgrid)
    rs = dft.scf(sup, tol_e=1e-11, tol_rho=1e-9)
    assert abs(rs.free_energy / nk - rk.free_energy) < 1e-8
    na = st.natoms
    for t in range(nk):
        assert np.abs(rs.forces[t * na:(t + 1) * na] - rk.forces).max() < 2e-6
    ek = np.sort(rk.eig[rk.occ > 1e-6])
    es = np.sort(rs.eig[rs.occ > 1e-6])
    assert len(ek) == len(es) and np.abs(ek - es).max() < 1e-7
    # the mesh matters: the Gamma point alone gives another energy
    assert abs(dft.scf(st, tol_e=1e-11, tol_rho=1e-9).free_energy - rk.free_energy) > 1e-3


def test_zone_folding_identity_pbe():
    """The folding identity with PBE exchange-correlation: the gradient terms of the mesh's
    density (sum over k of |psi_nk|^2) are those of the supercell's."""
    st = _tiny(xc="pbe")
    rk = kpoints.scf(st, kgrid=(2, 1, 1), tol_e=1e-11, tol_rho=1e-9)
    rs = dft.scf(workloads.supercell(st, (2, 1, 1)), tol_e=1e-11, tol_rho=1e-9)
    assert abs(rs.free_energy / 2 - rk.free_energy) < 1e-8
    assert np.abs(rs.forces[:st.natoms] - rk.forces).max() < 2e-6
    assert abs(rs.terms["xc"] / 2 - rk.terms["xc"]) < 1e-8
    # PBE differs from LDA on the mesh as well
    assert abs(kpoints.scf(_tiny(), kgrid=(2, 1, 1), tol_e=1e-11, tol_rho=1e-9).free_energy - rk.free_energy) > 1e-3


def test_kpoint_forces_are_energy_derivatives():
    st = _tiny(kgrid=(2, 1, 1), species=[dict(workloads.SPECIES_Z4_P)])
    r = kpoints.scf(st, tol_e=1e-12, tol_rho=1e-10)
    h = 1e-3
    for (I, a) in [(0, 1), (1, 2)]:
        p = st.pos.copy()
        p[I, a] += h
        ep = kpoints.scf(st, pos=p, tol_e=1e-12, tol_rho=1e-10).free_energy
        p[I, a] -= 2 * h
        em = kpoints.scf(st, pos=p, tol_e=1e-12, tol_rho=1e-10).free_energy
        assert abs(-(ep - em) / (2 * h) - r.forces[I, a]) < 2e-5, (I, a)


def test_integer_occupations_on_a_mesh():
    """kT = 0: f = 2 on the N_el / (2 w) lowest states of the whole mesh."""
    eps = np.array([[0.0, 1.0, 2.0], [0.5, 0.7, 3.0]])
    f, mu, S = kpoints.occupations(eps, np.array([0.5, 0.5]), 4.0, 0.0)
    assert np.array_equal(f, np.array([[2.0, 2.0, 0.0], [2.0, 2.0, 0.0]])) and S == 0.0
    assert mu == 1.5
    # Fermi-Dirac on a mesh: the weighted count is N_el
    f2, mu2, S2 = kpoints.occupations(eps, np.array([0.25, 0.75]), 3.0, 0.05)
    assert abs(float(np.sum(np.array([0.25, 0.75])[:, None] * f2)) - 3.0) < 1e-12 and S2 > 0.0
