"""Pins of the oracle's p-channel projectors (oracle/pseudo.py beta_p_g, oracle/dft.py
projectors and forces): beta_m(r) = N_p x_m exp(-r^2/(2 s^2)), <beta_m|beta_m> = 1, strength
d_p, three projectors per atom after its s projector."""
import dataclasses
import math

import numpy as np

import workloads
from oracle import basis, dft, pseudo

SP = dict(workloads.SPECIES_Z4_P)


def test_normalisation_by_parseval():
    """sum_G |<G|beta_m>|^2 = <beta_m|beta_m> = 1 in a cell much larger than the projector."""
    cell = np.eye(3) * 22.0
    omega = basis.volume(cell)
    m, G, g2 = basis.sphere(cell, 60.0)
    b = pseudo.beta_p_g(SP, G, omega)
    for k in range(3):
        assert abs(np.sum(np.abs(b[k]) ** 2) - 1.0) < 1e-10


def test_real_space_shape():
    """Omega^{-1/2} sum_G <G|beta_x> exp(iG.r) = N_p x exp(-r^2/(2 s^2)) at a few points:
    pins the sign and the factor -i G_x s^2 of the transform."""
    cell = np.eye(3) * 22.0
    omega = basis.volume(cell)
    m, G, g2 = basis.sphere(cell, 60.0)
    b = pseudo.beta_p_g(SP, G, omega)
    s = SP["rp_p"]
    norm = 1.0 / math.sqrt(math.pi ** 1.5 * s ** 5 / 2.0)
    for r in (np.array([0.7, 0.2, -0.3]), np.array([-1.1, 0.5, 0.9]), np.array([0.0, 1.3, 0.0])):
        val = np.sum(b[0] * np.exp(1j * (G @ r))) / math.sqrt(omega)
        ref = norm * r[0] * math.exp(-(r @ r) / (2 * s * s))
        assert abs(val.imag) < 1e-10 and abs(val.real - ref) < 1e-9


def test_rotation_invariance_of_the_p_channel():
    """sum_m |<beta_m|psi>|^2 is unchanged when psi is rotated by 90 degrees about z (a
    symmetry of the cubic cell's sphere): a wrong component or sign in one beta_m breaks it."""
    cell = np.eye(3) * 7.0
    omega = basis.volume(cell)
    m, G, g2 = basis.sphere(cell, 6.0)
    rng = np.random.default_rng(3)
    c = rng.normal(size=len(g2)) + 1j * rng.normal(size=len(g2))
    index = {tuple(v): i for i, v in enumerate(m.tolist())}
    rot = np.array([index[(-v[1], v[0], v[2])] for v in m.tolist()])  # psi'(G) = psi(R^-1 G)
    b = pseudo.beta_p_g(SP, G, omega)
    before = np.sum(np.abs(b.conj() @ c) ** 2)
    after = np.sum(np.abs(b.conj() @ c[rot]) ** 2)
    assert abs(before - after) < 1e-12 * before
    # each component alone is not invariant (the test can see a swapped component)
    assert abs(abs(b[0].conj() @ c) - abs(b[0].conj() @ c[rot])) > 1e-6


def test_projector_layout_and_switch_off():
    st = workloads.tiny(nat=2, ecut=3.0, seed=7, species=SP)
    model = dft.Model(st)
    beta = dft.projectors(model, st.pos)
    assert beta.shape[0] == 8 and list(model.proj_atom) == [0, 0, 0, 0, 1, 1, 1, 1]
    assert list(model.d) == [1.0, 0.6, 0.6, 0.6] * 2
    st0 = dataclasses.replace(st, species=[dict(SP, d_p=0.0)])
    assert dft.projectors(dft.Model(st0), st.pos).shape[0] == 2


def test_pchannel_scf_forces_are_energy_derivatives():
    """Oracle SCF with the p channel: Hellmann-Feynman forces against central differences of
    the free energy (h = 1e-3 bohr), which holds only if every projector's derivative is
    attributed to its own atom."""
    import oracle
    st = workloads.tiny(nat=2, ecut=3.0, seed=7, kT=0.01, species=SP)
    r = oracle.scf(st, tol_e=1e-12, tol_rho=1e-10)
    h = 1e-3
    for (I, a) in [(0, 1), (1, 0)]:
        p = st.pos.copy()
        p[I, a] += h
        ep = oracle.scf(st.with_positions(p), tol_e=1e-12, tol_rho=1e-10).free_energy
        p[I, a] -= 2 * h
        em = oracle.scf(st.with_positions(p), tol_e=1e-12, tol_rho=1e-10).free_energy
        assert abs(-(ep - em) / (2 * h) - r.forces[I, a]) < 2e-5, (I, a)
    r0 = oracle.scf(dataclasses.replace(st, species=[dict(SP, d_p=0.0)]), tol_e=1e-12, tol_rho=1e-10)
    assert abs(r.terms["nonlocal_"] - r0.terms["nonlocal_"]) > 1e-3
