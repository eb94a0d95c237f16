"""Pins of the oracle's self-consistent energy and forces: exact derivatives, invariances,
the fixed-point property and symmetry.  All cases are small enough for the CPU suite."""
import numpy as np
import pytest

import workloads
from oracle import dft, scf

TIGHT = dict(tol_e=1e-12, tol_rho=1e-10)


@pytest.fixture(scope="module")
def tiny_state():
    st = workloads.tiny(nat=2, ecut=3.0, kT=0.01)
    return st, scf(st, **TIGHT)


def test_forces_match_finite_differences(tiny_state):
    """F_I = -dF/dR_I, central differences h = 1e-3 bohr, on the Mermin free energy."""
    st, r = tiny_state
    h = 1e-3
    for I, a in [(0, 0), (1, 2), (0, 1), (1, 0)]:
        p = st.pos.copy(); p[I, a] += h
        fp = scf(st, pos=p, **TIGHT).free_energy
        p[I, a] -= 2 * h
        fm = scf(st, pos=p, **TIGHT).free_energy
        assert abs(-(fp - fm) / (2 * h) - r.forces[I, a]) < 1e-6


def pz81_join_quantum(omega, ngrid):
    """Energy step of one grid point whose density crosses r_s = 1.  The published PZ81
    constants join the two correlation branches only to their printed digits:
    eps_c(r_s -> 1-) = B + D = -0.0596 against gamma / (1 + beta1 + beta2) = -0.0596321 Ha,
    a step of 3.2066e-5 Ha per electron at rho_c = 3/(4 pi); one grid point carries
    (Omega/N) rho_c electrons, so F steps by (Omega/N) rho_c 3.2066e-5 Ha."""
    step = (-0.048 - 0.0116) - (-0.1423 / (1.0 + 1.0529 + 0.3334))
    return omega / ngrid * 3.0 / (4.0 * np.pi) * step


def test_energy_steps_are_the_pz81_join():
    """Hard Z = 10 atoms at 15 Ha: the valence density rises above rho_c = 3/(4 pi) (r_s < 1)
    at some grid points, so moving an atom makes points cross the branch join of the PZ81
    correlation fit.  Along a 9-point line the free energy minus the integral of -F (the
    forces are the derivative of F between crossings) must take only integer multiples of
    the quantum (Omega/N) rho_c * 3.2066e-5 Ha, and some crossing must occur; a force or
    energy error of another kind would leave a residue that is not such a multiple."""
    st = workloads.tiny(nat=2, ecut=15.0, kT=0.01, species=workloads.SPECIES_Z10)
    r = scf(st, **TIGHT)
    J = pz81_join_quantum(abs(np.linalg.det(st.cell)), np.prod(st.fft))
    xs = np.linspace(-2e-3, 2e-3, 9)
    E, F = [], []
    for x in xs:
        p = st.pos.copy(); p[0, 0] += x
        q = scf(st, pos=p, tol_e=1e-12, tol_rho=1e-10, rho0=r.rho_in)
        E.append(q.free_energy)
        F.append(q.forces[0, 0])
    E, F = np.array(E), np.array(F)
    integral = np.concatenate([[0.0], np.cumsum(-0.5 * (F[1:] + F[:-1]) * np.diff(xs))])
    k = ((E - E[0]) - integral) / J
    assert np.abs(k - np.round(k)).max() < 1e-3, k
    assert np.abs(np.round(k)).max() >= 1, k


def test_forces_match_finite_differences_integer_occupations():
    st = workloads.tiny(nat=2, ecut=3.0, kT=0.0, nbands=6, seed=11)
    r = scf(st, **TIGHT)
    h = 1e-3
    p = st.pos.copy(); p[0, 2] += h
    fp = scf(st, pos=p, **TIGHT).free_energy
    p[0, 2] -= 2 * h
    fm = scf(st, pos=p, **TIGHT).free_energy
    assert abs(-(fp - fm) / (2 * h) - r.forces[0, 2]) < 1e-6


def test_permutation_invariance(tiny_state):
    st, r = tiny_state
    r2 = scf(st.with_positions(st.pos[::-1]), **TIGHT)
    assert abs(r2.free_energy - r.free_energy) < 1e-10
    assert np.abs(r2.forces[::-1] - r.forces).max() < 1e-8


def test_lattice_translation_invariance(tiny_state):
    st, r = tiny_state
    r2 = scf(st.with_positions(st.pos + st.cell[1] - 2 * st.cell[2]), **TIGHT)
    assert abs(r2.free_energy - r.free_energy) < 1e-10
    assert np.abs(r2.forces - r.forces).max() < 1e-8


def test_grid_translation_invariance(tiny_state):
    """A shift by a grid vector A^T (k/N) maps the grid onto itself: same energy (SCF tol)."""
    st, r = tiny_state
    shift = (np.array([2, 1, 3]) / np.array(st.fft)) @ st.cell
    r2 = scf(st.with_positions(st.pos + shift), **TIGHT)
    assert abs(r2.free_energy - r.free_energy) < 1e-9
    assert np.abs(r2.forces - r.forces).max() < 1e-7


def test_net_force_is_eggbox_only(tiny_state):
    """sum_I F_I vanishes up to the grid (egg-box) term of the XC energy, which shrinks fast
    with a finer grid; a wrong-sign or missing force term would leave an O(|F|) remainder."""
    st, r = tiny_state
    coarse = np.abs(r.forces.sum(0)).max()
    fine = scf(workloads.Structure(**{**st.__dict__, "fft": (16, 16, 16)}), **TIGHT)
    assert np.abs(fine.forces.sum(0)).max() < 0.2 * max(coarse, 1e-6) + 1e-7
    assert np.abs(fine.forces.sum(0)).max() < 1e-3 * np.abs(fine.forces).max() + 1e-6


def test_fixed_point_restart(tiny_state):
    """Restarting from the converged rho_in converges at once to the same energy."""
    st, r = tiny_state
    r2 = scf(st, rho0=r.rho_in, **TIGHT)
    assert r2.n_iter <= 3
    assert abs(r2.free_energy - r.free_energy) < 1e-10


def test_result_independent_of_mixing(tiny_state):
    st, r = tiny_state
    r2 = scf(st, mix=0.3, q0=0.0, hist=4, **TIGHT)
    assert abs(r2.free_energy - r.free_energy) < 1e-9


def test_eigenpairs_and_density_consistent(tiny_state):
    """At convergence the states are eigenvectors of H[rho] and rho_out = rho_in."""
    st, r = tiny_state
    m = dft.Model(st)
    vion = m.to_real(dft.ionic_potential_g(m, st.pos)).real
    _, vh = dft.hartree(m, r.rho)
    _, vx = dft.xc(m, r.rho)
    beta = dft.projectors(m, st.pos)
    R = dft.apply_h(m, vion + vh + vx, beta, r.coeffs) - r.coeffs * r.eig[None, :]
    assert np.linalg.norm(R, axis=0).max() < 1e-7
    assert np.allclose(r.coeffs.conj().T @ r.coeffs, np.eye(st.nbands), atol=1e-12)
    assert abs(m.omega / m.N * r.rho.sum() - m.nel) < 1e-10


def test_variational_minimum(tiny_state):
    """The Kohn-Sham energy at fixed occupations is stationary: rotating an occupied state
    into an empty one by angle t raises E by O(t^2), not O(t)."""
    st, r = tiny_state
    m = dft.Model(st)
    beta = dft.projectors(m, st.pos)
    vion_g = dft.ionic_potential_g(m, st.pos)
    from oracle.ewald import ewald
    e_ew, _ = ewald(m.cell, m.z, st.pos)

    def energy(C):
        rho = dft.density(m, C, r.occ)
        return dft.energy_terms(m, st, C, r.occ, 0.0, 0.0, beta, vion_g, rho, e_ew)["total"]

    e0 = energy(r.coeffs)
    de = []
    for t in (1e-3, 2e-3):
        C = r.coeffs.copy()
        a, b = C[:, 0].copy(), C[:, -1].copy()
        C[:, 0] = np.cos(t) * a + np.sin(t) * b
        C[:, -1] = -np.sin(t) * a + np.cos(t) * b
        de.append(energy(C) - e0)
    assert de[0] > 0 and de[1] > 0
    assert abs(de[1] / de[0] - 4.0) < 0.05


def test_ideal_diamond_forces_vanish():
    """Ideal diamond (no jitter) at a reduced cutoff: every atom sits at an inversion-related
    site, so F = 0 by symmetry."""
    st = workloads.diamond8(jitter=0.0)
    st = workloads.Structure(**{**st.__dict__, "ecut": 4.0, "fft": (18, 18, 18)})
    r = scf(st, tol_e=1e-10, tol_rho=1e-8, mix=0.7, q0=0.0)
    assert np.abs(r.forces).max() < 1e-7


def test_iterative_eigensolver_matches_dense(tiny_state):
    """The LOBPCG route (FFT-applied H) reaches the same fixed point as dense LAPACK."""
    st, r = tiny_state
    r2 = scf(st, dense_max=0, **TIGHT)
    assert abs(r2.free_energy - r.free_energy) < 1e-9
    assert np.abs(r2.eig - r.eig).max() < 1e-8
    assert np.abs(r2.forces - r.forces).max() < 1e-6
