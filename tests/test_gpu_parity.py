"""CUDA path vs the FP64 CPU oracle, through the C ABI.

Tolerances: the plain FP64 path reaches the oracle's fixed point to the SCF
tolerance (energy 1e-7 Ha/atom, forces 1e-6 Ha/bohr here).  The mixed path (FP32
H.psi, FFTs and GEMM products, FP64 sums) must stay within 1e-5 Ha/atom and
1e-4 Ha/bohr.  Component kernels (H.psi, density) are compared element by element.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle import dft, kpoints
from tests.packing import full_from_packed

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sgo():
    from paper_1603_02732_gb300 import build
    build.build()
    import paper_1603_02732_gb300 as pkg
    pkg.load_library()
    return pkg


def _struct(grid=None, ecut=3.5, nat=2, seed=7, kT=0.01, nbands=None):
    st = workloads.tiny(nat=nat, ecut=ecut, seed=seed, kT=kT, nbands=nbands)
    if grid is not None:
        st = dataclasses.replace(st, fft=tuple(grid))
    return st


# every FFT radix: 9 (9), 10 12 15 (10,12,15), 16 9 2 10 (16,18,20), 12 2 (24),
# 15 2 / 9 6 / 10 4 (30,54,40), 9 2 / 12 3 / 16 8 (18,36,128); the mixed path's
# register plane transforms in both size classes: 45 40, 60 50, 72 64, 27 25, 20 48, and
# planes that give every register length a turn along x and along y (the multi-pass plane pass
# factors each differently: 12 = 3 x 4 ... 72 = 8 x 9)
GRIDS = [None, (10, 12, 15), (16, 18, 20), (24, 24, 24), (30, 54, 40), (18, 36, 128), (45, 40, 16),
         (60, 50, 12), (72, 64, 10), (27, 25, 32), (20, 48, 15), (36, 32, 15), (15, 36, 32),
         (12, 10, 12), (25, 15, 10), (32, 16, 10), (40, 20, 10), (48, 27, 10), (50, 30, 10),
         (54, 45, 10), (64, 60, 10), (24, 72, 10),
         # lane-pair register transforms (mixed path): planes 96 x 128 and 100 x 108, z 96 / 120;
         # the FP64 path takes these two planes by line blocks through a global buffer
         (96, 128, 12), (100, 108, 10), (20, 24, 96), (12, 10, 120)]


@pytest.mark.parametrize("grid", GRIDS)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_apply_hamiltonian_matches_dense_h(sgo, grid, precision):
    st = _struct(grid=grid)
    ctx = sgo.Context(st, precision=precision)
    m = dft.Model(st)
    miller = ctx.basis()
    # the packed basis is exactly the oracle's Ecut sphere (half + inversion)
    full = set(map(tuple, miller.tolist())) | set(map(tuple, (-miller).tolist()))
    assert full == set(map(tuple, m.m.tolist()))
    rng = np.random.default_rng(11)
    veff = rng.normal(size=m.grid) * 0.3
    x = rng.normal(size=(st.nbands, ctx.npw))
    y = ctx.apply_hamiltonian(veff, x)
    H = dft.dense_h(m, veff, dft.projectors(m, st.pos))
    c = full_from_packed(m, miller, x)
    y_ref = full_from_packed(m, miller, np.zeros_like(x))  # shape only
    y_ref = H @ c
    y_full = full_from_packed(m, miller, y)
    tol = 1e-11 if precision == "fp64" else 2e-5
    scale = np.abs(y_ref).max()
    assert np.abs(y_full - y_ref).max() < tol * scale


@pytest.mark.parametrize("grid", [None, (10, 12, 15), (18, 20, 24), (30, 54, 40), (96, 128, 12), (20, 24, 96)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_density_matches_oracle(sgo, grid, precision):
    st = _struct(grid=grid, nbands=7)
    ctx = sgo.Context(st, precision=precision)
    m = dft.Model(st)
    miller = ctx.basis()
    rng = np.random.default_rng(5)
    x = rng.normal(size=(7, ctx.npw))
    x, _ = np.linalg.qr(x.T)
    x = x.T.copy()
    occ = np.array([2.0, 2.0, 1.7, 1.1, 0.4, 0.0, 0.05])
    rho = ctx.density_of(x, occ)
    ref = dft.density(m, full_from_packed(m, miller, x), occ)
    tol = 1e-12 if precision == "fp64" else 1e-6
    assert np.abs(rho - ref).max() < tol * np.abs(ref).max()
    assert abs(m.omega / m.N * rho.sum() - occ.sum()) < (1e-10 if precision == "fp64" else 1e-5)


def _compare(st, res_gpu, ref, e_tol, f_tol):
    F, forces = res_gpu
    dE = abs(F - ref.free_energy) / st.natoms
    dF = float(np.abs(forces - ref.forces).max())
    assert dE < e_tol, (F, ref.free_energy, dE)
    assert dF < f_tol, (forces, ref.forces, dF)


@pytest.mark.parametrize("kT,nbands", [(0.01, None), (0.0, 6)])
def test_scf_tiny_fp64(sgo, kT, nbands):
    st = _struct(kT=kT, nbands=nbands, ecut=3.0)
    ref = oracle.scf(st, tol_e=1e-12, tol_rho=1e-10)
    ctx = sgo.Context(st, precision="fp64", scf_tol_e=1e-11, scf_tol_rho=1e-9, max_scf=120)
    _compare(st, ctx.energy_forces(), ref, 1e-8, 1e-6)
    eig, occ = ctx.eigen()
    assert np.abs(eig - ref.eig).max() < 1e-7
    assert np.abs(occ - ref.occ).max() < 1e-6
    t = ctx.terms()
    for k_gpu, k_ref in [("kinetic", "kinetic"), ("nonlocal", "nonlocal_"), ("local", "local"),
                         ("hartree", "hartree"), ("xc", "xc"), ("ewald", "ewald"), ("minus_ts", "minus_ts")]:
        assert abs(t[k_gpu] - ref.terms[k_ref]) < 1e-6, k_gpu
    rho = ctx.density()
    assert np.abs(rho - ref.rho).max() < 1e-6 * np.abs(ref.rho).max()


def test_scf_big_plane_fp64(sgo):
    """FP64 SCF, energy terms, density and forces on a 96 x 128 x 12 grid, whose planes the
    FP64 path takes by line blocks through a global buffer (H.psi, density and the grid
    transforms), against the oracle."""
    st = _struct(ecut=3.0, grid=(96, 128, 12))
    ref = oracle.scf(st, tol_e=1e-12, tol_rho=1e-10)
    ctx = sgo.Context(st, precision="fp64", scf_tol_e=1e-11, scf_tol_rho=1e-9, max_scf=120)
    _compare(st, ctx.energy_forces(), ref, 1e-8, 1e-6)
    eig, _ = ctx.eigen()
    assert np.abs(eig - ref.eig)[ref.occ > 1e-6].max() < 1e-7
    rho = ctx.density()
    assert np.abs(rho - ref.rho).max() < 1e-6 * np.abs(ref.rho).max()


@pytest.mark.parametrize("rr_cluster", [1, 0])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_scf_cluster_eigensolver(sgo, precision, rr_cluster):
    """A subspace too large for one CTA's shared memory (112 requested bands, 119 carried):
    the subspace diagonalisation runs on a thread-block cluster of 8 CTAs (Cholesky in
    deviation form, one-sided Jacobi; rr_cluster = 1, the default at this size) or on one
    CTA over a global scratch (rr_cluster = 0), in both precisions; SCF energy, occupied
    eigenvalues and forces against the oracle."""
    st = _struct(ecut=6.0, nbands=112)
    ref = oracle.scf(st, tol_e=1e-12, tol_rho=1e-10)
    if precision == "fp64":
        ctx = sgo.Context(st, precision="fp64", scf_tol_e=1e-11, scf_tol_rho=1e-9, max_scf=120,
                          rr_cluster=rr_cluster)
        _compare(st, ctx.energy_forces(), ref, 1e-8, 1e-6)
        tol_eig = 1e-7
    else:
        ctx = sgo.Context(st, precision="mixed", scf_tol_e=1e-7, scf_tol_rho=1e-5, max_scf=120,
                          rr_cluster=rr_cluster)
        _compare(st, ctx.energy_forces(), ref, 1e-5, 1e-4)
        tol_eig = 2e-4
    eig, _ = ctx.eigen()
    assert np.abs(eig - ref.eig)[ref.occ > 1e-6].max() < tol_eig
    assert ctx.stats()["jacobi_cap_hits"] == 0


@pytest.mark.parametrize("precision,case", [("fp64", "tiny"), ("mixed", "tiny"), ("fp64", "bands112"),
                                            ("fp64", "diamond8"), ("mixed", "diamond8")])
def test_scf_davidson(sgo, precision, case, request):
    """Block Davidson steps (eigensolver = 1: per step the projected, preconditioned residuals
    W of all bands and one Rayleigh-Ritz over the 2 n_b block [X, W]) reach the oracle's fixed
    point like Algorithm 1's CG steps: free energy, forces and the occupied eigenvalues, on a
    small cell and the 8-atom diamond cell in both precisions, and in FP64 on a 112-band
    subspace of a small cell (its 238 x 238 block, 46 % of the basis, goes to the cluster
    eigensolve; in FP32 that block does not converge, and the mixed path's cluster eigensolve
    of the block is exercised at full size by the 13-atom cluster's ledger instead).  A basis
    smaller than the block (2 n_b above the plane-wave count) is refused."""
    if case == "diamond8":
        st, ref = request.getfixturevalue("diamond_ref")
        mix = dict(mix_alpha=0.7, kerker_q0=0.0)
    else:
        st = _struct(ecut=3.0) if case == "tiny" else _struct(ecut=12.0, nbands=112)
        ref = oracle.scf(st, tol_e=1e-12, tol_rho=1e-10)
        mix = {}
    if precision == "fp64":
        ctx = sgo.Context(st, precision="fp64", scf_tol_e=1e-11, scf_tol_rho=1e-9, max_scf=120,
                          eigensolver="davidson", **mix)
        tol_e, tol_f, tol_eig = (1e-7, 1e-5, 1e-6) if case == "diamond8" else (1e-8, 1e-6, 1e-7)
    else:
        ctx = sgo.Context(st, precision="mixed", scf_tol_e=1e-7 * st.natoms, scf_tol_rho=1e-5, max_scf=120,
                          eigensolver="davidson", **mix)
        tol_e, tol_f, tol_eig = 1e-5, 1e-4, 2e-4
    _compare(st, ctx.energy_forces(), ref, tol_e, tol_f)
    eig, _ = ctx.eigen()
    assert np.abs(eig - ref.eig)[ref.occ > 1e-6].max() < tol_eig
    stats = ctx.stats()
    assert stats["jacobi_cap_hits"] == 0 and stats["eig_resid"] < 1e-4, stats
    if case == "tiny":
        with pytest.raises(sgo.SgoError) as e:
            sgo.Context(_struct(ecut=6.0, nbands=112), precision=precision, eigensolver="davidson")
        assert e.value.status == sgo.SGO_ERR_ARG


def test_davidson_batch_equals_single(sgo):
    """A batch of block-Davidson members gives each member's single-structure FP64 result
    bit for bit; a batch that mixes eigensolvers is refused."""
    sts = [_struct(seed=s, ecut=3.0) for s in (3, 4)]
    opts = dict(precision="fp64", scf_tol_e=1e-10, scf_tol_rho=1e-8, max_scf=100, eigensolver="davidson")
    singles = [sgo.Context(st, **opts).energy_forces() for st in sts]
    E, F, status = sgo.Batch([sgo.Context(st, **opts) for st in sts]).energy_forces()
    assert list(status) == [0, 0]
    for i in range(2):
        assert E[i] == singles[i][0] and np.array_equal(F[i], singles[i][1])
    with pytest.raises(sgo.SgoError) as e:
        sgo.Batch([sgo.Context(sts[0], **opts), sgo.Context(sts[1], precision="fp64")]).energy_forces()
    assert e.value.status == sgo.SGO_ERR_ARG


@pytest.fixture(scope="module")
def pbe_refs():
    """Oracle PBE SCF results of the small cell and the 8-atom diamond cell."""
    tiny = dataclasses.replace(_struct(ecut=3.0), xc="pbe")
    dia = dataclasses.replace(workloads.diamond8(), xc="pbe")
    return {"tiny": (tiny, oracle.scf(tiny, tol_e=1e-12, tol_rho=1e-10)),
            "diamond8": (dia, oracle.scf(dia, mix=0.7, q0=0.0))}


@pytest.mark.parametrize("case", ["tiny", "diamond8"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_scf_pbe(sgo, pbe_refs, precision, case):
    """PBE exchange-correlation (xc = 1; the paper's functional, Sec. III): the potential
    de/drho - div(2 de/dsigma grad rho) with the gradient and divergence in G space on the
    FFT box, and E_xc at rho_out; SCF free energy, forces, occupied eigenvalues and the xc
    term against the oracle's PBE (oracle/gga.py)."""
    st, ref = pbe_refs[case]
    mix = dict(mix_alpha=0.7, kerker_q0=0.0) if case == "diamond8" else {}
    if precision == "fp64":
        ctx = sgo.Context(st, precision="fp64", scf_tol_e=1e-11, scf_tol_rho=1e-9, max_scf=150, **mix)
        tol_e, tol_f, tol_eig = (1e-7, 1e-5, 1e-6) if case == "diamond8" else (1e-8, 1e-6, 1e-7)
    else:
        ctx = sgo.Context(st, precision="mixed", scf_tol_e=1e-7 * st.natoms, scf_tol_rho=1e-5, max_scf=150, **mix)
        tol_e, tol_f, tol_eig = 1e-5, 1e-4, 2e-4
    _compare(st, ctx.energy_forces(), ref, tol_e, tol_f)
    eig, _ = ctx.eigen()
    assert np.abs(eig - ref.eig)[ref.occ > 1e-6].max() < tol_eig
    assert abs(ctx.terms()["xc"] - ref.terms["xc"]) / st.natoms < (1e-7 if precision == "fp64" else 1e-4)


def test_pbe_forces_match_finite_differences_gpu(sgo):
    """FP64 PBE: forces against central differences of the GPU free energy (h = 1e-3 bohr);
    they agree only if the GPU's v_xc is the derivative of its E_xc."""
    st = dataclasses.replace(_struct(ecut=3.0), xc="pbe")
    ctx = sgo.Context(st, precision="fp64", scf_tol_e=1e-12, scf_tol_rho=1e-10, max_scf=150)
    _, F = ctx.energy_forces()
    h = 1e-3
    for I, a in [(0, 0), (1, 1)]:
        p = st.pos.copy()
        p[I, a] += h
        ep, _ = ctx.energy_forces(p)
        p[I, a] -= 2 * h
        em, _ = ctx.energy_forces(p)
        assert abs(-(ep - em) / (2 * h) - F[I, a]) < 2e-5, (I, a)
    with pytest.raises(sgo.SgoError) as e:
        sgo.Batch([ctx, sgo.Context(_struct(ecut=3.0), precision="fp64")])
    assert e.value.status == sgo.SGO_ERR_ARG


def _struct_p(grid=None, ecut=3.0, seed=7):
    """The small cell with a p channel on its species."""
    st = workloads.tiny(nat=2, ecut=ecut, seed=seed, kT=0.01, species=workloads.SPECIES_Z4_P)
    return dataclasses.replace(st, fft=tuple(grid)) if grid is not None else st


@pytest.mark.parametrize("grid", [None, (30, 54, 40), (60, 50, 12)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_apply_hamiltonian_pchannel(sgo, grid, precision):
    """Species with a p channel (three projectors x_m exp(-r^2/(2 rp_p^2)) per atom after the s
    projector): H psi against the oracle's dense H, whose nonlocal part sums the eight
    projectors of the two atoms with their own strengths."""
    st = _struct_p(grid=grid)
    ctx = sgo.Context(st, precision=precision)
    m = dft.Model(st)
    miller = ctx.basis()
    rng = np.random.default_rng(13)
    veff = rng.normal(size=m.grid) * 0.3
    x = rng.normal(size=(st.nbands, ctx.npw))
    y = ctx.apply_hamiltonian(veff, x)
    H = dft.dense_h(m, veff, dft.projectors(m, st.pos))
    y_ref = H @ full_from_packed(m, miller, x)
    tol = 1e-11 if precision == "fp64" else 2e-5
    assert np.abs(full_from_packed(m, miller, y) - y_ref).max() < tol * np.abs(y_ref).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_scf_pchannel(sgo, precision):
    """SCF energy, forces, occupied eigenvalues and the nonlocal term with the p channel against
    the oracle."""
    st = _struct_p()
    ref = oracle.scf(st, tol_e=1e-12, tol_rho=1e-10)
    if precision == "fp64":
        ctx = sgo.Context(st, precision="fp64", scf_tol_e=1e-11, scf_tol_rho=1e-9, max_scf=120)
        tol_e, tol_f, tol_eig, tol_t = 1e-8, 1e-6, 1e-7, 1e-7
    else:
        ctx = sgo.Context(st, precision="mixed", scf_tol_e=1e-7, scf_tol_rho=1e-5, max_scf=120)
        tol_e, tol_f, tol_eig, tol_t = 1e-5, 1e-4, 2e-4, 1e-4
    _compare(st, ctx.energy_forces(), ref, tol_e, tol_f)
    eig, _ = ctx.eigen()
    assert np.abs(eig - ref.eig)[ref.occ > 1e-6].max() < tol_eig
    assert abs(ctx.terms()["nonlocal"] - ref.terms["nonlocal_"]) / st.natoms < tol_t


def test_pchannel_forces_and_mixed_batch(sgo):
    """FP64 with the p channel: forces against central differences of the GPU free energy, and
    a batch of a p-channel member and an s-only member gives each one's single result bit for
    bit (members with different projector counts share every launch)."""
    st = _struct_p()
    opts = dict(precision="fp64", scf_tol_e=1e-12, scf_tol_rho=1e-10, max_scf=150)
    ctx = sgo.Context(st, **opts)
    E0, F = ctx.energy_forces()
    h = 1e-3
    for I, a in [(0, 2), (1, 0)]:
        p = st.pos.copy()
        p[I, a] += h
        ep, _ = ctx.energy_forces(p)
        p[I, a] -= 2 * h
        em, _ = ctx.energy_forces(p)
        assert abs(-(ep - em) / (2 * h) - F[I, a]) < 2e-5, (I, a)
    sts = [_struct_p(seed=3), _struct(seed=4, ecut=3.0)]
    singles = [sgo.Context(t, **opts).energy_forces() for t in sts]
    E, Fb, status = sgo.Batch([sgo.Context(t, **opts) for t in sts]).energy_forces()
    assert list(status) == [0, 0]
    for i in range(2):
        assert E[i] == singles[i][0] and np.array_equal(Fb[i], singles[i][1])


def _struct_k(kgrid, pchan=False, seed=7):
    """The small cell on a k mesh (12^3 box: the off-centre spheres of the mesh points reach
    further than the Gamma sphere), nine bands per k point."""
    st = workloads.tiny(nat=2, ecut=3.0, seed=seed, kT=0.01, nbands=9,
                        species=workloads.SPECIES_Z4_P if pchan else None)
    return dataclasses.replace(st, fft=(12, 12, 12), kgrid=tuple(kgrid))


@pytest.mark.parametrize("kgrid,pchan", [((2, 1, 1), True), ((1, 2, 2), False), ((2, 2, 2), False)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_kpoint_mesh_matches_oracle(sgo, kgrid, pchan, precision):
    """A Gamma-centred k mesh (sgo_opts.kgrid, computed by zone folding on the supercell)
    against the oracle's Bloch-sum SCF over the mesh (oracle/kpoints.py: complex psi_k on
    each k + G sphere, one Fermi level over the mesh): free energy per cell, the forces on the
    cell's atoms, the occupied band energies of the whole mesh and the energy terms."""
    st = _struct_k(kgrid, pchan)
    ref = kpoints.scf(st, tol_e=1e-12, tol_rho=1e-10)
    if precision == "fp64":
        ctx = sgo.Context(st, precision="fp64", scf_tol_e=1e-11, scf_tol_rho=1e-9, max_scf=150)
        tol_e, tol_f, tol_eig = 1e-8, 1e-6, 1e-7
    else:
        ctx = sgo.Context(st, precision="mixed", scf_tol_e=1e-7 * st.natoms, scf_tol_rho=1e-5, max_scf=150)
        tol_e, tol_f, tol_eig = 1e-5, 1e-4, 2e-4
    nk = int(np.prod(kgrid))
    assert ctx.natoms == st.natoms and ctx.nbands == nk * st.nbands
    _compare(st, ctx.energy_forces(), ref, tol_e, tol_f)
    eig, occ = ctx.eigen()
    from tests.test_gpu_fullsize import mesh_common_spectrum
    e_ref, e_gpu = mesh_common_spectrum(ref.eig, ref.occ, eig)
    assert len(e_ref) >= nk * (st.nelec / 2 - 1) and np.abs(e_gpu - e_ref).max() < tol_eig
    t = ctx.terms()
    for k_gpu, k_ref in [("kinetic", "kinetic"), ("nonlocal", "nonlocal_"), ("hartree", "hartree"), ("xc", "xc"),
                         ("ewald", "ewald")]:
        assert abs(t[k_gpu] - ref.terms[k_ref]) / st.natoms < 10 * tol_e, k_gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_kpoint_mesh_pbe(sgo, precision):
    """A 2 x 1 x 1 mesh with PBE exchange-correlation against the oracle's Bloch-sum PBE SCF:
    free energy per cell, forces and the xc term."""
    st = dataclasses.replace(_struct_k((2, 1, 1)), xc="pbe")
    ref = kpoints.scf(st, tol_e=1e-12, tol_rho=1e-10)
    if precision == "fp64":
        ctx = sgo.Context(st, precision="fp64", scf_tol_e=1e-11, scf_tol_rho=1e-9, max_scf=150)
        tol_e, tol_f = 1e-8, 1e-6
    else:
        ctx = sgo.Context(st, precision="mixed", scf_tol_e=1e-7 * st.natoms, scf_tol_rho=1e-5, max_scf=150)
        tol_e, tol_f = 1e-5, 1e-4
    _compare(st, ctx.energy_forces(), ref, tol_e, tol_f)
    assert abs(ctx.terms()["xc"] - ref.terms["xc"]) / st.natoms < 10 * tol_e


def test_kpoint_members_in_a_batch(sgo):
    """FP64: k-mesh members (different meshes) and a Gamma member in one batch give each
    one's single result bit for bit; the device-array batch call refuses k-mesh members;
    forces of a k-mesh context against central differences of its free energy."""
    opts = dict(precision="fp64", scf_tol_e=1e-12, scf_tol_rho=1e-10, max_scf=150)
    sts = [_struct_k((2, 1, 1), seed=3), _struct_k((1, 1, 2), pchan=True, seed=4), _struct(seed=5, ecut=3.0)]
    singles = [sgo.Context(t, **opts).energy_forces() for t in sts]
    ctxs = [sgo.Context(t, **opts) for t in sts]
    b = sgo.Batch(ctxs)
    E, Fb, status = b.energy_forces()
    assert list(status) == [0, 0, 0]
    for i in range(3):
        assert E[i] == singles[i][0] and np.array_equal(Fb[i], singles[i][1])
    import torch
    n3 = sum(c.natoms for c in ctxs) * 3
    pos = torch.tensor(np.concatenate([t.pos.reshape(-1) for t in sts]), dtype=torch.float64, device="cuda")
    e_d = torch.zeros(3, dtype=torch.float64, device="cuda")
    f_d = torch.zeros(n3, dtype=torch.float64, device="cuda")
    s_d = torch.zeros(3, dtype=torch.int32, device="cuda")
    with pytest.raises(sgo.SgoError):
        b.energy_forces_device(pos.data_ptr(), e_d.data_ptr(), f_d.data_ptr(), s_d.data_ptr())
    st = sts[0]
    ctx = ctxs[0]
    E0, F = ctx.energy_forces()
    h = 1e-3
    for I, a in [(0, 1), (1, 2)]:
        p = st.pos.copy()
        p[I, a] += h
        ep, _ = ctx.energy_forces(p)
        p[I, a] -= 2 * h
        em, _ = ctx.energy_forces(p)
        assert abs(-(ep - em) / (2 * h) - F[I, a]) < 2e-5, (I, a)


def test_scf_tiny_mixed(sgo):
    st = _struct(ecut=3.0)
    ref = oracle.scf(st, tol_e=1e-12, tol_rho=1e-10)
    ctx = sgo.Context(st, precision="mixed", scf_tol_e=1e-7, scf_tol_rho=1e-5, max_scf=120)
    _compare(st, ctx.energy_forces(), ref, 1e-5, 1e-4)


@pytest.fixture(scope="module")
def diamond_ref():
    st = workloads.diamond8()
    return st, oracle.scf(st, mix=0.7, q0=0.0)


def test_diamond8_fp64(sgo, diamond_ref):
    """8-atom diamond cell, Ecut 10 Ha, 32^3, 20 bands, integer occupations (FP64)."""
    st, ref = diamond_ref
    ctx = sgo.Context(st, precision="fp64", mix_alpha=0.7, kerker_q0=0.0)
    _compare(st, ctx.energy_forces(), ref, 1e-7, 1e-5)
    eig, _ = ctx.eigen()
    assert np.abs(eig[:16] - ref.eig[:16]).max() < 1e-6


def test_diamond8_mixed(sgo, diamond_ref):
    st, ref = diamond_ref
    ctx = sgo.Context(st, precision="mixed", mix_alpha=0.7, kerker_q0=0.0, scf_tol_e=1e-6, scf_tol_rho=1e-5)
    _compare(st, ctx.energy_forces(), ref, 1e-5, 1e-4)


def test_batch_equals_single_fp64(sgo):
    """Every batch member's FP64 result equals its own single-structure run bit for bit."""
    sts = [_struct(seed=s, ecut=3.0) for s in (3, 4, 9)]
    sts[1] = _struct(seed=4, ecut=3.5, nat=3, grid=(16, 18, 20))
    opts = dict(precision="fp64", scf_tol_e=1e-10, scf_tol_rho=1e-8, max_scf=100)
    singles = []
    for st in sts:
        singles.append(sgo.Context(st, **opts).energy_forces())
    ctxs = [sgo.Context(st, **opts) for st in sts]
    E, F, status = sgo.Batch(ctxs).energy_forces()
    assert list(status) == [0, 0, 0]
    for i in range(3):
        assert E[i] == singles[i][0]
        assert np.array_equal(F[i], singles[i][1])
    # order of members does not change results
    E2, F2, _ = sgo.Batch([sgo.Context(st, **opts) for st in sts[::-1]]).energy_forces()
    assert np.array_equal(E2[::-1], E)


def test_geometry_error_is_reported(sgo):
    st = _struct()
    ctx = sgo.Context(st, precision="fp64")
    bad = st.pos.copy()
    bad[1] = bad[0] + np.array([0.1, 0.0, 0.0])
    with pytest.raises(sgo.SgoError) as e:
        ctx.energy_forces(bad)
    assert e.value.status == sgo.SGO_ERR_GEOMETRY
    bad[0, 0] = np.nan
    with pytest.raises(sgo.SgoError):
        ctx.energy_forces(bad)
    # the context stays usable
    F, _ = ctx.energy_forces(st.pos)
    assert math.isfinite(F)


def test_not_converged_status(sgo):
    st = _struct()
    ctx = sgo.Context(st, precision="fp64", max_scf=2, n_nonscf=0)
    with pytest.raises(sgo.SgoError) as e:
        ctx.energy_forces()
    assert e.value.status == sgo.SGO_ERR_NOT_CONVERGED


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_state_moves_between_contexts(sgo, precision):
    """sgo_get_state / sgo_set_state (Sec. II C: a relaxation step restarts from the previous
    density and wavefunctions): a fresh context given a converged donor's state starts warm
    and reproduces the donor's result within a few SCF iterations."""
    st = workloads.de_candidate(47)
    opts = dict(precision=precision, scf_tol_e=1e-8, scf_tol_rho=1e-7) if precision == "fp64" else \
        dict(precision=precision, scf_tol_e=1e-7 * st.natoms, scf_tol_rho=1e-5)
    fresh = sgo.Context(st, **opts)
    with pytest.raises(sgo.SgoError) as e:
        fresh.get_state()
    assert e.value.status == sgo.SGO_ERR_ARG
    donor = sgo.Context(st, **opts)
    E0, F0 = donor.energy_forces()
    n0 = donor.stats()["n_iter"]
    rho, psi = donor.get_state()
    assert rho.shape == tuple(donor.grid) and psi.shape == (st.nbands, donor.npw)
    # rho_in(G) of a real density: rho(-G) = rho(G)^*, and rho(0) N = N_el / Omega
    assert abs(rho[0, 0, 0].real * abs(np.linalg.det(st.cell)) - st.nelec) < 1e-6 * st.nelec
    assert np.allclose(rho[0, 0, 1], np.conj(rho[0, 0, -1]), atol=1e-12)
    fresh.set_state(rho, psi)
    E1, F1 = fresh.energy_forces()
    s1 = fresh.stats()
    assert s1["warm"] and s1["n_iter"] <= 3 < n0, (s1, n0)
    tol_e = 1e-7 if precision == "fp64" else 2e-6
    assert abs(E1 - E0) / st.natoms < tol_e
    assert np.abs(F1 - F0).max() < (1e-5 if precision == "fp64" else 1e-4)
    with pytest.raises(sgo.SgoError):
        fresh.set_state(rho, np.full_like(psi, np.nan))


def test_watchdog_expiry_is_reported(sgo):
    """Every device wait of the tensor-core kernels is bounded by watchdog_ms; a bound far
    below the time a TMA load takes makes the waits give up.  The kernels drain their own
    copies and MMAs (under a separate fixed bound), free their TMEM and return; the member
    reports SGO_ERR_TIMEOUT, and the process's contexts stay usable."""
    st = _struct(ecut=3.0)
    ctx = sgo.Context(st, precision="mixed", watchdog_ms=1e-6, scf_tol_e=1e-7, scf_tol_rho=1e-5)
    with pytest.raises(sgo.SgoError) as e:
        ctx.energy_forces()
    assert e.value.status == sgo.SGO_ERR_TIMEOUT
    ok = sgo.Context(st, precision="mixed", scf_tol_e=1e-7, scf_tol_rho=1e-5)
    F, f = ok.energy_forces()
    assert math.isfinite(F) and np.all(np.isfinite(f))


def test_torch_allocator_hook(sgo):
    """sgo_set_allocator: with PyTorch's caching allocator installed, every device buffer of a
    context and of its evaluation comes from torch's pool (torch.cuda.memory_allocated() rises
    while the context lives and falls back to where it was when it is destroyed), and the
    results equal those of a context on cudaMalloc memory."""
    import gc

    import torch
    st = _struct()
    tol = {"fp64": dict(scf_tol_e=1e-8, scf_tol_rho=1e-7), "mixed": dict(scf_tol_e=1e-7, scf_tol_rho=1e-5)}
    ref = {p: sgo.Context(st, precision=p, **tol[p]).energy_forces() for p in ("fp64", "mixed")}
    torch.cuda.synchronize()
    gc.collect()
    base = torch.cuda.memory_allocated()
    sgo.use_torch_allocator()
    try:
        ctxs = [sgo.Context(st, precision=p, **tol[p]) for p in ("fp64", "mixed")]
        held = torch.cuda.memory_allocated() - base
        assert held > 0
        for c, p in zip(ctxs, ("fp64", "mixed")):
            E, F = c.energy_forces()
            assert abs(E - ref[p][0]) < 1e-10 and np.abs(F - ref[p][1]).max() < 1e-9, p
        E, F, status = sgo.Batch(ctxs[:1]).energy_forces()
        assert np.all(status == 0)
        gc.collect()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() - base >= held
        del ctxs, c, E, F, status
        gc.collect()
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == base
    finally:
        sgo.use_default_allocator()
    # contexts made afterwards are on cudaMalloc again
    c = sgo.Context(st, precision="fp64", **tol["fp64"])
    assert torch.cuda.memory_allocated() == base
    assert abs(c.energy_forces()[0] - ref["fp64"][0]) < 1e-10


def test_autograd_adjoint(sgo):
    import torch
    st = _struct(ecut=3.0)
    ctx = sgo.Context(st, precision="fp64", scf_tol_e=1e-11, scf_tol_rho=1e-9)
    pos = torch.tensor(st.pos, dtype=torch.float64, requires_grad=True)
    E = sgo.SgoEnergy.apply(ctx, pos)
    E.backward()
    _, F = ctx.energy_forces(st.pos)
    assert torch.allclose(pos.grad, torch.as_tensor(-F), atol=1e-12)


def test_relaxation_through_autograd_matches_batch_driver(sgo):
    """The relaxation driven by SgoEnergy (energy forward, force adjoint backward) asks for
    the same positions as the batched driver loop (sgo_relax_batch) on the FP64 path."""
    st = _struct(ecut=3.0, nat=3, seed=5)
    opts = dict(precision="fp64", scf_tol_e=1e-10, scf_tol_rho=1e-8, max_scf=120)
    d1 = sgo.Relax(st.cell, st.pos, method="pcg", fmax=1e-3, max_evals=12)
    state1, n1 = sgo.relax_autograd(sgo.Context(st, **opts), d1, max_evals=12)
    d2 = sgo.Relax(st.cell, st.pos, method="pcg", fmax=1e-3, max_evals=12)
    rounds, status = sgo.Batch([sgo.Context(st, **opts)]).relax([d2], max_rounds=12)
    assert status[0] == 0
    assert d1.info() == d2.info()
    assert np.abs(d1.positions() - d2.positions()).max() < 1e-9
    e1, x1 = d1.best()
    e2, x2 = d2.best()
    assert abs(e1 - e2) < 1e-9 and np.abs(x1 - x2).max() < 1e-9


def test_forces_match_finite_differences_gpu(sgo):
    """FP64 path: F = -dF/dR by central differences (h = 1e-3 bohr)."""
    st = _struct(ecut=3.0)
    opts = dict(precision="fp64", scf_tol_e=1e-12, scf_tol_rho=1e-10, max_scf=150)
    ctx = sgo.Context(st, **opts)
    _, F = ctx.energy_forces()
    h = 1e-3
    for I, a in [(0, 0), (1, 2)]:
        p = st.pos.copy(); p[I, a] += h
        ep, _ = ctx.energy_forces(p)
        p[I, a] -= 2 * h
        em, _ = ctx.energy_forces(p)
        assert abs(-(ep - em) / (2 * h) - F[I, a]) < 2e-6


@pytest.mark.parametrize("precision,tc,tol", [("fp64", 0, 1e-13), ("mixed", 1, 2e-6), ("mixed", 0, 2e-6)])
def test_subspace_matrix_gemm(sgo, precision, tc, tol):
    """C = X^T Y through the subspace GEMM (tcgen05 3xTF32 on the mixed path with gemm_tc=1)
    vs NumPy FP64, relative to |x_i||y_j|; single-chunk and multi-chunk K."""
    for st in (workloads.tiny(nat=2, ecut=3.5), workloads.de_candidate(0)):
        ctx = sgo.Context(st, precision=precision, gemm_tc=tc)
        rng = np.random.default_rng(8)
        n = st.nbands
        x = rng.normal(size=(n, ctx.npw))
        y = rng.normal(size=(n, ctx.npw))
        c = ctx.subspace_matrix(x, y)
        ref = x @ y.T
        scale = np.sqrt((x ** 2).sum(1))[:, None] * np.sqrt((y ** 2).sum(1))[None, :]
        assert np.abs(c - ref).max() <= tol * scale.max(), (st.name, np.abs(c - ref).max() / scale.max())


@pytest.mark.parametrize("precision,tc,tol", [("fp64", 0, 1e-13), ("mixed", 1, 2e-6), ("mixed", 0, 2e-6)])
def test_block_update_gemm(sgo, precision, tc, tol):
    """Y <- alpha M^T X + beta Y through the block-update GEMM (tcgen05 3xTF32 on the mixed
    path with gemm_tc=1) vs NumPy FP64, relative to sum_i |m_ij| |x_i| + |beta| |y_j|;
    a rotation (beta = 0) and a projection update (alpha = -1, beta = 1), all and part
    of the bands."""
    for st in (workloads.tiny(nat=2, ecut=3.5), workloads.de_candidate(0)):
        ctx = sgo.Context(st, precision=precision, gemm_tc=tc)
        rng = np.random.default_rng(9)
        for n in (st.nbands, max(1, st.nbands - 5)):
            x = rng.normal(size=(n, ctx.npw))
            y = rng.normal(size=(n, ctx.npw))
            m = rng.normal(size=(n, n))
            for alpha, beta in ((1.0, 0.0), (-1.0, 1.0)):
                out = ctx.block_update(x, m, alpha, beta, y)
                ref = alpha * (m.T @ x) + beta * y
                scale = abs(alpha) * (np.abs(m).T @ np.abs(x)) + abs(beta) * np.abs(y)
                err = np.abs(out - ref) / scale
                assert err.max() <= tol, (st.name, n, alpha, beta, err.max())


def test_overlap_gemm_bias(sgo):
    """Why the overlap S = X^T X stays on CUDA cores in the mixed path: its diagonal sums
    positive terms, which the FP32 CUDA-core GEMM leaves unbiased, while the tensor-core
    3xTF32 path (K chunks of 512 accumulated in TMEM) comes out low by a few 1e-6 relative.
    The overlap sets the band norms and hence rho and F."""
    st = workloads.de_candidate(0)
    rng = np.random.default_rng(3)
    bias = {}
    for tc in (0, 1):
        ctx = sgo.Context(st, precision="mixed", gemm_tc=tc)
        x = rng.normal(size=(st.nbands, ctx.npw))
        x /= np.linalg.norm(x, axis=1, keepdims=True)
        bias[tc] = float(np.mean(np.diag(ctx.subspace_matrix(x, x)) - 1.0))
    assert abs(bias[0]) < 5e-8, bias
    assert abs(bias[1]) < 2e-5, bias


def test_graph_loop_equals_host_loop(sgo):
    """The SCF loop driven by captured CUDA graphs (a conditional WHILE node ended on the
    device) gives bit-identical results to the host-driven loop, for both precisions and a
    batch whose members converge at different iterations."""
    sts = [_struct(seed=s, ecut=3.0) for s in (3, 4, 9)]
    sts[1] = _struct(seed=4, ecut=3.5, nat=3, grid=(16, 18, 20))
    for prec, tol in (("fp64", dict(scf_tol_e=1e-10, scf_tol_rho=1e-8)), ("mixed", dict(scf_tol_e=1e-7, scf_tol_rho=1e-5))):
        res = {}
        for graph in (0, 1):
            ctxs = [sgo.Context(st, precision=prec, graph=graph, autotune=0, max_scf=100, **tol) for st in sts]
            b = sgo.Batch(ctxs)
            E, F, status = b.energy_forces()
            E2, F2, status2 = b.energy_forces()  # second call replays the cached graphs
            assert list(status) == [0, 0, 0] and list(status2) == [0, 0, 0]
            assert np.array_equal(E, E2)
            res[graph] = (E, F, [c.stats() for c in ctxs])
        assert np.array_equal(res[0][0], res[1][0]), prec
        for i in range(3):
            assert np.array_equal(res[0][1][i], res[1][1][i]), prec
        assert res[0][2] == res[1][2], prec


@pytest.mark.parametrize("grid", [(45, 40, 48), (100, 108, 10)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_grid_fft_matches_fp64_fft(sgo, grid, precision):
    """The SCF's grid transform (the potential's inverse and the output density's forward
    FFT) against numpy's FP64 FFT, both signs: FP64 on the plain path, float-float
    arithmetic on the mixed path, so both stay within 1e-12 of the largest output (an FP32
    transform would sit near 1e-7).  (100, 108) planes take the line-block kernels."""
    ctx = sgo.Context(_struct(grid=grid, ecut=3.0), precision=precision)
    rng = np.random.default_rng(5)
    x = rng.normal(size=grid) + 1j * rng.normal(size=grid)
    for sign in (-1, 1):
        got = ctx.grid_fft(x, sign)
        ref = np.fft.fftn(x) if sign < 0 else np.fft.ifftn(x) * x.size
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < 1e-12, (sign, err)


def test_sub_batches_equal_one_batch(sgo):
    """Splitting a batch into sub-batches (each on its own graphs and stream, overlapping on
    the GPU) leaves every member's energy, forces and iteration count bit-identical, through
    both the host-pointer and the device-pointer entry points (whose outputs are indexed by
    the member's place in the whole batch)."""
    import torch
    sts = [_struct(seed=s, ecut=3.0) for s in (3, 4, 9, 5, 6)]
    sts[1] = _struct(seed=4, ecut=3.5, nat=3, grid=(16, 18, 20))
    for prec, tol in (("fp64", dict(scf_tol_e=1e-10, scf_tol_rho=1e-8)), ("mixed", dict(scf_tol_e=1e-7, scf_tol_rho=1e-5))):
        res = {}
        for k in (1, 2, 3):
            ctxs = [sgo.Context(st, precision=prec, autotune=0, sub_batches=k, max_scf=100, **tol) for st in sts]
            b = sgo.Batch(ctxs)
            E, F, status = b.energy_forces()
            assert list(status) == [0] * len(sts), (prec, k)
            pos = torch.tensor(np.concatenate([st.pos.reshape(-1) for st in sts]), device="cuda")
            e_dev = torch.zeros(len(sts), dtype=torch.float64, device="cuda")
            f_dev = torch.zeros_like(pos)
            s_dev = torch.full((len(sts),), -1, dtype=torch.int32, device="cuda")
            b.energy_forces_device(pos.data_ptr(), e_dev.data_ptr(), f_dev.data_ptr(), s_dev.data_ptr())
            torch.cuda.synchronize()
            assert s_dev.tolist() == [0] * len(sts), (prec, k)
            assert np.array_equal(e_dev.cpu().numpy(), E), (prec, k)
            assert np.array_equal(f_dev.cpu().numpy(), np.concatenate([f.reshape(-1) for f in F])), (prec, k)
            res[k] = (E, F, [c.stats() for c in ctxs])
        for k in (2, 3):
            assert np.array_equal(res[1][0], res[k][0]), (prec, k)
            for i in range(len(sts)):
                assert np.array_equal(res[1][1][i], res[k][1][i]), (prec, k, i)
            assert res[1][2] == res[k][2], (prec, k)


def test_relax_batch_reaches_the_oracle_minimum(sgo):
    """Local relaxation (Sec. II C) of a small batch through sgo_relax_batch (PCG driver,
    warm-started batched evaluations) ends where the oracle's PCG relaxation on the oracle
    DFT ends: both converge to |F| < 1e-3 Ha/bohr, at geometries within 5e-3 bohr (after
    removing the centroid) and energies within 1e-5 Ha/atom."""
    from oracle import dft
    from oracle import relax as rx
    sts = [workloads.tiny(nat=2, ecut=3.0, seed=7, kT=0.01), _struct(seed=3, ecut=3.0, nat=3)]
    fmax = 1e-3
    import bench
    ctxs = [sgo.Context(st, precision="mixed", **bench._tols("mixed", st)) for st in sts]
    b = sgo.Batch(ctxs)
    drivers = [sgo.Relax(st.cell, st.pos, method="pcg", fmax=fmax, max_evals=60) for st in sts]
    rounds, status = b.relax(drivers, max_rounds=80)
    assert list(status) == [0] * len(sts)
    E, F, st_ = b.energy_forces([d.positions() for d in drivers])
    for i, st in enumerate(sts):
        assert drivers[i].info()["state"] == 1, i
        assert np.linalg.norm(F[i], axis=1).max() < fmax
        tr = rx.relax(lambda p, st=st: dft.evaluate(st, pos=p), st.cell, st.pos, method="pcg", fmax=fmax,
                      max_evals=60)
        assert tr.converged, i
        a = drivers[i].positions() - drivers[i].positions().mean(axis=0)
        o = tr.final - tr.final.mean(axis=0)
        assert np.abs(a - o).max() < 5e-3, (i, np.abs(a - o).max())
        assert abs(E[i] - tr.energies[-1]) / st.natoms < 1e-5, i


def test_relaxation_on_a_k_mesh(sgo):
    """The batched PCG relaxation (sgo_relax_batch) of a cell on a 2 x 1 x 1 k mesh: the driver
    sees the cell's atoms (the folded supercell stays inside the library) and stops with
    |F| < 1e-3 Ha/bohr; the oracle's Bloch-sum SCF at the final geometry agrees that the forces
    vanish there (below 1e-3 plus the mixed path's force tolerance, 1e-4)."""
    import bench
    st = _struct_k((2, 1, 1))
    fmax = 1e-3
    ctx = sgo.Context(st, precision="mixed", **bench._tols("mixed", st))
    b = sgo.Batch([ctx])
    drv = sgo.Relax(st.cell, st.pos, method="pcg", fmax=fmax, max_evals=60)
    rounds, status = b.relax([drv], max_rounds=80)
    assert list(status) == [0] and drv.info()["state"] == 1
    E, F, _ = b.energy_forces([drv.positions()])
    assert F[0].shape == (st.natoms, 3) and np.linalg.norm(F[0], axis=1).max() < fmax
    ref = kpoints.scf(st, pos=drv.positions(), tol_e=1e-11, tol_rho=1e-9)
    assert np.abs(ref.forces).max() < fmax + 1e-4
    assert abs(E[0] - ref.free_energy) / st.natoms < 1e-5


def test_de_generation_matches_the_oracle(sgo):
    """One DE generation (Sec. II B) of four 3-atom individuals through sgo_de_generation
    (offspring from given random numbers, PCG relaxation of each child on the batch, greedy
    selection) against the same generation built from the oracle's operators, relaxation
    and DFT: each child's best relaxed energy agrees to 5e-5 Ha/atom and the selection
    agrees wherever the child and parent energies differ by more than that."""
    import bench
    from oracle import de
    from oracle import relax as rx
    base = _struct(seed=3, ecut=3.0, nat=3)
    rng = np.random.default_rng(9)
    inv = np.linalg.inv(base.cell)
    pop = []
    while len(pop) < 4:
        x = rng.uniform(size=(3, 3)) @ base.cell
        d = [np.linalg.norm(de._mi((x[j] - x[i]) @ inv) @ base.cell) for i in range(3) for j in range(i + 1, 3)]
        if min(d) > 2.2:
            pop.append(x)
    pop = np.array(pop)
    f = np.array([dft.evaluate(base, pos=x)[0] for x in pop])
    u = rng.uniform(size=(4, de.RANDOMS))
    species = np.zeros(3, np.int32)
    ctxs = [sgo.Context(dataclasses.replace(base, pos=x), precision="mixed", **bench._tols("mixed", base))
            for x in pop]
    b = sgo.Batch(ctxs)
    pop2, f2, rep, cf = b.de_generation(base.cell, species, pop, f, u, max_rounds=60, fmax=1e-3, max_evals=60)
    kids = de.offspring(base.cell, species, pop, f, u)
    for i in range(4):
        tr = rx.relax(lambda p: dft.evaluate(base, pos=p), base.cell, kids[i], method="pcg", fmax=1e-3,
                      max_evals=60)
        e_ref = min(tr.energies)
        assert abs(cf[i] - e_ref) / 3 < 5e-5, (i, cf[i], e_ref)
        if abs(e_ref - f[i]) / 3 > 5e-5:
            assert rep[i] == (e_ref < f[i]), i
        assert f2[i] <= f[i]


def test_autotuned_batch(sgo):
    """The autotuner keeps one of its candidates for each knob, and the tuned batch's
    energies and forces agree with the default-knob batch to the mixed tolerances (the knobs
    change only the split-K summation order)."""
    sts = [workloads.de_candidate(i) for i in (0, 5)]
    import bench
    res = {}
    for tune in (0, 1):
        ctxs = [sgo.Context(st, precision="mixed", autotune=tune, **bench._tols("mixed", st)) for st in sts]
        b = sgo.Batch(ctxs)
        E, F, status = b.energy_forces()
        assert list(status) == [0, 0]
        res[tune] = (E, F, b.tuning())
    k = res[1][2]
    assert k["tn_tc_k_chunk"] in (256, 512, 1024, 2048)
    assert k["nn_tc_tiles_per_cta"] in (2, 4, 8, 16)
    assert k["tn_simt_k_chunk"] in (128, 256, 512)
    assert res[0][2] == dict(tn_tc_k_chunk=512, nn_tc_tiles_per_cta=4, tn_simt_k_chunk=256)
    for i, st in enumerate(sts):
        assert abs(res[0][0][i] - res[1][0][i]) / st.natoms < 2e-6
        assert np.abs(res[0][1][i] - res[1][1][i]).max() < 5e-5
