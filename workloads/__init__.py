"""Seeded synthetic structures shaped like the paper's DFT workloads.

The paper (Sec. III A, Table 1) searches crystals of 8-10 atoms, 2D monolayers of
8-12 atoms and Pt clusters of 10-23 atoms in a large vacuum box, with a DE
population of 8 (Sec. II D, last paragraph).  Its real pseudopotentials and
structures are not available, so every structure here is synthetic and seeded.

This module is shared by the CPU oracle and the CUDA path.  It only builds
inputs -- cells, species parameters, atom positions, cutoffs, band counts and
FFT grid sizes -- and holds none of the method's arithmetic (no basis, no
Hamiltonian, no energy).  Generated structures are deterministic functions of
their seed.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

# ---------------------------------------------------------------------------
# Synthetic analytic pseudopotential parameter sets ("ppv1").
#   local:  v(r) = -Z erf(r/rc)/r + a_sr exp(-r^2/sigma_sr^2)
#   KB s-projector: beta(r) = N exp(-r^2/(2 rp^2)), <beta|beta> = 1, strength d_nl
# The paper uses real norm-conserving / ultrasoft PBE potentials (Sec. II D);
# these invented parameters stand in for them and are frozen.
# ---------------------------------------------------------------------------
SPECIES_Z4 = dict(z_val=4.0, rc=1.0, a_sr=0.5, sigma_sr=0.8, rp=0.9, d_nl=1.0)
SPECIES_Z10 = dict(z_val=10.0, rc=1.2, a_sr=0.5, sigma_sr=1.0, rp=1.1, d_nl=0.8)

SPECIES_KEYS = ("z_val", "rc", "a_sr", "sigma_sr", "rp", "d_nl")
# optional p channel of the nonlocal part: beta_m(r) = N_p x_m exp(-r^2/(2 rp_p^2)), strength d_p
SPECIES_P_KEYS = ("rp_p", "d_p")
SPECIES_Z4_P = dict(SPECIES_Z4, rp_p=1.0, d_p=0.6)


@dataclasses.dataclass
class Structure:
    """One evaluation input: cell rows a_i (bohr), species table, atoms, cutoffs."""

    name: str
    cell: np.ndarray            # (3,3), rows are lattice vectors, bohr
    species: List[dict]         # parameter dicts (SPECIES_KEYS)
    species_of_atom: np.ndarray  # (n,) int
    pos: np.ndarray             # (n,3) Cartesian bohr
    ecut: float                 # plane-wave cutoff, Ha (|G|^2/2 <= ecut)
    nbands: int
    fft: tuple                  # (N1, N2, N3)
    kT: float = 0.0             # Fermi-Dirac smearing, Ha; 0 = integer occupations
    xc: str = "lda"             # exchange-correlation: "lda" (PZ81) or "pbe"
    kgrid: tuple = (1, 1, 1)    # Gamma-centred k mesh n1 x n2 x n3; (1, 1, 1) = the Gamma point

    @property
    def natoms(self) -> int:
        return int(self.pos.shape[0])

    @property
    def nelec(self) -> float:
        return float(sum(self.species[s]["z_val"] for s in self.species_of_atom))

    def with_positions(self, pos) -> "Structure":
        return dataclasses.replace(self, pos=np.array(pos, dtype=np.float64).reshape(-1, 3))

    def species_array(self) -> np.ndarray:
        """(nspecies, 6) float64 table in SPECIES_KEYS order (the C-ABI layout)."""
        return np.array([[sp[k] for k in SPECIES_KEYS] for sp in self.species], dtype=np.float64)

    def to_json(self) -> dict:
        return dict(name=self.name, cell=self.cell.tolist(), species=self.species,
                    species_of_atom=self.species_of_atom.tolist(), pos=self.pos.tolist(),
                    ecut=self.ecut, nbands=self.nbands, fft=list(self.fft), kT=self.kT)

    @staticmethod
    def from_json(d: dict) -> "Structure":
        return Structure(name=d["name"], cell=np.array(d["cell"], dtype=np.float64),
                         species=list(d["species"]),
                         species_of_atom=np.array(d["species_of_atom"], dtype=np.int32),
                         pos=np.array(d["pos"], dtype=np.float64), ecut=float(d["ecut"]),
                         nbands=int(d["nbands"]), fft=tuple(int(x) for x in d["fft"]),
                         kT=float(d["kT"]))


# ---------------------------------------------------------------------------
# FFT grid sizes.  |m_i| = |a_i . G| / 2pi <= |a_i| sqrt(2 Ecut) / 2pi bounds the
# Miller index along axis i; N_i >= 4 m_i + 1 keeps |psi|^2 and V*psi alias-free.
# ---------------------------------------------------------------------------
def _is_smooth(n: int) -> bool:
    for p in (2, 3, 5):
        while n % p == 0:
            n //= p
    return n == 1


def good_fft_size(nmin: int) -> int:
    n = max(int(nmin), 1)
    while not _is_smooth(n):
        n += 1
    return n


def miller_bound(cell, ecut: float) -> np.ndarray:
    cell = np.asarray(cell, dtype=np.float64)
    return np.floor(np.linalg.norm(cell, axis=1) * math.sqrt(2.0 * ecut) / (2.0 * math.pi)).astype(int)


def fft_grid(cell, ecut: float) -> tuple:
    return tuple(good_fft_size(4 * int(m) + 1) for m in miller_bound(cell, ecut))


# ---------------------------------------------------------------------------
# Geometry helpers (input validity only).
# ---------------------------------------------------------------------------
def min_image_distances(cell, pos) -> np.ndarray:
    """All pairwise minimum-image distances (n,n); diagonal = +inf."""
    cell = np.asarray(cell, dtype=np.float64)
    pos = np.asarray(pos, dtype=np.float64)
    n = pos.shape[0]
    inv = np.linalg.inv(cell)
    d = np.full((n, n), np.inf)
    shifts = np.array([[i, j, k] for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)],
                      dtype=np.float64) @ cell
    for a in range(n):
        for b in range(n):
            if a == b:
                continue
            df = (pos[a] - pos[b]) @ inv
            df -= np.round(df)
            v = df @ cell
            d[a, b] = np.min(np.linalg.norm(v[None, :] + shifts, axis=1))
    return d


def _random_cluster(rng, n, dmin, box):
    """Random sequential insertion in a sphere centred in a cubic box (configs 3 and 5)."""
    radius = 0.5 * dmin * (n / 0.35) ** (1.0 / 3.0)
    pts: List[np.ndarray] = []
    fails = 0
    centre = np.full(3, 0.5 * box)
    while len(pts) < n:
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        p = centre + u * radius * rng.uniform() ** (1.0 / 3.0)
        if all(np.linalg.norm(p - q) >= dmin for q in pts):
            pts.append(p)
            fails = 0
        else:
            fails += 1
            if fails >= 10000:
                radius *= 1.05
                fails = 0
    return np.array(pts)


# ---------------------------------------------------------------------------
# The five workload shapes.
# ---------------------------------------------------------------------------
def diamond8(jitter: float = 0.05, seed: int = 1001) -> Structure:
    """8-atom diamond-cubic cell, a = 10.26 bohr, Z_val = 4, Ecut 10 Ha, 32^3, 20 bands."""
    a = 10.26
    frac = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0],
                     [.25, .25, .25], [.25, .75, .75], [.75, .25, .75], [.75, .75, .25]])
    rng = np.random.default_rng(seed)
    pos = frac * a + (rng.normal(scale=jitter, size=frac.shape) if jitter > 0 else 0.0)
    return Structure("diamond8", np.eye(3) * a, [dict(SPECIES_Z4)], np.zeros(8, np.int32),
                     pos, 10.0, 20, (32, 32, 32), 0.0)


def diamond8_k222() -> Structure:
    """The 8-atom diamond cell on a 2 x 2 x 2 Gamma-centred k mesh (the rough sampling of a
    crystal's relaxation steps), Fermi-Dirac kT = 0.01 Ha, 20 bands per k point."""
    return dataclasses.replace(diamond8(), name="diamond8_k222", kgrid=(2, 2, 2), kT=0.01)


def honeycomb24(seed: int = 1002, jitter: float = 0.05) -> Structure:
    """24-atom planar honeycomb, 2sqrt3 x 2sqrt3 R30 supercell a = 13.0, c = 26.0 bohr."""
    A, c = 13.0, 26.0
    a0 = A / (2.0 * math.sqrt(3.0))
    p1 = a0 * np.array([1.0, 0.0])
    p2 = a0 * np.array([0.5, math.sqrt(3.0) / 2.0])
    basis = [np.zeros(2), (p1 + p2) / 3.0]
    A1 = 2.0 * (p1 + p2)
    A2 = 2.0 * (2.0 * p2 - p1)
    ang = -math.atan2(A1[1], A1[0])
    rot = np.array([[math.cos(ang), -math.sin(ang)], [math.sin(ang), math.cos(ang)]])
    A1, A2 = rot @ A1, rot @ A2
    sc = np.array([A1, A2])
    inv = np.linalg.inv(sc)
    pts = []
    for i in range(-12, 13):
        for j in range(-12, 13):
            for b in basis:
                r = rot @ (i * p1 + j * p2 + b)
                f = r @ inv
                if np.all(f >= -1e-9) and np.all(f < 1.0 - 1e-9):
                    pts.append(r)
    pts = np.array(pts)
    assert pts.shape[0] == 24, pts.shape
    cell = np.array([[A1[0], A1[1], 0.0], [A2[0], A2[1], 0.0], [0.0, 0.0, c]])
    pos = np.concatenate([pts, np.full((24, 1), 0.5 * c)], axis=1)
    rng = np.random.default_rng(seed)
    pos = pos + rng.normal(scale=jitter, size=pos.shape)
    return Structure("honeycomb24", cell, [dict(SPECIES_Z4)], np.zeros(24, np.int32), pos,
                     15.0, 64, (48, 48, 96), 0.01)


def cluster13(seed: int = 1003) -> Structure:
    """13 Z_val=10 atoms, random compact (d_min 4.5 bohr) in a 20 bohr cube, Ecut 15, 85 bands."""
    rng = np.random.default_rng(seed)
    box = 20.0
    pos = _random_cluster(rng, 13, 4.5, box)
    cell = np.eye(3) * box
    return Structure("cluster13", cell, [dict(SPECIES_Z10)], np.zeros(13, np.int32), pos,
                     15.0, 85, fft_grid(cell, 15.0), 0.01)


def cluster13_pbe() -> Structure:
    """The 13-atom cluster with PBE exchange-correlation (the functional of the paper's searches)."""
    return dataclasses.replace(cluster13(), name="cluster13_pbe", xc="pbe")


def cluster55(seed: int = 1005) -> Structure:
    """55 Z_val=10 atoms (d_min 4.5 bohr) in a 28 bohr cube, Ecut 20 Ha, 330 bands, 128^3."""
    rng = np.random.default_rng(seed)
    box = 28.0
    pos = _random_cluster(rng, 55, 4.5, box)
    return Structure("cluster55", np.eye(3) * box, [dict(SPECIES_Z10)], np.zeros(55, np.int32),
                     pos, 20.0, 330, (128, 128, 128), 0.01)


def de_candidate(i: int, natoms: int = None, ecut: float = 12.0) -> Structure:
    """DE population member i: a perturbed cell of 8-32 Z_val=4 atoms (Sec. II B init).

    Cell A = s (I + eps), eps symmetric with entries U(-0.1, 0.1), volume
    135 bohr^3/atom x U(0.8, 1.2); positions uniform with min-image distance 3.5 bohr;
    bands = ceil(1.25 n_occ) rounded up to even; kT = 0.01 Ha.
    """
    rng = np.random.default_rng(4000 + i)
    n = int(rng.integers(8, 33)) if natoms is None else int(natoms)
    e = rng.uniform(-0.1, 0.1, size=(3, 3))
    e = 0.5 * (e + e.T)
    m = np.eye(3) + e
    vol = 135.0 * n * rng.uniform(0.8, 1.2)
    s = (vol / abs(np.linalg.det(m))) ** (1.0 / 3.0)
    cell = s * m
    inv = np.linalg.inv(cell)
    shifts = np.array([[a, b, c] for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)],
                      dtype=np.float64) @ cell
    pos: List[np.ndarray] = []
    while len(pos) < n:
        p = rng.uniform(size=3) @ cell
        ok = True
        for q in pos:
            df = (p - q) @ inv
            df -= np.round(df)
            if np.min(np.linalg.norm(df @ cell + shifts, axis=1)) < 3.5:
                ok = False
                break
        if ok:
            pos.append(p)
    nocc = 2 * n  # 4n electrons, 2 per band
    nb = int(math.ceil(1.25 * nocc))
    nb += nb % 2
    return Structure(f"de{i:03d}", cell, [dict(SPECIES_Z4)], np.zeros(n, np.int32), np.array(pos),
                     ecut, nb, fft_grid(cell, ecut), 0.01)


def de_population(n: int = 64, start: int = 0) -> List[Structure]:
    """The 64-candidate DE population batch (uneven cells, atom and plane-wave counts)."""
    return [de_candidate(i) for i in range(start, start + n)]


def de_search_population(n: int = 8, natoms: int = 8, seed: int = 5000, dmin: float = 3.0) -> List[Structure]:
    """A DE search population (Sec. II B; the paper's population of 8): n structures of
    natoms Z_val=4 atoms in the 10.26 bohr cubic cell of the diamond8 workload (Ecut 10 Ha,
    32^3 grid, 20 bands, kT = 0.01 Ha), positions uniform with min-image distance dmin."""
    base = diamond8(jitter=0.0)
    cell = base.cell
    inv = np.linalg.inv(cell)
    shifts = np.array([[a, b, c] for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)],
                      dtype=np.float64) @ cell
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        pos: List[np.ndarray] = []
        while len(pos) < natoms:
            p = rng.uniform(size=3) @ cell
            ok = True
            for q in pos:
                df = (p - q) @ inv
                df -= np.round(df)
                if np.min(np.linalg.norm(df @ cell + shifts, axis=1)) < dmin:
                    ok = False
                    break
            if ok:
                pos.append(p)
        out.append(dataclasses.replace(base, name=f"dex{k}", pos=np.array(pos), kT=0.01))
    return out


def supercell(st: Structure, reps) -> Structure:
    """The reps[0] x reps[1] x reps[2] supercell of st at the Gamma point: lattice vectors
    reps_i a_i, the atoms of every translate t (t-major: t = 0 first, the atoms in st's
    order), reps_1 reps_2 reps_3 times the bands and the FFT grid scaled per axis."""
    reps = tuple(int(x) for x in reps)
    ts = [(a, b, c) for a in range(reps[0]) for b in range(reps[1]) for c in range(reps[2])]
    pos = np.concatenate([st.pos + np.array(t, dtype=np.float64) @ st.cell for t in ts])
    return dataclasses.replace(st, name=f"{st.name}_x{reps[0]}{reps[1]}{reps[2]}",
                               cell=st.cell * np.array(reps, dtype=np.float64)[:, None],
                               species_of_atom=np.tile(st.species_of_atom, len(ts)), pos=pos,
                               nbands=st.nbands * len(ts), fft=tuple(n * r for n, r in zip(st.fft, reps)),
                               kgrid=(1, 1, 1))


def tiny(nat: int = 2, ecut: float = 3.0, seed: int = 7, kT: float = 0.01, nbands: int = None,
         skew: bool = True, species=None) -> Structure:
    """A small skewed cell for fast CPU and GPU unit tests (tens to hundreds of plane waves)."""
    rng = np.random.default_rng(seed)
    cell = np.array([[6.0, 0.0, 0.0], [0.6, 6.4, 0.0], [0.3, -0.4, 6.8]]) if skew else np.eye(3) * 6.5
    sp = dict(SPECIES_Z4) if species is None else dict(species)
    pos = []
    inv = np.linalg.inv(cell)
    while len(pos) < nat:
        p = rng.uniform(size=3) @ cell
        if all(np.linalg.norm(((p - q) @ inv - np.round((p - q) @ inv)) @ cell) > 2.5 for q in pos):
            pos.append(p)
    nel = nat * sp["z_val"]
    nb = nbands if nbands is not None else int(math.ceil(nel / 2 * 1.25)) + 1
    return Structure("tiny", cell, [sp], np.zeros(nat, np.int32), np.array(pos), ecut, nb,
                     fft_grid(cell, ecut), kT)


CONFIGS = {
    "diamond8": diamond8,
    "diamond8_k222": diamond8_k222,
    "honeycomb24": honeycomb24,
    "cluster13": cluster13,
    "cluster13_pbe": cluster13_pbe,
    "cluster55": cluster55,
}
