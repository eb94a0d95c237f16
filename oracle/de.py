"""Differential-evolution operators of the global search (Sec. II B): the level above the
local relaxation.

TEST INFRASTRUCTURE (oracle): only tests/ and bench.py's CPU legs use it; it imports
nothing from the product package.  Plain NumPy, written from Sec. II B.  The random
numbers the operators draw are inputs (SGO_DE_RANDOMS uniforms in [0, 1) per offspring),
so that this module and the library's operators (csrc/de.cpp) can be compared exactly.

An individual is a structure of natoms atoms (species fixed per atom slot) in a cell
shared by the population; its fitness is its relaxed free energy.  For every individual
X_i of a generation:
* triangle mutation (Eq. 2): three distinct others r1, r2, r3 != i and
  V = (X1 + X2 + X3)/3 + (p2 - p1)(X1 - X2) + (p3 - p2)(X2 - X3) + (p1 - p3)(X3 - X1),
  p_k = |f_k| / (|f_1| + |f_2| + |f_3|), in fractional coordinates with minimum-image
  differences (X_k - X_1 wrapped into [-1/2, 1/2)), then wrapped into the cell;
* cut-and-splice crossover of V (parent P1) with X_i (parent P2): plane-cut-splice (a
  random plane through each parent's centre) or sphere-cut-splice (a sphere of random
  radius around each parent's centre); the child keeps P1's atoms on one side and fills
  every species up to its count with P2's atoms from the other side, nearest the cut
  first, which gives the right composition in one pass (the paper rotates the plane until
  the counts match);
* distance repair: any pair closer than d_min (minimum image) is pushed apart along its
  separation, the later atom moving, in passes until none is (at most 100 passes);
* greedy selection: the relaxed child replaces X_i when its energy is lower;
* migration between subpopulations (consecutive slices): ring order, the best of one
  replaces the worst of the next when better;
* similarity (the initialisation's check between structures): sorted minimum-image pair
  distances, similar when their RMS difference is below a tolerance.

Pins (tests/test_oracle_de.py): Eq. 2 reduces to the centroid when the three fitnesses are
equal; the child always has the parents' composition; a plane through the centre of a
symmetric cluster splits it in halves; the repair leaves every distance >= d_min; greedy
selection never raises an energy.
"""
from __future__ import annotations

import numpy as np

RANDOMS = 7      # uniforms per offspring: 3 partners, 2 plane normal, 1 scheme, 1 sphere radius
D_MIN = 2.0      # bohr


def _wrap(s):
    return s - np.floor(s)


def _mi(ds):
    return ds - np.round(ds)


def partners(i, np_, u):
    """r1, r2, r3: distinct, != i, drawn without replacement from u[0:3]."""
    pool = [k for k in range(np_) if k != i]
    out = []
    for k in range(3):
        j = min(int(u[k] * len(pool)), len(pool) - 1)
        out.append(pool.pop(j))
    return out


def triangle_mutation(cell, X1, X2, X3, f1, f2, f3):
    """Eq. 2 in fractional coordinates; returns Cartesian positions wrapped into the cell."""
    A = np.asarray(cell, float)
    inv = np.linalg.inv(A)
    s1 = X1 @ inv
    d2 = _mi(X2 @ inv - s1)
    d3 = _mi(X3 @ inv - s1)
    s2, s3 = s1 + d2, s1 + d3
    tot = abs(f1) + abs(f2) + abs(f3)
    if tot > 0:
        p1, p2, p3 = abs(f1) / tot, abs(f2) / tot, abs(f3) / tot
    else:
        p1 = p2 = p3 = 1.0 / 3.0
    v = (s1 + s2 + s3) / 3.0 + (p2 - p1) * (s1 - s2) + (p3 - p2) * (s2 - s3) + (p1 - p3) * (s3 - s1)
    return _wrap(v) @ A


def _normal(u1, u2):
    z = 1.0 - 2.0 * u1
    r = np.sqrt(max(0.0, 1.0 - z * z))
    phi = 2.0 * np.pi * u2
    return np.array([r * np.cos(phi), r * np.sin(phi), z])


def cut_and_splice(species, P1, P2, u_normal, u_scheme, u_radius, scheme="random"):
    """Child of P1 (kept side) and P2 (fill), composition of the parents.  scheme: 'plane',
    'sphere', or 'random' (plane when u_scheme < 1/2).  Plane: kept P1 atoms have
    (x - c1).n > 0, P2 fills with its atoms of smallest (x - c2).n; sphere (radius
    u_radius * max |x - c1| over P1): kept P1 atoms have |x - c1| < R, P2 fills with its
    atoms of largest |x - c2|.  Ties go to the lower index; child slots of each species
    take the kept atoms (index order), then the fill atoms (index order)."""
    species = np.asarray(species)
    c1, c2 = P1.mean(axis=0), P2.mean(axis=0)
    plane = scheme == "plane" or (scheme == "random" and u_scheme < 0.5)
    if plane:
        nv = _normal(*u_normal)
        k1 = (P1 - c1) @ nv
        keep = k1 > 0.0
        key2 = (P2 - c2) @ nv             # fill: smallest first
    else:
        d1 = np.linalg.norm(P1 - c1, axis=1)
        R = u_radius * d1.max()
        keep = d1 < R
        key2 = -np.linalg.norm(P2 - c2, axis=1)   # fill: farthest first
    child = np.empty_like(P1)
    for s in np.unique(species):
        slots = np.where(species == s)[0]
        kept = [k for k in slots if keep[k]]
        need = len(slots) - len(kept)
        order = sorted(slots, key=lambda k: (key2[k], k))
        fill = sorted(order[:need])
        for slot, k in zip(slots, kept):
            child[slot] = P1[k]
        for slot, k in zip(slots[len(kept):], fill):
            child[slot] = P2[k]
    return child


def repair(cell, X, d_min=D_MIN, passes=100):
    """Push apart every pair closer than d_min (minimum image): the later atom of a pair
    moves along the separation to distance d_min; repeated in passes (index order)."""
    A = np.asarray(cell, float)
    inv = np.linalg.inv(A)
    X = np.array(X, float)
    n = len(X)
    for _ in range(passes):
        moved = False
        for i in range(n):
            for j in range(i + 1, n):
                dv = _mi((X[j] - X[i]) @ inv) @ A
                d = np.linalg.norm(dv)
                if d < d_min:
                    e = dv / d if d > 1e-12 else np.array([1.0, 0.0, 0.0])
                    X[j] = X[j] + (d_min - d) * e
                    moved = True
        if not moved:
            break
    return _wrap(X @ inv) @ A


def offspring(cell, species, pop, f, u, scheme="random", d_min=D_MIN):
    """One child per individual from the uniforms u[i, 0:RANDOMS]."""
    pop = np.asarray(pop, float)
    kids = np.empty_like(pop)
    for i in range(len(pop)):
        r1, r2, r3 = partners(i, len(pop), u[i])
        V = triangle_mutation(cell, pop[r1], pop[r2], pop[r3], f[r1], f[r2], f[r3])
        C = cut_and_splice(species, V, pop[i], (u[i][3], u[i][4]), u[i][5], u[i][6], scheme)
        kids[i] = repair(cell, C, d_min)
    return kids


def fingerprint(cell, X):
    """The structure's sorted minimum-image pair distances (the similarity check at
    initialisation compares structures by them)."""
    A = np.asarray(cell, float)
    inv = np.linalg.inv(A)
    X = np.asarray(X, float)
    d = [np.linalg.norm(_mi((X[j] - X[i]) @ inv) @ A) for i in range(len(X)) for j in range(i + 1, len(X))]
    return np.sort(np.array(d))


def similar(cell, X, Y, tol=0.05):
    """Two structures are similar when their fingerprints differ by less than tol (bohr, root
    mean square over the pairs)."""
    a, b = fingerprint(cell, X), fingerprint(cell, Y)
    return bool(np.sqrt(np.mean((a - b) ** 2)) < tol) if len(a) else True


def migrate(pop, f, nsub):
    """Ring migration between nsub equal subpopulations (consecutive slices of the
    population): the best individual of subpopulation s replaces the worst of subpopulation
    (s + 1) mod nsub when it is better.  Best and worst are taken on the population as it was
    before the migration (every migrant moves one step round the ring); one subpopulation
    has no neighbour and nothing moves."""
    pop = np.array(pop, float)
    f = np.array(f, float)
    if nsub == 1:
        return pop, f
    size = len(f) // nsub
    subs = [range(s_ * size, (s_ + 1) * size) for s_ in range(nsub)]
    best = [min(r, key=lambda k: (f[k], k)) for r in subs]
    worst = [max(r, key=lambda k: (f[k], -k)) for r in subs]
    src_x = [pop[b].copy() for b in best]
    src_f = [f[b] for b in best]
    dst_f = [f[w] for w in worst]
    for s_ in range(nsub):
        t = (s_ + 1) % nsub
        if src_f[s_] < dst_f[t]:
            pop[worst[t]] = src_x[s_]
            f[worst[t]] = src_f[s_]
    return pop, f


def select(pop, f, kids, fk):
    """Greedy selection: the lower energy of parent and child survives."""
    pop = np.array(pop, float)
    f = np.array(f, float)
    better = np.asarray(fk) < f
    pop[better] = np.asarray(kids)[better]
    f[better] = np.asarray(fk)[better]
    return pop, f, better
