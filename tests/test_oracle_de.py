"""Pins of the oracle's differential-evolution operators (Sec. II B) against special cases
and invariants."""
import itertools

import numpy as np

from oracle import de

CELL = np.array([[12.0, 0.0, 0.0], [1.0, 11.5, 0.0], [0.5, -0.8, 12.5]])


def test_partners_are_distinct_and_exclude_the_target():
    for i in range(5):
        for u in itertools.product([0.0, 0.3, 0.61, 0.999], repeat=3):
            r = de.partners(i, 5, u)
            assert len(set(r)) == 3 and i not in r


def test_equal_fitness_mutation_is_the_centroid():
    """p1 = p2 = p3 cancels the difference terms of Eq. 2: V is the centroid of the three
    donors (minimum image), wrapped into the cell."""
    rng = np.random.default_rng(1)
    X = [rng.uniform(0, 1, size=(6, 3)) @ CELL for _ in range(3)]
    V = de.triangle_mutation(CELL, *X, -3.0, -3.0, -3.0)
    inv = np.linalg.inv(CELL)
    s = [x @ inv for x in X]
    c = s[0] + (de._mi(s[1] - s[0]) + de._mi(s[2] - s[0])) / 3.0
    assert np.allclose(V @ inv, c - np.floor(c), atol=1e-12)


def test_mutation_is_translation_equivariant():
    """The coefficients of Eq. 2 sum to one: a common translation of the donors
    translates V (modulo the cell)."""
    rng = np.random.default_rng(2)
    X = [rng.uniform(0, 1, size=(5, 3)) @ CELL for _ in range(3)]
    f = (-2.0, -5.0, -3.5)
    t = np.array([0.7, -1.3, 2.2])
    V = de.triangle_mutation(CELL, *X, *f)
    Vt = de.triangle_mutation(CELL, *[x + t for x in X], *f)
    inv = np.linalg.inv(CELL)
    assert np.allclose(de._mi((Vt - V - t) @ inv), 0.0, atol=1e-12)


def test_child_has_the_parents_composition():
    rng = np.random.default_rng(3)
    species = np.array([0, 0, 1, 0, 1, 1, 0, 2])
    for k in range(40):
        P1 = rng.uniform(0, 10, size=(8, 3))
        P2 = rng.uniform(0, 10, size=(8, 3))
        u = rng.uniform(size=4)
        C = de.cut_and_splice(species, P1, P2, (u[0], u[1]), u[2], u[3])
        for slot in range(8):  # every child atom is an atom of that species from a parent
            src = [P[m] for P in (P1, P2) for m in range(8) if species[m] == species[slot]]
            assert min(np.abs(C[slot] - s).max() for s in src) == 0.0
        # no parent atom is used twice
        used = {(p, m) for slot in range(8) for p, P in enumerate((P1, P2)) for m in range(8)
                if np.array_equal(C[slot], P[m])}
        assert len(used) == 8


def test_plane_through_a_symmetric_cluster_keeps_it_whole():
    """A cube of 8 atoms cut through its centre by a horizontal plane: P1's upper four and
    P2's lower four rebuild the cube."""
    cube = np.array(list(itertools.product([0.0, 2.5], repeat=3))) + 5.0
    species = np.zeros(8, int)
    C = de.cut_and_splice(species, cube, cube[::-1].copy(), (0.0, 0.0), 0.0, 0.5, scheme="plane")
    assert sorted(map(tuple, C)) == sorted(map(tuple, cube))
    up = C[:4]
    assert np.all(up[:, 2] > 5.0 + 1e-9)   # kept slots hold P1's upper half (normal +z)


def test_repair_leaves_every_distance_at_least_dmin():
    rng = np.random.default_rng(4)
    X = rng.uniform(0, 4.0, size=(10, 3)) + 4.0
    Y = de.repair(CELL, X, d_min=2.0)
    inv = np.linalg.inv(CELL)
    for i in range(10):
        for j in range(i + 1, 10):
            d = np.linalg.norm(de._mi((Y[j] - Y[i]) @ inv) @ CELL)
            assert d >= 2.0 - 1e-9
    # a configuration that already satisfies d_min is left in place (up to the wrap)
    Z = de.repair(CELL, Y, d_min=2.0)
    assert np.allclose(Z, Y, atol=1e-12)


def test_greedy_selection_never_raises_an_energy():
    rng = np.random.default_rng(5)
    pop = rng.uniform(size=(6, 4, 3))
    kids = rng.uniform(size=(6, 4, 3))
    f = rng.normal(size=6)
    fk = rng.normal(size=6)
    p2, f2, better = de.select(pop, f, kids, fk)
    assert np.all(f2 <= f) and np.array_equal(f2, np.minimum(f, fk))
    assert np.array_equal(p2[better], kids[better]) and np.array_equal(p2[~better], pop[~better])


def test_similarity_is_invariant_under_translation_and_permutation():
    rng = np.random.default_rng(6)
    X = rng.uniform(0, 1, size=(6, 3)) @ CELL
    Y = X[rng.permutation(6)] + np.array([3.1, -2.2, 0.7])
    assert de.similar(CELL, X, Y, tol=1e-9)
    Z = X.copy()
    Z[2] += np.array([0.8, 0.0, 0.0])
    assert not de.similar(CELL, X, Z, tol=0.05)


def test_ring_migration_moves_each_best_to_the_next_subpopulation():
    pop = np.arange(8, dtype=float).reshape(8, 1, 1)
    f = np.array([-1.0, -3.0, 0.0, 2.0, -5.0, 1.0, -2.0, 4.0])
    p2, f2 = de.migrate(pop, f, 4)
    # subpopulations {0,1} {2,3} {4,5} {6,7}; bests (before any copy) slots 1, 2, 4, 6 and
    # worsts 0, 3, 5, 7: slot 1 (-3) replaces slot 3 (2), slot 2 (0) replaces slot 5 (1),
    # slot 4 (-5) replaces slot 7 (4), slot 6 (-2) replaces slot 0 (-1)
    assert f2.tolist() == [-2.0, -3.0, 0.0, -3.0, -5.0, 0.0, -2.0, -5.0]
    assert p2[:, 0, 0].tolist() == [6.0, 1.0, 2.0, 1.0, 4.0, 2.0, 6.0, 4.0]
    assert np.all(f2 <= f)


def test_ring_migration_moves_a_migrant_one_step_only():
    """Three subpopulations with one dominant individual: it reaches the next subpopulation
    only.  Were best and worst re-read after each copy, the migrant would be the best of
    subpopulation 1 on the next pass, cascade round the ring and overwrite slot 1 as well."""
    pop = np.arange(6, dtype=float).reshape(6, 1, 1)
    f = np.array([-9.0, 0.0, 5.0, 6.0, 7.0, 8.0])
    p2, f2 = de.migrate(pop, f, 3)
    assert f2.tolist() == [-9.0, 0.0, 5.0, -9.0, 7.0, 5.0]
    assert p2[:, 0, 0].tolist() == [0.0, 1.0, 2.0, 0.0, 4.0, 2.0]
    # one subpopulation has no neighbour: nothing moves (no duplicate of its best)
    p1, f1 = de.migrate(pop, f, 1)
    assert np.array_equal(p1, pop) and np.array_equal(f1, f)
