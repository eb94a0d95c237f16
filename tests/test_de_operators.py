"""The library's DE operators (csrc/de.cpp, through the C ABI) against the oracle's
(oracle/de.py): the same population, energies and random numbers must give the same
children.  Host code only: runs without a GPU.  On the GPU,
tests/test_gpu_parity.py::test_de_generation_matches_the_oracle runs a whole generation."""
import numpy as np
import pytest

from oracle import de


@pytest.fixture(scope="module")
def sgo():
    from paper_1603_02732_gb300 import build
    build.build()
    import paper_1603_02732_gb300 as pkg
    pkg.load_library()
    return pkg


def _population(np_, na, seed, cell):
    rng = np.random.default_rng(seed)
    pop = rng.uniform(0, 1, size=(np_, na, 3)) @ cell
    f = -10.0 - rng.uniform(size=np_)
    return pop, f


CELLS = [np.diag([10.26, 10.26, 10.26]), np.array([[12.0, 0.0, 0.0], [1.0, 11.5, 0.0], [0.5, -0.8, 12.5]])]


@pytest.mark.parametrize("scheme", ["random", "plane", "sphere"])
@pytest.mark.parametrize("cell", range(2))
def test_offspring_match_oracle(sgo, scheme, cell):
    A = CELLS[cell]
    species = np.array([0, 0, 1, 0, 1, 0, 0, 1])
    for seed in range(6):
        pop, f = _population(8, 8, seed, A)
        u = np.random.default_rng(100 + seed).uniform(size=(8, de.RANDOMS))
        got = sgo.de_offspring(A, species, pop, f, u, scheme=scheme, d_min=2.0)
        ref = de.offspring(A, species, pop, f, u, scheme=scheme, d_min=2.0)
        assert np.abs(got - ref).max() < 1e-9, (seed, np.abs(got - ref).max())


def test_offspring_argument_checks(sgo):
    A = CELLS[0]
    pop, f = _population(3, 4, 0, A)
    with pytest.raises(sgo.SgoError):   # fewer than four individuals: no three partners
        sgo.de_offspring(A, np.zeros(4), pop, f, np.zeros((3, de.RANDOMS)))


def test_migration_and_similarity_match_oracle(sgo):
    rng = np.random.default_rng(12)
    A = CELLS[1]
    for nsub in (1, 2, 4):
        pop, f = _population(8, 5, 20 + nsub, A)
        f[rng.integers(0, 8)] = f.min()      # a tie, resolved by index on both sides
        p1, f1 = sgo.de_migrate(pop, f, nsub)
        p2, f2 = de.migrate(pop, f, nsub)
        assert np.array_equal(f1, f2) and np.array_equal(p1, p2), nsub
    X = rng.uniform(0, 1, size=(7, 3)) @ A
    for shift in (0.0, 0.02, 0.3):
        Y = X.copy()
        Y[3] += shift
        for tol in (1e-9, 0.01, 0.05):
            assert sgo.de_similar(A, X, Y, tol) == de.similar(A, X, Y, tol), (shift, tol)
