"""The library's relaxation driver (csrc/relax.cpp, through the C ABI) against the oracle's
(oracle/relax.py): both walk the same energy/force function from the same start, and
every configuration they ask to evaluate must agree.  Host code only: runs without a GPU.
On the GPU, tests/test_gpu_parity.py::test_relax_batch_reaches_a_minimum drives it with
the batched DFT evaluation."""
import numpy as np
import pytest

from oracle import relax as rx


@pytest.fixture(scope="module")
def sgo():
    from paper_1603_02732_gb300 import build
    build.build()
    import paper_1603_02732_gb300 as pkg
    pkg.load_library()
    return pkg


THETA = (0.15, 1.3, 2.9)


def _cases():
    rng = np.random.default_rng(11)
    big = np.eye(3) * 40.0
    dimer = np.array([[20.0, 20.0, 20.0], [20.0, 20.0, 20.0 + THETA[2] + 0.35]])
    trimer = np.array([[20.0, 20.0, 20.0], [23.3, 20.1, 20.0], [21.2, 22.9, 20.2]])
    cluster = 20.0 + rng.uniform(-2.6, 2.6, size=(5, 3))
    # a periodic crystal: 4 atoms in a skewed 7-bohr cell, images inside the cutoff
    cell = np.array([[7.0, 0.0, 0.0], [0.7, 6.8, 0.0], [0.3, -0.5, 7.2]])
    frac = np.array([[0.0, 0.0, 0.0], [0.5, 0.52, 0.0], [0.48, 0.0, 0.5], [0.0, 0.5, 0.47]])
    crystal = frac @ cell + rng.normal(scale=0.15, size=(4, 3))
    return [("dimer", big, dimer), ("trimer", big, trimer), ("cluster5", big, cluster), ("crystal4", cell, crystal)]


def _model(cell, theta):
    """The 'DFT' of these tests: a periodic shifted-force Morse field with parameters the
    fit starts far from."""
    def ef(pos):
        return 0.0, rx.ff_forces(theta, cell, np.asarray(pos, float).reshape(-1, 3), 8.0)
    return ef


def _drive(sgo, cell, pos0, ef, method, **opts):
    r = sgo.Relax(cell, pos0, method=method, **opts)
    seq = [r.positions()]
    E, F = ef(seq[-1])
    state = 0
    while True:
        nxt, state = r.step(E, F)
        if state != 0:
            break
        seq.append(nxt)
        E, F = ef(nxt)
    return seq, state, nxt


@pytest.mark.parametrize("method", ["pcg", "cg", "bfgs"])
@pytest.mark.parametrize("case", range(4))
def test_driver_matches_oracle(sgo, method, case):
    name, cell, pos0 = _cases()[case]
    ef = _model(cell, THETA)
    kw = dict(fmax=1e-5, max_evals=40)
    tr = rx.relax(ef, cell, pos0, method=method, **kw)
    seq, state, final = _drive(sgo, cell, pos0, ef, method, **kw)
    assert len(seq) == len(tr.positions), (name, len(seq), len(tr.positions))
    for k, (a, b) in enumerate(zip(seq, tr.positions)):
        assert np.abs(a - b).max() < 1e-7, (name, k, np.abs(a - b).max())
    assert state == (1 if tr.converged else 2), name
    assert np.abs(final - tr.final).max() < 1e-7


def test_driver_argument_checks(sgo):
    import ctypes
    lib = sgo.load_library()
    out = ctypes.c_void_p()
    cell = np.eye(3).ravel()
    pos = np.zeros(3)
    o = sgo.sgo_relax_opts()
    lib.sgo_relax_opts_default(ctypes.byref(o))
    o.method = 7
    assert lib.sgo_relax_create(1, sgo._ptr(cell), sgo._ptr(pos), ctypes.byref(o), ctypes.byref(out)) == sgo.SGO_ERR_ARG
    assert lib.sgo_relax_create(0, sgo._ptr(cell), sgo._ptr(pos), None, ctypes.byref(out)) == sgo.SGO_ERR_ARG
    r = sgo.Relax(np.eye(3) * 10, np.zeros((1, 3)))
    with pytest.raises(sgo.SgoError):
        r.step(0.0, np.array([np.nan, 0.0, 0.0]))
    # a lone atom feels no force: converged at the first evaluation
    nxt, st = r.step(0.0, np.zeros(3))
    assert st == 1 and np.all(nxt == 0.0)


def test_driver_budget_and_repeat_after_stop(sgo):
    """max_evals = 1 stops after the first evaluation (state 2); later calls repeat the
    final positions without consuming forces; the best configuration is the lowest-energy
    one evaluated."""
    cell = np.eye(3) * 40.0
    pos = np.array([[20.0, 20.0, 20.0], [20.0, 20.0, 23.5]])
    ef = _model(cell, THETA)
    r = sgo.Relax(cell, pos, method="bfgs", fmax=1e-9, max_evals=1)
    E, F = ef(pos)
    nxt, st = r.step(-1.0, F)
    assert st == 2 and np.array_equal(nxt, pos)
    nxt2, st2 = r.step(5.0, np.full(6, np.nan))   # ignored after the stop
    assert st2 == 2 and np.array_equal(nxt2, pos)
    e, x = r.best()
    assert e == -1.0 and np.array_equal(x, pos)
    assert r.info() == dict(evals=1, state=2)


def test_batch_entry_points_check_arguments_on_the_host(sgo):
    import ctypes
    lib = sgo.load_library()
    rounds = ctypes.c_int(7)
    assert lib.sgo_relax_batch(None, None, 5, ctypes.byref(rounds), None) == sgo.SGO_ERR_ARG
    assert rounds.value == 0
    cell = np.eye(3).ravel()
    assert lib.sgo_de_generation(None, sgo._ptr(cell), None, None, None, None, 0, 2.0, None, 5, None,
                                 None) == sgo.SGO_ERR_ARG
