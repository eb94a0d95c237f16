"""The stored oracle ledgers (tests/golden/ledger_*.json, written by make_ledger.py from oracle/
alone) against the identities every converged oracle result obeys, so that a corrupted or
mis-generated file fails on the CPU before a GPU test compares against it: the terms add up
to F, E - F = kT S, the occupations hold every valence electron (weighted over a k mesh), the
eigenvalues come sorted, and the net force vanishes up to the FFT grid's egg-box term."""
import glob
import json
import os

import numpy as np
import pytest

import workloads

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
LEDGERS = sorted(glob.glob(os.path.join(HERE, "ledger_*.json")))


def _structure(name):
    if name in workloads.CONFIGS:
        return workloads.CONFIGS[name]()
    assert name.startswith("de") and name[2:].isdigit(), name
    return workloads.de_candidate(int(name[2:]))


@pytest.mark.parametrize("path", LEDGERS, ids=[os.path.basename(p) for p in LEDGERS])
def test_ledger_identities(path):
    d = json.load(open(path))
    name = os.path.basename(path)[len("ledger_"):-len(".json")]
    st = _structure(name)
    t = d["terms"]
    parts = ("kinetic", "nonlocal_", "local", "hartree", "xc", "ewald", "minus_ts")
    assert abs(sum(t[k] for k in parts) - d["free_energy"]) < 1e-10
    assert t["total"] == d["free_energy"]
    assert abs((d["energy"] - d["free_energy"]) + t["minus_ts"]) < 1e-10
    occ, eig = np.array(d["occ"]), np.array(d["eig"])
    assert occ.shape == eig.shape
    if occ.ndim == 2:  # a k mesh: equal weights over the mesh points
        assert list(d["kgrid"]) == list(st.kgrid) and occ.shape[0] == int(np.prod(st.kgrid))
        nel = float(np.sum(occ)) / occ.shape[0]
    else:
        nel = float(np.sum(occ))
    assert abs(nel - st.nelec) < 1e-9
    assert np.all((occ >= 0.0) & (occ <= 2.0))
    assert np.all(np.diff(eig, axis=-1) >= -1e-12)
    assert d["natoms"] == st.natoms and np.array(d["forces"]).shape == (st.natoms, 3)
    # translation invariance holds up to the grid's egg-box term (below 3e-5 Ha/bohr here)
    assert np.abs(np.array(d["forces"]).sum(axis=0)).max() < 1e-4
