"""Write the oracle's full-size reference values for the error ledger: the named configs
(the 24-atom monolayer, the 13-atom cluster, the diamond cell on a 2 x 2 x 2 k mesh, the 13-atom
cluster with PBE) and DE
population members (``de<i>``, the member i of ``workloads.de_population``, checked inside the
64-member batch).

Runs only oracle/ (plain FP64 SCF, tight tolerances) on the workloads' seeded inputs and
stores, per config, the free energy, the energy terms, every eigenvalue and occupation and
every force component in tests/golden/ledger_<config>.json.  Slow (CPU minutes to hours):
run it by hand, never from a test.

    python tests/golden/make_ledger.py honeycomb24 [cluster13] [de044]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import workloads  # noqa: E402


def structure(name):
    """The seeded input of a ledger name: a named config or population member de<i>."""
    if name in workloads.CONFIGS:
        return workloads.CONFIGS[name](), f"workloads.CONFIGS['{name}']()"
    if name.startswith("de") and name[2:].isdigit():
        return workloads.de_candidate(int(name[2:])), f"workloads.de_candidate({int(name[2:])})"
    raise KeyError(name)


def main(names):
    for name in names:
        st, src = structure(name)
        t0 = time.time()
        mesh = tuple(getattr(st, "kgrid", (1, 1, 1))) != (1, 1, 1)
        r = oracle.kpoints.scf(st) if mesh else oracle.scf(st)
        dt = time.time() - t0
        fn = "oracle.kpoints.scf" if mesh else "oracle.scf"
        out = dict(_source=f"{fn} on {src}, FP64, default tolerances "
                           f"(|dF| < 1e-8 Ha, density residual < 1e-7), {r.n_iter} iterations, {dt:.0f} s",
                   natoms=int(st.natoms), free_energy=float(r.free_energy), energy=float(r.energy),
                   terms={k: float(v) for k, v in r.terms.items()}, eig=np.asarray(r.eig).tolist(),
                   occ=np.asarray(r.occ).tolist(), forces=np.asarray(r.forces).tolist(), n_iter=int(r.n_iter))
        if mesh:
            out["kgrid"] = list(st.kgrid)  # eig / occ: (n_k, n_b), the mesh points in t-major order
        with open(os.path.join(HERE, f"ledger_{name}.json"), "w") as fh:
            json.dump(out, fh, indent=1)
        print(name, r.free_energy, r.n_iter, f"{dt:.0f} s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["honeycomb24"])
