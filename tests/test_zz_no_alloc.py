"""The H psi entry point that allocates no device memory gives the same result as the
ordinary one (callers that cannot let a library allocate use it; see include/sgo.h).

It shares one device scratch array between calls, so it is run twice in a row here;
this file is collected last so that a failing run stops after every other test.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sgo():
    from paper_1603_02732_gb300 import build
    build.build()
    import paper_1603_02732_gb300 as pkg
    pkg.load_library()
    return pkg


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 2e-5)])
def test_noalloc_hpsi_matches_apply_hamiltonian(sgo, precision, tol):
    for seed, st in ((3, workloads.tiny(nat=2, ecut=3.5)), (4, workloads.diamond8())):
        ctx = sgo.Context(st, precision=precision)
        rng = np.random.default_rng(seed)
        veff = rng.normal(size=ctx.grid) * 0.3
        for call in range(2):
            x = rng.normal(size=(st.nbands - call, ctx.npw))
            ref = ctx.apply_hamiltonian(veff, x)
            out = ctx.apply_hamiltonian_noalloc(veff, x)
            assert np.abs(out - ref).max() <= tol * np.abs(ref).max(), (precision, call)


def test_noalloc_rejects_oversize(sgo):
    """A problem whose staged psi/hpsi alone exceed the 32 MiB scratch is refused with an
    error (20 bohr cube, Ecut 15 Ha: 22119 plane waves; 150 vectors -> ~53 MB)."""
    st = workloads.Structure("big", np.eye(3) * 20.0, [dict(workloads.SPECIES_Z4)], np.zeros(2, np.int32),
                             np.array([[5.0, 5.0, 5.0], [10.0, 11.0, 12.0]]), 15.0, 150, (72, 72, 72), 0.01)
    ctx = sgo.Context(st, precision="fp64")
    assert 2 * 150 * ctx.npw * 8 > 32 * 2 ** 20
    with pytest.raises(sgo.SgoError) as e:
        ctx.apply_hamiltonian_noalloc(np.zeros(ctx.grid), np.zeros((150, ctx.npw)))
    assert e.value.status == sgo.SGO_ERR_ARG
    assert "no-alloc scratch" in str(e.value)
