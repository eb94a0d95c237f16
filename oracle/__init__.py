"""Plain FP64 CPU oracle of the plane-wave DFT energy + force evaluation.

TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference arm may import or run anything in this package; the
product path (paper_1603_02732_gb300) never does, and this package imports
nothing from it.  It is written from the physics the paper's DFT level computes
(Sec. II A and II D: self-consistent energy and atomic forces of a structure,
the Kohn-Sham problem of Algorithm 1, rho_in -> rho_out -> mixing), using NumPy,
SciPy's LAPACK/LOBPCG and numpy.fft as library steps, in float64.

Every function is pinned by tests/test_oracle_*.py against closed forms,
textbook constants, brute force or invariants.  The whole-pipeline numbers have
no counterpart in the paper (it prints none for this synthetic model): parity
against the paper itself is unpinned; each component is pinned separately.
"""
from . import basis, dft, ewald, gga, kpoints, lda, pseudo  # noqa: F401
from .dft import Model, Result, evaluate, scf  # noqa: F401
