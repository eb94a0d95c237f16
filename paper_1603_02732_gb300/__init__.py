"""GB300 plane-wave DFT energy + force engine: Python binding of libsgo.so.

The paper's bottom search level (Sec. II A, Sec. II D) evaluates the energy and
atomic forces of a structure self-consistently; every differential-evolution
candidate (Sec. II B) and relaxation step (Sec. II C) calls it.  All work runs
in the CUDA kernels of libsgo.so behind the C ABI declared in include/sgo.h;
this module only marshals arguments (ctypes).  There is no CPU fallback: if the
library is missing the import of the binding fails.

    ctx = Context(structure, precision="mixed")   # a workloads.Structure-like object
    F, forces = ctx.energy_forces()
    batch = Batch([ctx1, ctx2, ...]); E, Fs, st = batch.energy_forces()
    E = SgoEnergy.apply(ctx, pos)                  # torch autograd, dE/dR = -forces
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsgo.so")

STATUS = {0: "ok", 1: "invalid argument", 2: "invalid geometry", 3: "CUDA error", 4: "out of device memory",
          5: "SCF not converged", 6: "device wait timed out", 7: "non-finite result"}
SGO_OK, SGO_ERR_ARG, SGO_ERR_GEOMETRY, SGO_ERR_CUDA, SGO_ERR_OOM, SGO_ERR_NOT_CONVERGED, SGO_ERR_TIMEOUT, \
    SGO_ERR_NAN = range(8)
TERM_NAMES = ("kinetic", "nonlocal", "local", "hartree", "xc", "ewald", "minus_ts", "free_energy")


class SgoError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


class sgo_species(ctypes.Structure):
    _fields_ = [("z_val", ctypes.c_double), ("rc", ctypes.c_double), ("a_sr", ctypes.c_double),
                ("sigma_sr", ctypes.c_double), ("rp", ctypes.c_double), ("d_nl", ctypes.c_double),
                ("rp_p", ctypes.c_double), ("d_p", ctypes.c_double)]


class sgo_relax_opts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("fmax", ctypes.c_double), ("max_step", ctypes.c_double),
                ("refit", ctypes.c_int), ("rc", ctypes.c_double), ("accept", ctypes.c_double),
                ("max_evals", ctypes.c_int)]


RELAX_METHODS = {"pcg": 0, "cg": 1, "bfgs": 2}
DE_SCHEMES = {"random": 0, "plane": 1, "sphere": 2}
DE_RANDOMS = 7


def relax_opts(method="pcg", **opts) -> "sgo_relax_opts":
    o = sgo_relax_opts()
    load_library().sgo_relax_opts_default(ctypes.byref(o))
    o.method = RELAX_METHODS[method]
    for k, v in opts.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown relaxation option {k}")
        setattr(o, k, v)
    return o


def de_migrate(pop, f, nsub):
    """Ring migration between nsub subpopulations (sgo_de_migrate); returns new arrays."""
    pop = np.array(pop, dtype=np.float64, order="C")
    f = np.array(f, dtype=np.float64)
    _check(load_library().sgo_de_migrate(len(f), int(nsub), pop.shape[1], _ptr(pop), _ptr(f)), "sgo_de_migrate")
    return pop, f


def de_similar(cell, a, b, tol=0.05) -> bool:
    """Similarity of two structures by their sorted pair distances (sgo_de_similar)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    cell = np.ascontiguousarray(cell, dtype=np.float64).reshape(9)
    out = ctypes.c_int()
    _check(load_library().sgo_de_similar(len(a), _ptr(cell), _ptr(a), _ptr(b), float(tol), ctypes.byref(out)),
           "sgo_de_similar")
    return bool(out.value)


def de_offspring(cell, species, pop, f, u, scheme="random", d_min=2.0):
    """Children of a DE population (sgo_de_offspring, Sec. II B): pop (np, natoms, 3) bohr,
    f (np,) energies, u (np, DE_RANDOMS) uniforms in [0, 1)."""
    lib = load_library()
    pop = np.ascontiguousarray(pop, dtype=np.float64)
    np_, na = pop.shape[0], pop.shape[1]
    f = np.ascontiguousarray(f, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(np_, DE_RANDOMS)
    sp = np.ascontiguousarray(species, dtype=np.int32)
    cell = np.ascontiguousarray(cell, dtype=np.float64).reshape(9)
    out = np.zeros_like(pop)
    _check(lib.sgo_de_offspring(np_, na, _ptr(cell), _ptr(sp, ctypes.c_int), _ptr(pop), _ptr(f), _ptr(u),
                                DE_SCHEMES[scheme], float(d_min), _ptr(out)), "sgo_de_offspring")
    return out


class sgo_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("kT", ctypes.c_double), ("scf_tol_e", ctypes.c_double),
                ("scf_tol_rho", ctypes.c_double), ("max_scf", ctypes.c_int), ("pulay_hist", ctypes.c_int),
                ("mix_alpha", ctypes.c_double), ("kerker_q0", ctypes.c_double), ("ncg", ctypes.c_int),
                ("ncg_first", ctypes.c_int), ("n_nonscf", ctypes.c_int), ("fft", ctypes.c_int * 3),
                ("seed", ctypes.c_ulonglong), ("gemm_tc", ctypes.c_int), ("graph", ctypes.c_int),
                ("autotune", ctypes.c_int), ("sub_batches", ctypes.c_int), ("eig_tol", ctypes.c_double),
                ("max_polish", ctypes.c_int), ("rr_fp64", ctypes.c_int), ("watchdog_ms", ctypes.c_double),
                ("extra_bands", ctypes.c_int), ("rr_cluster", ctypes.c_int), ("eigensolver", ctypes.c_int),
                ("xc", ctypes.c_int), ("cg_adapt", ctypes.c_double), ("kgrid", ctypes.c_int * 3)]


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_vp = ctypes.c_void_p
_alloc_fn = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_free_fn = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

_SIGS = {
    "sgo_opts_default": (None, [ctypes.POINTER(sgo_opts)]),
    "sgo_set_allocator": (ctypes.c_int, [_alloc_fn, _free_fn, _vp]),
    "sgo_create": (ctypes.c_int, [_dp, ctypes.c_int, ctypes.POINTER(sgo_species), ctypes.c_int, _ip, _dp,
                                  ctypes.c_double, ctypes.c_int, ctypes.POINTER(sgo_opts), _vp,
                                  ctypes.POINTER(_vp)]),
    "sgo_scf": (ctypes.c_int, [_vp, _dp, _ip, _dp]),
    "sgo_energy_forces": (ctypes.c_int, [_vp, _dp, _dp, _dp]),
    "sgo_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
    "sgo_energy_forces_batch": (ctypes.c_int, [_vp, ctypes.POINTER(_dp), _dp, ctypes.POINTER(_dp), _ip]),
    "sgo_energy_forces_batch_device": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "sgo_batch_timer": (ctypes.c_int, [_vp, ctypes.c_char_p]),
    "sgo_batch_timer_read": (ctypes.c_int, [_vp, _dp]),
    "sgo_batch_launches": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_longlong)]),
    "sgo_get_eigen": (ctypes.c_int, [_vp, _dp, _dp]),
    "sgo_get_terms": (ctypes.c_int, [_vp, _dp]),
    "sgo_get_info": (ctypes.c_int, [_vp, _ip]),
    "sgo_get_basis": (ctypes.c_int, [_vp, _ip]),
    "sgo_get_stats": (ctypes.c_int, [_vp, _dp]),
    "sgo_get_density": (ctypes.c_int, [_vp, _dp]),
    "sgo_get_state": (ctypes.c_int, [_vp, _dp, _dp]),
    "sgo_set_state": (ctypes.c_int, [_vp, _dp, _dp]),
    "sgo_apply_hamiltonian": (ctypes.c_int, [_vp, _dp, ctypes.c_int, _dp, _dp]),
    "sgo_apply_hamiltonian_noalloc": (ctypes.c_int, [_vp, _dp, ctypes.c_int, _dp, _dp]),
    "sgo_subspace_matrix": (ctypes.c_int, [_vp, ctypes.c_int, _dp, _dp, _dp]),
    "sgo_block_update": (ctypes.c_int, [_vp, ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp]),
    "sgo_batch_tuning": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    "sgo_relax_opts_default": (None, [ctypes.POINTER(sgo_relax_opts)]),
    "sgo_relax_create": (ctypes.c_int, [ctypes.c_int, _dp, _dp, ctypes.POINTER(sgo_relax_opts), ctypes.POINTER(_vp)]),
    "sgo_relax_step": (ctypes.c_int, [_vp, ctypes.c_double, _dp, _dp, _ip]),
    "sgo_relax_positions": (ctypes.c_int, [_vp, _dp]),
    "sgo_relax_info": (ctypes.c_int, [_vp, _ip, _ip]),
    "sgo_relax_batch": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.c_int, _ip, _ip]),
    "sgo_relax_destroy": (None, [_vp]),
    "sgo_relax_best": (ctypes.c_int, [_vp, _dp, _dp]),
    "sgo_de_offspring": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _dp, _ip, _dp, _dp, _dp, ctypes.c_int,
                                        ctypes.c_double, _dp]),
    "sgo_de_migrate": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp]),
    "sgo_de_similar": (ctypes.c_int, [ctypes.c_int, _dp, _dp, _dp, ctypes.c_double, _ip]),
    "sgo_de_generation": (ctypes.c_int, [_vp, _dp, _ip, _dp, _dp, _dp, ctypes.c_int, ctypes.c_double,
                                         ctypes.POINTER(sgo_relax_opts), ctypes.c_int, _ip, _dp]),
    "sgo_density": (ctypes.c_int, [_vp, ctypes.c_int, _dp, _dp, _dp]),
    "sgo_grid_fft": (ctypes.c_int, [_vp, ctypes.c_int, _dp, _dp]),
    "sgo_set_warm": (ctypes.c_int, [_vp, ctypes.c_int]),
    "sgo_batch_destroy": (None, [_vp]),
    "sgo_destroy": (None, [_vp]),
    "sgo_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "sgo_last_error": (ctypes.c_char_p, []),
}

_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libsgo.so (built by paper_1603_02732_gb300.build.build()); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1603_02732_gb300.build.build() "
                          "(no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, what: str):
    if status != SGO_OK:
        detail = load_library().sgo_last_error()
        raise SgoError(status, what, detail.decode() if detail else "")


def _ptr(a: np.ndarray, ctype=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:  # torch is plumbing only
        pass
    return None


_allocator_refs = None  # the installed callbacks (ctypes must keep them alive)


def use_torch_allocator():
    """Route the library's device memory through PyTorch's caching allocator: contexts and
    batches created afterwards take their buffers from torch's pool (they count in
    torch.cuda.memory_allocated() and obey its memory fraction), and their buffers go back to
    it when they are destroyed.  Undo with use_default_allocator()."""
    global _allocator_refs
    import torch

    def alloc(nbytes, stream, _user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))
        except RuntimeError:  # out of memory: the library reports SGO_ERR_CUDA
            return None

    def release(ptr, _stream, _user):
        torch.cuda.caching_allocator_delete(int(ptr))

    refs = (_alloc_fn(alloc), _free_fn(release))
    _check(load_library().sgo_set_allocator(refs[0], refs[1], None), "sgo_set_allocator")
    _allocator_refs = refs


def use_default_allocator():
    """Back to cudaMalloc/cudaFree for new buffers (blocks from torch's pool still go back to
    it; keep torch's callbacks alive until every context made under them is destroyed)."""
    global _allocator_refs
    _check(load_library().sgo_set_allocator(_alloc_fn(), _free_fn(), None), "sgo_set_allocator")
    _retired.append(_allocator_refs)
    _allocator_refs = None


_retired = []


def default_opts(**kw) -> sgo_opts:
    lib = load_library()
    o = sgo_opts()
    lib.sgo_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precision":
            v = {"fp64": 0, "mixed": 1}.get(v, v) if isinstance(v, str) else int(v)
        if k == "eigensolver":
            v = {"cg": 0, "davidson": 1}.get(v, v) if isinstance(v, str) else int(v)
        if k == "xc":
            v = {"lda": 0, "pbe": 1}.get(v, v) if isinstance(v, str) else int(v)
        if k in ("fft", "kgrid"):
            arr = getattr(o, k)
            for i in range(3):
                arr[i] = int(v[i])
            continue
        setattr(o, k, v)
    return o


class Context:
    """One structure on the GPU (sgo_create).  `st` has cell, species (list of dicts with
    z_val, rc, a_sr, sigma_sr, rp, d_nl and optionally rp_p, d_p), species_of_atom, pos, ecut,
    nbands, fft, kT (and optionally xc and a k mesh kgrid).  Positions and forces are the
    cell's (natoms x 3); with a k mesh, nbands, eigen(), state() and the grids are those of the
    folded supercell (sgo_opts.kgrid)."""

    def __init__(self, st, precision="fp64", stream=None, **opts):
        self.lib = load_library()
        self.st = st
        kw = dict(kT=float(st.kT), fft=tuple(int(x) for x in st.fft), precision=precision,
                  xc=getattr(st, "xc", "lda"), kgrid=tuple(int(x) for x in getattr(st, "kgrid", (1, 1, 1))))
        kw.update(opts)
        self.opts = default_opts(**kw)
        cell = np.ascontiguousarray(st.cell, dtype=np.float64).reshape(9)
        sp = (sgo_species * len(st.species))(*[sgo_species(*(float(s.get(k, 0.0)) for k in
                                                             ("z_val", "rc", "a_sr", "sigma_sr", "rp", "d_nl",
                                                              "rp_p", "d_p")))
                                              for s in st.species])
        spec = np.ascontiguousarray(st.species_of_atom, dtype=np.int32)
        pos = np.ascontiguousarray(st.pos, dtype=np.float64).reshape(-1)
        self.natoms = len(spec)
        h = _vp()
        s = stream if stream is not None else _current_stream()
        _check(self.lib.sgo_create(_ptr(cell), len(st.species), sp, self.natoms, _ptr(spec, ctypes.c_int),
                                   _ptr(pos), float(st.ecut), int(st.nbands), ctypes.byref(self.opts), s,
                                   ctypes.byref(h)), "sgo_create")
        self.h = h
        info = self.info()
        self.nbands = info["nbands"]
        self.npw, self.nhalf, self.grid = info["npw"], info["nhalf"], info["grid"]

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.sgo_destroy(h)
            self.h = None

    # --- evaluation -------------------------------------------------------
    def energy_forces(self, pos=None, check=True):
        F = ctypes.c_double()
        f = np.zeros((self.natoms, 3))
        p = None if pos is None else _ptr(np.ascontiguousarray(pos, dtype=np.float64).reshape(-1))
        st = self.lib.sgo_energy_forces(self.h, p, ctypes.byref(F), _ptr(f))
        if check:
            _check(st, "sgo_energy_forces")
        return F.value, f

    def scf(self, pos=None, check=True):
        it = ctypes.c_int()
        res = ctypes.c_double()
        p = None if pos is None else _ptr(np.ascontiguousarray(pos, dtype=np.float64).reshape(-1))
        st = self.lib.sgo_scf(self.h, p, ctypes.byref(it), ctypes.byref(res))
        if check:
            _check(st, "sgo_scf")
        return it.value, res.value

    def set_warm(self, on=True):
        _check(self.lib.sgo_set_warm(self.h, 1 if on else 0), "sgo_set_warm")

    # --- inspection -------------------------------------------------------
    def info(self):
        a = np.zeros(10, np.int32)
        _check(self.lib.sgo_get_info(self.h, _ptr(a, ctypes.c_int)), "sgo_get_info")
        return dict(npw=int(a[0]), nhalf=int(a[1]), ncolpairs=int(a[2]), grid=(int(a[3]), int(a[4]), int(a[5])),
                    nbands=int(a[6]), natoms=int(a[7]), n_iter=int(a[8]), precision=int(a[9]))

    def stats(self):
        s = np.zeros(8)
        _check(self.lib.sgo_get_stats(self.h, _ptr(s)), "sgo_get_stats")
        return dict(n_iter=int(s[0]), jacobi_sweeps=int(s[1]), resid=float(s[2]), dF=float(s[3]),
                    polish_steps=int(s[4]), eig_resid=float(s[5]), jacobi_cap_hits=int(s[6]), warm=bool(s[7]))

    def get_state(self):
        """(rho_in(G) complex (N1, N2, N3), psi (nbands, npw)): the warm-start state the last
        evaluation left (sgo_get_state)."""
        rho = np.zeros(self.grid, dtype=np.complex128)
        psi = np.zeros((self.nbands, self.npw))
        _check(self.lib.sgo_get_state(self.h, rho.ctypes.data_as(_dp), _ptr(psi)), "sgo_get_state")
        return rho, psi

    def set_state(self, rho_g, psi):
        """Install a warm-start state (sgo_set_state); the next evaluation starts from it."""
        rho = np.ascontiguousarray(rho_g, dtype=np.complex128).reshape(self.grid)
        psi = np.ascontiguousarray(psi, dtype=np.float64).reshape(self.nbands, self.npw)
        _check(self.lib.sgo_set_state(self.h, rho.ctypes.data_as(_dp), _ptr(psi)), "sgo_set_state")

    def eigen(self):
        e = np.zeros(self.nbands)
        o = np.zeros(self.nbands)
        _check(self.lib.sgo_get_eigen(self.h, _ptr(e), _ptr(o)), "sgo_get_eigen")
        return e, o

    def terms(self):
        t = np.zeros(8)
        _check(self.lib.sgo_get_terms(self.h, _ptr(t)), "sgo_get_terms")
        return dict(zip(TERM_NAMES, t.tolist()))

    def basis(self):
        m = np.zeros((1 + self.nhalf, 3), np.int32)
        _check(self.lib.sgo_get_basis(self.h, _ptr(m, ctypes.c_int)), "sgo_get_basis")
        return m

    def density(self):
        r = np.zeros(self.grid)
        _check(self.lib.sgo_get_density(self.h, _ptr(r)), "sgo_get_density")
        return r

    # --- component calls --------------------------------------------------
    def apply_hamiltonian(self, veff, psi):
        veff = np.ascontiguousarray(veff, dtype=np.float64)
        psi = np.ascontiguousarray(np.atleast_2d(psi), dtype=np.float64)
        out = np.zeros_like(psi)
        _check(self.lib.sgo_apply_hamiltonian(self.h, _ptr(veff), psi.shape[0], _ptr(psi), _ptr(out)),
               "sgo_apply_hamiltonian")
        return out

    def apply_hamiltonian_noalloc(self, veff, psi):
        """H psi through the entry point that allocates no device memory (see include/sgo.h)."""
        veff = np.ascontiguousarray(veff, dtype=np.float64)
        psi = np.ascontiguousarray(np.atleast_2d(psi), dtype=np.float64)
        out = np.zeros_like(psi)
        _check(self.lib.sgo_apply_hamiltonian_noalloc(self.h, _ptr(veff), psi.shape[0], _ptr(psi), _ptr(out)),
               "sgo_apply_hamiltonian_noalloc")
        return out

    def subspace_matrix(self, x, y):
        """C = X^T Y through the subspace GEMM kernels (tensor cores on the mixed path)."""
        x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
        y = np.ascontiguousarray(np.atleast_2d(y), dtype=np.float64)
        out = np.zeros((x.shape[0], x.shape[0]))
        _check(self.lib.sgo_subspace_matrix(self.h, x.shape[0], _ptr(x), _ptr(y), _ptr(out)), "sgo_subspace_matrix")
        return out

    def block_update(self, x, m, alpha, beta, y):
        """Y <- alpha M^T X + beta Y through the block-update GEMM kernels (tensor cores on
        the mixed path); returns the new Y."""
        x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
        m = np.ascontiguousarray(m, dtype=np.float64)
        y = np.array(np.atleast_2d(y), dtype=np.float64, order="C")
        _check(self.lib.sgo_block_update(self.h, x.shape[0], _ptr(x), _ptr(m), float(alpha), float(beta), _ptr(y)),
               "sgo_block_update")
        return y

    def grid_fft(self, x, sign):
        """One 3D transform of the SCF's grid FFT (sign -1: r -> G, +1: G -> r, unnormalised)
        of a complex grid of shape (N1, N2, N3)."""
        x = np.ascontiguousarray(x, dtype=np.complex128).reshape(self.grid)
        out = np.zeros(self.grid, dtype=np.complex128)
        _check(self.lib.sgo_grid_fft(self.h, int(sign), x.ctypes.data_as(_dp), out.ctypes.data_as(_dp)),
               "sgo_grid_fft")
        return out

    def density_of(self, psi, occ):
        psi = np.ascontiguousarray(np.atleast_2d(psi), dtype=np.float64)
        occ = np.ascontiguousarray(occ, dtype=np.float64)
        r = np.zeros(self.grid)
        _check(self.lib.sgo_density(self.h, psi.shape[0], _ptr(psi), _ptr(occ), _ptr(r)), "sgo_density")
        return r


class Relax:
    """Local-relaxation driver of one structure (sgo_relax_*, see include/sgo.h): hand it the
    energy and forces at the positions it asks for; it answers with the next positions."""

    def __init__(self, cell, pos, method="pcg", **opts):
        self.lib = load_library()
        o = relax_opts(method, **opts)
        pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        self.natoms = len(pos)
        cell = np.ascontiguousarray(cell, dtype=np.float64).reshape(9)
        h = _vp()
        _check(self.lib.sgo_relax_create(self.natoms, _ptr(cell), _ptr(pos), ctypes.byref(o), ctypes.byref(h)),
               "sgo_relax_create")
        self.h = h

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.sgo_relax_destroy(h)
            self.h = None

    def positions(self):
        out = np.zeros((self.natoms, 3))
        _check(self.lib.sgo_relax_positions(self.h, _ptr(out)), "sgo_relax_positions")
        return out

    def step(self, energy, forces):
        """Returns (next positions, state): 0 evaluate them, 1 converged, 2 stopped."""
        f = np.ascontiguousarray(forces, dtype=np.float64).reshape(-1)
        out = np.zeros((self.natoms, 3))
        st = ctypes.c_int()
        _check(self.lib.sgo_relax_step(self.h, float(energy), _ptr(f), _ptr(out), ctypes.byref(st)), "sgo_relax_step")
        return out, st.value

    def best(self):
        """(energy, positions) of the lowest-energy configuration evaluated so far."""
        e = ctypes.c_double()
        out = np.zeros((self.natoms, 3))
        _check(self.lib.sgo_relax_best(self.h, ctypes.byref(e), _ptr(out)), "sgo_relax_best")
        return e.value, out

    def info(self):
        ev, st = ctypes.c_int(), ctypes.c_int()
        _check(self.lib.sgo_relax_info(self.h, ctypes.byref(ev), ctypes.byref(st)), "sgo_relax_info")
        return dict(evals=ev.value, state=st.value)


class Batch:
    """A population evaluated in lockstep (sgo_batch_create / sgo_energy_forces_batch)."""

    def __init__(self, ctxs: Sequence[Context]):
        self.lib = load_library()
        self.ctxs = list(ctxs)
        arr = (_vp * len(self.ctxs))(*[c.h for c in self.ctxs])
        h = _vp()
        _check(self.lib.sgo_batch_create(len(self.ctxs), arr, ctypes.byref(h)), "sgo_batch_create")
        self.h = h
        self.offsets = np.cumsum([0] + [3 * c.natoms for c in self.ctxs])

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.sgo_batch_destroy(h)
            self.h = None

    def energy_forces(self, pos: Optional[List[np.ndarray]] = None):
        n = len(self.ctxs)
        E = np.zeros(n)
        forces = [np.zeros((c.natoms, 3)) for c in self.ctxs]
        st = np.zeros(n, np.int32)
        fptr = (_dp * n)(*[_ptr(f) for f in forces])
        if pos is not None:
            keep = [np.ascontiguousarray(p, dtype=np.float64).reshape(-1) for p in pos]
            pptr = (_dp * n)(*[_ptr(p) for p in keep])
        else:
            pptr = None
        _check(self.lib.sgo_energy_forces_batch(self.h, pptr, _ptr(E), fptr, _ptr(st, ctypes.c_int)),
               "sgo_energy_forces_batch")
        return E, forces, st

    def timer(self, kernel: Optional[str]):
        """Time one kernel class live (CUDA events) during later calls; None stops."""
        _check(self.lib.sgo_batch_timer(self.h, None if kernel is None else kernel.encode()), "sgo_batch_timer")

    def timer_read(self):
        out = np.zeros(4)
        _check(self.lib.sgo_batch_timer_read(self.h, _ptr(out)), "sgo_batch_timer_read")
        return dict(ms=out[0], launches=int(out[1]), bytes=out[2], flops=out[3])

    def tuning(self):
        """GEMM tile knobs the batch's autotuner picked (see include/sgo.h)."""
        k = (ctypes.c_int * 3)()
        _check(self.lib.sgo_batch_tuning(self.h, k), "sgo_batch_tuning")
        return dict(tn_tc_k_chunk=k[0], nn_tc_tiles_per_cta=k[1], tn_simt_k_chunk=k[2])

    def launches(self) -> int:
        """Kernel launches issued since the previous call."""
        v = ctypes.c_longlong()
        _check(self.lib.sgo_batch_launches(self.h, ctypes.byref(v)), "sgo_batch_launches")
        return int(v.value)

    def relax(self, drivers: Sequence["Relax"], max_rounds: int = 100):
        """Relax every member with its driver (sgo_relax_batch); returns (rounds, statuses)."""
        arr = (_vp * len(drivers))(*[d.h for d in drivers])
        rounds = ctypes.c_int()
        st = np.zeros(len(drivers), np.int32)
        _check(self.lib.sgo_relax_batch(self.h, arr, int(max_rounds), ctypes.byref(rounds), _ptr(st, ctypes.c_int)),
               "sgo_relax_batch")
        return rounds.value, st

    def de_generation(self, cell, species, pop, f, u, scheme="random", d_min=2.0, max_rounds=40, method="pcg",
                      **relax):
        """One DE generation (sgo_de_generation): offspring, their relaxation on this batch,
        greedy selection.  Returns (pop, f, replaced, child energies), new arrays."""
        pop = np.array(pop, dtype=np.float64, order="C")
        f = np.array(f, dtype=np.float64)
        u = np.ascontiguousarray(u, dtype=np.float64)
        sp = np.ascontiguousarray(species, dtype=np.int32)
        cell = np.ascontiguousarray(cell, dtype=np.float64).reshape(9)
        rep = np.zeros(len(f), np.int32)
        cf = np.zeros(len(f))
        o = relax_opts(method, **relax)
        _check(self.lib.sgo_de_generation(self.h, _ptr(cell), _ptr(sp, ctypes.c_int), _ptr(pop), _ptr(f), _ptr(u),
                                          DE_SCHEMES[scheme], float(d_min), ctypes.byref(o), int(max_rounds),
                                          _ptr(rep, ctypes.c_int), _ptr(cf)), "sgo_de_generation")
        return pop, f, rep.astype(bool), cf

    def energy_forces_device(self, pos_dev, energies_dev, forces_dev, status_dev):
        """Device-pointer form: arguments are integer device addresses (e.g. tensor.data_ptr())."""
        _check(self.lib.sgo_energy_forces_batch_device(self.h, _vp(pos_dev), _vp(energies_dev), _vp(forces_dev),
                                                       _vp(status_dev)), "sgo_energy_forces_batch_device")


def _make_autograd():
    import torch

    class SgoEnergy(torch.autograd.Function):
        """E(R) with the hand-written Hellmann-Feynman adjoint as backward: dE/dR = -F.
        Valid at self-consistency (no differentiation through the SCF loop)."""

        @staticmethod
        def forward(ctx, sgo_context, pos):
            p = pos.detach().to("cpu", torch.float64).numpy()
            E, F = sgo_context.energy_forces(p)
            ctx.save_for_backward(torch.as_tensor(-F, dtype=pos.dtype, device=pos.device))
            return torch.as_tensor(E, dtype=pos.dtype, device=pos.device)

        @staticmethod
        def backward(ctx, grad):
            (dEdR,) = ctx.saved_tensors
            return None, grad * dEdR

    return SgoEnergy


def relax_autograd(ctx: "Context", driver: "Relax", max_evals: int = 100):
    """Local relaxation (Sec. II C) of one structure with its energy and gradient taken from
    SgoEnergy: the forward pass is the self-consistent energy, the backward pass the force
    adjoint (dE/dR = -F); the driver (PCG with the force-fitted preconditioner, CG or BFGS)
    turns them into the next positions.  Every evaluation after the first restarts from the
    previous density and wavefunctions.  Returns (state, evaluations): state 1 converged,
    2 stopped by the driver, 0 stopped at max_evals."""
    import torch
    pos = driver.positions()
    state, n = 0, 0
    ctx.set_warm(True)
    while state == 0 and n < max_evals:
        x = torch.tensor(pos, dtype=torch.float64, requires_grad=True)
        E = SgoEnergy.apply(ctx, x)
        E.backward()
        pos, state = driver.step(float(E.detach()), -x.grad.numpy())
        n += 1
    return state, n


class _Lazy:
    _cls = None

    def __getattr__(self, k):
        if _Lazy._cls is None:
            _Lazy._cls = _make_autograd()
        return getattr(_Lazy._cls, k)


SgoEnergy = _Lazy()
