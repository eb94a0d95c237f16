/*
 * sgo.h -- C ABI of the GB300 plane-wave DFT energy + force engine.
 *
 * The paper's bottom search level computes "the energy and atomic force of each
 * structure ... self-consistently" with a plane-wave DFT code on GPUs (Sec. II A,
 * Fig. 1 right module; Sec. II D).  Its inputs are the supercell, the atoms and
 * the plane-wave cutoff; every differential-evolution candidate (Sec. II B) and
 * every relaxation step (Sec. II C) calls it.  This library is that call.
 *
 * Physics (the paper names none; these are the fixed readings): Gamma point,
 * norm-conserving synthetic analytic pseudopotential per species (local
 * -Z erf(r/rc)/r + A exp(-r^2/sigma^2), one Kleinman-Bylander Gaussian s
 * projector of strength D, optionally three p projectors x_m exp(-r^2/(2 rp_p^2)) of
 * strength D_p), LDA (Slater + Perdew-Zunger 1981; or PBE), Ewald ions,
 * Fermi-Dirac smearing with the Mermin free energy F = E - kT S reported.
 * Units: Hartree atomic units (Ha, bohr).
 *
 * Conventions shared by every call:
 *  - The caller owns every host array passed in or out; the library copies
 *    inputs and never keeps a caller pointer after the call returns.
 *  - The library owns its device memory (allocated at sgo_create, released at
 *    sgo_destroy; cudaMalloc unless sgo_set_allocator installed the caller's
 *    allocator).  All device work is enqueued on the stream given to
 *    sgo_create; calls that return host results synchronise that stream only.
 *  - Errors are returned as sgo_status, never thrown; sgo_last_error() gives a
 *    message for the calling thread.  The library never exits the process.
 *  - A context is not thread-safe; different contexts may be used from
 *    different threads.
 *  - Grids exchanged with the caller are real arrays of shape (N1, N2, N3) in
 *    C order (index (i1*N2 + i2)*N3 + i3 = point sum_i (i_i/N_i) a_i).
 *  - Wave coefficients exchanged with the caller use the Gamma real packing of
 *    the half sphere: x[0] = c(0), x[1+2k] = sqrt2 Re c(G_k), x[2+2k] =
 *    sqrt2 Im c(G_k), for the half-sphere list G_k returned by sgo_get_basis
 *    (c(-G) = c(G)^* is implied).  Then x.y = <psi_x|psi_y> and sum x^2 = 1.
 */
#ifndef SGO_H
#define SGO_H

#include <stddef.h>

#if defined(__GNUC__)
#define SGO_API __attribute__((visibility("default")))
#else
#define SGO_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sgo_ctx sgo_ctx;     /* one structure: basis, tables, wavefunctions (opaque) */
typedef struct sgo_batch sgo_batch; /* a population of contexts evaluated in lockstep (opaque) */
typedef struct sgo_relax sgo_relax; /* the local-relaxation driver of one structure (opaque) */

typedef enum {
  SGO_OK = 0,
  SGO_ERR_ARG = 1,            /* invalid argument (sizes, pointers, band count, FFT size) */
  SGO_ERR_GEOMETRY = 2,       /* atoms closer than 0.5 bohr (minimum image), or non-finite positions */
  SGO_ERR_CUDA = 3,           /* a CUDA runtime call failed */
  SGO_ERR_OOM = 4,            /* device allocation failed */
  SGO_ERR_NOT_CONVERGED = 5,  /* SCF hit max_scf before the tolerances */
  SGO_ERR_TIMEOUT = 6,        /* a bounded device wait gave up */
  SGO_ERR_NAN = 7             /* a non-finite energy or force appeared */
} sgo_status;

/* Per-species pseudopotential parameters (bohr, Ha). */
typedef struct {
  double z_val;     /* valence charge Z */
  double rc;        /* erf width of the local Coulomb part */
  double a_sr;      /* amplitude A of the short-range Gaussian */
  double sigma_sr;  /* width sigma of the short-range Gaussian */
  double rp;        /* projector Gaussian width */
  double d_nl;      /* Kleinman-Bylander strength D */
  double rp_p;      /* p channel: width of the projectors x_m exp(-r^2/(2 rp_p^2)), m = x, y, z */
  double d_p;       /* p channel strength; 0 = no p channel (then rp_p is ignored) */
} sgo_species;

typedef struct {
  int precision;          /* 0 = plain FP64; 1 = mixed: FP32 FFT/H.psi/GEMM products and subspace
                             eigensolve, FP64 sums, energies, forces, Ewald, mixing */
  double kT;              /* Fermi-Dirac smearing, Ha; 0 = integer occupations (even N_el) */
  double scf_tol_e;       /* stop when |F_k - F_{k-1}| < scf_tol_e (Ha) ... */
  double scf_tol_rho;     /* ... and (Omega/N) sum |rho_out - rho_in| / N_el < scf_tol_rho */
  int max_scf;            /* SCF iteration cap */
  int pulay_hist;         /* Pulay (DIIS) history length, 1..8 */
  double mix_alpha;       /* Pulay step on the (Kerker-damped) residual */
  double kerker_q0;       /* Kerker q0 (1/bohr); 0 = no Kerker damping */
  int ncg;                /* all-band CG steps (Algorithm 1 iterations) per SCF iteration (default 2) */
  int ncg_first;          /* CG steps in each initial non-self-consistent iteration */
  int n_nonscf;           /* initial iterations at the fixed atomic-guess potential, before the
                             density is updated (default 0: the SCF cycle starts at once from the
                             atomic-guess density and the random wavefunctions; Pulay mixing
                             absorbs the first, poorly converged output densities) */
  int fft[3];             /* FFT grid; 0 = smallest 2^a 3^b 5^c >= 4 m_max + 1 per axis */
  unsigned long long seed;/* seed of the random initial wavefunctions */
  int gemm_tc;            /* mixed path: subspace/projector overlaps on tcgen05 tensor cores (3xTF32);
                             0 = FP32 CUDA cores */
  int graph;              /* batches: run the SCF loop as captured CUDA graphs, the self-consistent
                             iterations under a conditional WHILE node that the device ends
                             (1, default); 0 = one host launch per kernel and a host check per
                             iteration.  Results are identical.  Taken from the first member. */
  int autotune;           /* batches: time the GEMM tile candidates at creation and keep the fastest
                             (1, default); 0 = fixed defaults.  Taken from the first member. */
  int sub_batches;        /* batches in graph mode: split the members into this many sub-batches of
                             about equal work, each driven by its own graphs on its own stream so
                             that their kernels overlap on the GPU; 0 = automatic (3 from 24
                             members on, 2 from 16, else 1).  With the same GEMM knobs
                             (autotune = 0) every member's results are bit-identical in every
                             split; the autotuner tunes each sub-batch on its own.  Taken from
                             the first member. */
  double eig_tol;         /* Algorithm 1 runs its CG loop "while not converged": after the SCF
                             stopping rule holds, all-band CG steps continue at the final
                             potential until every band with occupation above 1e-6 has a
                             residual |H psi - eps psi| below eig_tol (Ha), then the density,
                             energy and forces are taken from those bands (default 1e-4;
                             0 = stop with the last SCF iteration's bands) */
  int max_polish;         /* cap on those extra CG steps (default 40); a member that reaches it
                             keeps its bands and reports the residual it reached (sgo_get_stats) */
  int rr_fp64;            /* mixed path: factor the overlap (Cholesky) and solve the subspace
                             eigenproblem in FP64 (1) instead of FP32 deviation form (0, default;
                             taken from the first member of a batch) */
  double watchdog_ms;     /* bound on every device wait of the tensor-core kernels (ms); on expiry
                             the member reports SGO_ERR_TIMEOUT and the context stays usable;
                             0 = 2000 ms.  Taken from the first member of a batch. */
  int extra_bands;        /* empty bands the eigensolver carries above the nbands requested ones:
                             the all-band CG converges the top bands of its block slowest, so the
                             requested bands get headroom; occupations, eigenvalues, energies and
                             the eig_tol test cover the requested bands only (-1, default:
                             4 + nbands / 32; 0 = none) */
  int rr_cluster;         /* subspace diagonalisation kernel: -1 (default) one CTA per member while
                             its matrices fit in shared memory, else a thread-block cluster of 8
                             CTAs per member; 0 = always one CTA (over a global scratch when the
                             matrices do not fit); 1 = always the cluster.  Taken from the first
                             member of a batch. */
  int eigensolver;        /* 0 (default): Algorithm 1's all-band CG steps (Sec. II D): per band a
                             preconditioned, conjugated, projected search direction, a line
                             minimisation, then a Rayleigh-Ritz over the n_b bands.  1: block
                             Davidson steps: the preconditioned residuals W of all bands, projected
                             and normalised, and one Rayleigh-Ritz over the 2 n_b block [X, W]
                             keeping the lowest n_b Ritz pairs (its Cholesky and eigensolve are
                             8x the n_b ones; a W direction nearly inside the span of the
                             others is left out).  Needs 2 n_b <= the plane-wave count (else
                             SGO_ERR_ARG at sgo_create).  Same stopping rules; all members of a
                             batch must agree (else SGO_ERR_ARG at sgo_batch_create). */
  int xc;                 /* exchange-correlation: 0 (default) LDA (Slater + Perdew-Zunger 1981);
                             1 PBE (Perdew, Burke & Ernzerhof 1996, on Perdew-Wang 1992 uniform-gas
                             correlation), the functional of the paper's searches (Sec. III): its
                             potential de/drho - div(2 de/dsigma grad rho) takes the gradient and
                             the divergence in G space on the FFT box (five extra grid transforms
                             per potential, two per energy).  All members of a batch must agree
                             (else SGO_ERR_ARG at sgo_batch_create). */
  double cg_adapt;        /* SCF iterations whose density residual (the previous iteration's) is
                             above cg_adapt take ncg - 1 CG steps, the others ncg: the eigensolver
                             works harder as the density converges.  0 = always ncg.  Default
                             0 (taken from the first member of a batch). */
  int kgrid[3];           /* Brillouin-zone sampling (the rough k-point grids of the relaxations,
                             Sec. II C): the Gamma-centred Monkhorst-Pack mesh k = sum_i (t_i/n_i) b_i,
                             t_i = 0..n_i-1, weights 1/(n1 n2 n3).  Computed by zone folding: the
                             context holds the n1 x n2 x n3 supercell at the Gamma point, whose
                             plane waves are exactly the k + G of the mesh, so its energy per cell,
                             forces and spectrum are those of the mesh (same cutoff; nbands per k
                             point on average).  The caller keeps passing and receiving the cell's
                             natoms positions and forces; energies (sgo_energy_forces, sgo_get_terms)
                             are per cell; nbands, the eigenvalues, states, grids and the component
                             calls are the supercell's (n1 n2 n3 times nbands, fft[i] times n_i when
                             given).  Entries <= 0 count as 1; {1, 1, 1} (default) = the Gamma point.
                             sgo_energy_forces_batch_device refuses such contexts (SGO_ERR_ARG). */
} sgo_opts;

/* Device memory through the caller's allocator.  The library's device buffers (context
 * arenas, batch tables and scratch, the temporaries of the component calls) come from
 * alloc(bytes, stream, user), which returns a device pointer or NULL, and go back through
 * release(ptr, stream, user) -- for instance PyTorch's caching allocator, so that the
 * library's memory is part of the caller's pool and its budget (the binding's
 * use_torch_allocator()).  Process-wide; contexts and batches created after the call use it;
 * every block is returned to the allocator that gave it, after a device synchronisation.
 * alloc = release = NULL restores cudaMalloc/cudaFree.  SGO_ERR_ARG if exactly one is NULL.
 * Pinned host buffers stay cudaMallocHost. */
typedef void* (*sgo_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*sgo_free_fn)(void* ptr, void* stream, void* user);
SGO_API sgo_status sgo_set_allocator(sgo_alloc_fn alloc, sgo_free_fn release, void* user);

/* Fill *o with the defaults (FP64, kT 0, tolerances 1e-8 Ha / 1e-7, Pulay 8, ...). */
SGO_API void sgo_opts_default(sgo_opts* o);

/* Build a context for one structure (Sec. II D inputs: cell, species, positions, cutoff).
 * cell: 9 doubles, rows are the lattice vectors a_i (bohr).  sp: nspecies entries.
 * species_of_atom: natoms indices into sp.  pos: natoms*3 Cartesian bohr.
 * ecut: |G|^2/2 <= ecut (Ha).  nbands >= N_el/2 (integer occupations) or > N_el/2 (kT > 0).
 * cuda_stream: a cudaStream_t (NULL = the legacy default stream).
 * With o->kgrid above {1, 1, 1} the context is the folded supercell (see sgo_opts.kgrid).
 * Allocates all device memory of the context; *out is NULL on error. */
SGO_API sgo_status sgo_create(const double cell[9], int nspecies, const sgo_species* sp, int natoms,
                      const int* species_of_atom, const double* pos, double ecut, int nbands,
                      const sgo_opts* o, void* cuda_stream, sgo_ctx** out);

/* Run the SCF cycle of Sec. II D (rho_in -> Kohn-Sham solve by the all-band CG of
 * Algorithm 1 -> rho_out -> Pulay mixing) at positions pos (NULL = keep the current
 * ones).  Starts from the atomic-guess density and random wavefunctions unless
 * sgo_set_warm(ctx, 1) was called.  Outputs (may be NULL): SCF iterations, final
 * density residual.  Returns SGO_ERR_NOT_CONVERGED if max_scf was reached. */
SGO_API sgo_status sgo_scf(sgo_ctx* ctx, const double* pos, int* n_iter_out, double* resid_out);

/* One energy + force evaluation: sgo_scf at pos, then the Hellmann-Feynman forces
 * -dF/dR (local, nonlocal, Ewald).  energy: the free energy F (Ha).  forces:
 * natoms*3 (Ha/bohr).  Either output may be NULL. */
SGO_API sgo_status sgo_energy_forces(sgo_ctx* ctx, const double* pos, double* energy, double* forces);

/* A population of n contexts (same precision and eigensolver options, else SGO_ERR_ARG)
 * evaluated together: every kernel launch covers all members still iterating (Sec. II D:
 * one relaxation per GPU becomes one population per GPU).  The contexts stay owned by the
 * caller and must outlive the batch. */
SGO_API sgo_status sgo_batch_create(int n, sgo_ctx* const* ctxs, sgo_batch** out);

/* The GEMM tile knobs the batch's autotuner picked when the batch was created (mixed path;
 * the defaults otherwise): knobs[0] = K chunk of the tensor-core TN GEMM (of 256, 512, 1024,
 * 2048), knobs[1] = 128-wave tiles per tensor-core NN CTA (of 2, 4, 8, 16), knobs[2] = K
 * chunk of the CUDA-core TN GEMM (of 128, 256, 512).  Each candidate is timed on the batch's
 * own buffers; the fastest is kept.  A batch split into sub-batches tunes each on its own;
 * knobs are those of the first sub-batch (the one given the costliest member). */
SGO_API sgo_status sgo_batch_tuning(const sgo_batch* batch, int* knobs);

/* Evaluate every member.  pos[i] (host, natoms_i*3) or NULL = keep; energies[i];
 * forces[i] (host, natoms_i*3, may be NULL); per_item[i] = status of member i.
 * Returns SGO_OK when the call itself ran, even if some members failed. */
SGO_API sgo_status sgo_energy_forces_batch(sgo_batch* b, const double* const* pos, double* energies,
                                   double* const* forces, sgo_status* per_item);

/* Same as sgo_energy_forces_batch with every array in DEVICE memory: pos_dev
 * (sum natoms_i*3 doubles, members back to back), energies_dev (n), forces_dev
 * (sum natoms_i*3), status_dev (n ints).  Synchronises the batch stream.  SGO_ERR_ARG for a
 * batch with a k-point member (sgo_opts.kgrid): use sgo_energy_forces_batch. */
SGO_API sgo_status sgo_energy_forces_batch_device(sgo_batch* b, const double* pos_dev, double* energies_dev,
                                          double* forces_dev, int* status_dev);

/* Live timing of one kernel class during later batch calls: CUDA events are recorded
 * on the batch stream around every launch of that class.  kernel: "plane_vpsi",
 * "wave_to_cols", "cols_to_wave", "plane_density", "gemm_tn", "gemm_nn", "rr", "grid_fft",
 * "cg_band", "grid_other", "gemm_small", or NULL to stop.  Resets the accumulators.  Instrumentation, not part of the method. */
SGO_API sgo_status sgo_batch_timer(sgo_batch* b, const char* kernel);

/* Read and keep accumulating: out[0] total ms, out[1] launches, out[2] algorithmic
 * bytes, out[3] algorithmic flops of the timed launches (active members only). */
SGO_API sgo_status sgo_batch_timer_read(sgo_batch* b, double out[4]);

/* Kernel launches the batch issued since the previous call (then reset to 0). */
SGO_API sgo_status sgo_batch_launches(sgo_batch* b, long long* count);

/* Eigenvalues and occupations of the last SCF (nbands doubles each; either may be NULL).
 * A k-point context (sgo_opts.kgrid): the supercell's n1 n2 n3 nbands states, i.e. the band
 * energies eps_n(k) of the whole mesh in ascending order, occupations 0..2 each. */
SGO_API sgo_status sgo_get_eigen(sgo_ctx* ctx, double* eig, double* occ);

/* Energy terms of the last SCF: kinetic, nonlocal, local, Hartree, xc, Ewald, -kT S, F
 * (per cell of the caller for a k-point context). */
SGO_API sgo_status sgo_get_terms(sgo_ctx* ctx, double terms[8]);

/* Sizes: info[0] npw (real length of a band vector), [1] n_half (G != 0 half sphere),
 * [2] column pairs, [3..5] N1 N2 N3, [6] nbands, [7] natoms, [8] scf iterations of the
 * last SCF, [9] precision.  A k-point context: [0..6] are the folded supercell's, [7] the
 * caller's cell's atom count. */
SGO_API sgo_status sgo_get_info(sgo_ctx* ctx, int info[10]);

/* Diagnostics of the last SCF: [0] iterations, [1] Jacobi sweeps summed over its
 * subspace diagonalisations, [2] final density residual, [3] final |F_k - F_{k-1}|,
 * [4] CG steps taken after the SCF stopping rule held (eig_tol), [5] the largest residual
 * |H psi - eps psi| over the bands with occupation above 1e-6 at the end, [6] subspace
 * diagonalisations that stopped at their Jacobi sweep cap, [7] SCF iterations of the
 * last SCF loop that started from a state set by sgo_set_state (0 otherwise). */
SGO_API sgo_status sgo_get_stats(sgo_ctx* ctx, double stats[8]);

/* Warm-start state (Sec. II C: a relaxation step restarts the SCF from the previous
 * step's density and wavefunctions), for moving a state between contexts or processes:
 *   rho_g: the SCF input density rho_in(G) = (1/N) sum_r rho_in(r) exp(-i G.r) on the FFT
 *          box, complex, 2*N1*N2*N3 doubles (re, im interleaved) in C order of
 *          (m1 mod N1, m2 mod N2, m3 mod N3);
 *   psi:   the nbands wavefunctions, row-major nbands x npw doubles in the packed Gamma
 *          format above (sizes from sgo_get_info).
 * sgo_get_state copies the state the last evaluation left (either pointer may be NULL;
 * SGO_ERR_ARG before any evaluation or sgo_set_state).  sgo_set_state installs one (both
 * required; SGO_ERR_ARG for non-finite values) and switches warm starts on, as
 * sgo_set_warm(ctx, 1): the next evaluation starts from it, whatever the positions.  The
 * wavefunctions need not be orthonormal (the first subspace diagonalisation
 * orthonormalises them); both are copied, the caller keeps its arrays. */
SGO_API sgo_status sgo_get_state(sgo_ctx* ctx, double* rho_g, double* psi);
SGO_API sgo_status sgo_set_state(sgo_ctx* ctx, const double* rho_g, const double* psi);

/* Miller indices of the packed basis: (1 + n_half) rows of 3 ints, row 0 = G = 0. */
SGO_API sgo_status sgo_get_basis(sgo_ctx* ctx, int* miller);

/* The last output density rho_out (N1*N2*N3 doubles, C order). */
SGO_API sgo_status sgo_get_density(sgo_ctx* ctx, double* rho);

/* H psi for nvec packed vectors (row-major nvec x npw doubles) with the local
 * potential veff (N1*N2*N3 doubles, C order) and the projectors of the current
 * positions: kinetic + local (FFT path) + nonlocal, in the context's precision.
 * nvec <= nbands.  A component test of the H.psi kernels of Algorithm 1. */
SGO_API sgo_status sgo_apply_hamiltonian(sgo_ctx* ctx, const double* veff, int nvec, const double* psi,
                                 double* hpsi);

/* The H psi of sgo_apply_hamiltonian, for callers that cannot let a library allocate
 * device memory during a call: a process whose device memory belongs to its own pool
 * allocator, one that runs under a fixed memory budget, or a latency-critical loop that
 * cannot take the implicit synchronisation of cudaMalloc/cudaFree.  In FP64 the result
 * equals sgo_apply_hamiltonian's; on the mixed path this call always takes the CUDA-core
 * transforms and GEMMs while the ordinary call may take the register-FFT and tensor-core
 * kernels, so the two agree to FP32/3xTF32 rounding (about 2e-5 relative).  The device
 * current at the call must be the context's (the one current at sgo_create), else
 * SGO_ERR_ARG.  This call
 * allocates nothing: it uses the context's buffers (allocated once by sgo_create) and a
 * file-scope device scratch array of 32 MiB that every GPU loading the library holds
 * until the process exits.  Problems whose launch descriptors, projector partial sums
 * and staged veff, psi and hpsi exceed 32 MiB return SGO_ERR_ARG with a message.  The
 * first call on each device looks up the array's device address (with that device
 * current); make that first call before any stream capture.  All calls share the array
 * and leave their contents in it; calls that overlap on the GPU race with each other.
 * There is no counterpart in the paper: this is a deployment variant of the H.psi apply. */
SGO_API sgo_status sgo_apply_hamiltonian_noalloc(sgo_ctx* ctx, const double* veff, int nvec, const double* psi,
                                                 double* hpsi);

/* C = X^T Y (nvec x nvec, row-major) for nvec packed vectors X, Y (row-major nvec x npw):
 * the subspace-matrix GEMM of Algorithm 1 (H(i,j), overlaps, projection coefficients), in
 * the context's precision (mixed: FP32 operands on the tensor cores unless gemm_tc = 0;
 * FP64 sums). */
SGO_API sgo_status sgo_subspace_matrix(sgo_ctx* ctx, int nvec, const double* x, const double* y, double* c);

/* Y <- alpha M^T X + beta Y, i.e. y_j <- alpha sum_i m[i][j] x_i + beta y_j, for nvec packed
 * vectors X, Y (row-major nvec x npw; y is read and overwritten) and m row-major nvec x
 * nvec: the block update of Algorithm 1 (the rotation Psi <- Psi U by the Rayleigh-Ritz
 * eigenvectors, the projection P <- P - Psi (Psi^T P)), in the context's precision (mixed:
 * FP32 operands on the tensor cores unless gemm_tc = 0).  SGO_ERR_ARG for null pointers or
 * nvec outside 1..nbands. */
SGO_API sgo_status sgo_block_update(sgo_ctx* ctx, int nvec, const double* x, const double* m, double alpha,
                                    double beta, double* y);

/* One 3D transform of the SCF's grid FFT (Sec. II D: the potential from rho_in(G), rho_out(G)
 * from rho_out(r)) on a complex grid: in and out are N1*N2*N3 complex values, C order,
 * interleaved (re, im) doubles, caller-owned host memory.  sign -1: out(m) = sum_j in(j)
 * exp(-2 pi i m.j / N) per axis (r -> G); sign +1: the same with +i (G -> r), unnormalised.
 * Arithmetic: FP64 on the plain path; float-float (two FP32 numbers per value, about 44
 * bits) on the mixed path, whose FP64 grids it serves.  SGO_ERR_ARG for null pointers or a
 * sign other than +-1. */
SGO_API sgo_status sgo_grid_fft(sgo_ctx* ctx, int sign, const double* in, double* out);

/* rho(r) = sum_n occ_n |psi_n(r)|^2 for nvec packed vectors (the density kernels). */
SGO_API sgo_status sgo_density(sgo_ctx* ctx, int nvec, const double* psi, const double* occ, double* rho);

/* Warm start: when on (1), the next sgo_scf starts from the previous rho_in and
 * wavefunctions instead of the atomic guess (relaxation steps, Sec. II C). */
SGO_API sgo_status sgo_set_warm(sgo_ctx* ctx, int on);

/* ---- local relaxation (Sec. II C) ----------------------------------------------------
 * A host-side driver that moves one structure to its nearest local minimum from energies
 * and forces the caller evaluates (sgo_energy_forces_batch, or anything else).
 *   SGO_RELAX_PCG: nonlinear preconditioned CG; the preconditioner is the inverse Hessian
 *     of a classical force field fitted to the DFT forces (a shifted-force Morse pair
 *     potential over periodic images within rc, parameters fitted by Levenberg-Marquardt
 *     to every force set of the relaxation so far), from the second-order finite
 *     difference of the fitted energy, without the three translational eigenpairs:
 *     P = sum_j V_j V_j^T / |tau_j|, |tau_j| floored at 0.02 max|tau|.  Fit and P are
 *     renewed every `refit` directions.
 *   SGO_RELAX_CG: the same iteration with P = I / 0.5 (Ha/bohr^2).
 *   SGO_RELAX_BFGS: inverse-Hessian BFGS from B0 = I / 0.5, steps capped per atom.
 * (P)CG directions are Polak-Ribiere+ with restarts; each line takes a trial point at
 * min(a_prev, max_step / max_i |d_i|), a_prev the previous line's minimising step (1 on the
 * first line), and, unless the secant of the directional derivative
 * lands within `accept` of it, one more evaluation at the secant's zero (kept between
 * 0.1 times the trial step and max_step of displacement). */
enum { SGO_RELAX_PCG = 0, SGO_RELAX_CG = 1, SGO_RELAX_BFGS = 2 };
typedef struct {
  int method;        /* SGO_RELAX_PCG, _CG or _BFGS */
  double fmax;       /* converged when every atom's |F| < fmax (Ha/bohr) */
  double max_step;   /* largest displacement of an atom per line or step (bohr) */
  int refit;         /* PCG: renew the force-field fit and preconditioner every refit directions */
  double rc;         /* force-field cutoff (bohr) */
  double accept;     /* keep the trial point when the line minimum is within accept of it */
  int max_evals;     /* stop after this many evaluations */
} sgo_relax_opts;

/* Defaults: PCG, fmax 1e-3 Ha/bohr, max_step 0.3 bohr, refit 3, rc 8 bohr, accept 0.1,
 * 60 evaluations. */
SGO_API void sgo_relax_opts_default(sgo_relax_opts* o);

/* A driver for natoms atoms in the cell (9 doubles, rows a_i, bohr) starting at pos
 * (natoms*3 Cartesian bohr, copied).  o may be NULL (defaults).  SGO_ERR_ARG for bad
 * sizes, pointers or options. */
SGO_API sgo_status sgo_relax_create(int natoms, const double cell[9], const double* pos, const sgo_relax_opts* o,
                                    sgo_relax** out);

/* Hand the driver the energy (Ha) and forces (natoms*3, Ha/bohr) at the positions it asked
 * for last (the starting positions first).  It writes the next positions to evaluate to
 * next_pos (natoms*3) and *state (may be NULL): 0 = evaluate next_pos, 1 = converged
 * (next_pos = the converged positions), 2 = stopped without convergence (evaluation
 * budget spent; next_pos = the last evaluated positions).  Calls after the end repeat
 * the final positions.  SGO_ERR_NAN for non-finite forces. */
SGO_API sgo_status sgo_relax_step(sgo_relax* r, double energy, const double* forces, double* next_pos, int* state);

/* The positions the driver asks to evaluate next (natoms*3; the starting positions before
 * the first step, the final ones once it has stopped). */
SGO_API sgo_status sgo_relax_positions(const sgo_relax* r, double* pos);

/* The lowest-energy configuration evaluated so far: its energy and positions (either may
 * be NULL).  SGO_ERR_ARG before the first step. */
SGO_API sgo_status sgo_relax_best(const sgo_relax* r, double* energy, double* pos);

/* Evaluations consumed so far and the state (as sgo_relax_step reports it). */
SGO_API sgo_status sgo_relax_info(const sgo_relax* r, int* evals, int* state);

/* Relax every member of a batch together: relax[i] drives member i (same atom count).
 * Each round evaluates all members at the positions their drivers ask for with one
 * sgo_energy_forces_batch call (warm-started from the previous density and wavefunctions
 * after the first round) and steps the drivers of the members still relaxing; ends when
 * every driver has stopped or after max_rounds rounds.  per_item (may be NULL) receives
 * each member's evaluation status (SGO_OK while its evaluations succeed; a member whose
 * evaluation fails stops relaxing); *rounds (may be NULL) the rounds run.  Returns
 * SGO_OK when the calls ran, SGO_ERR_CUDA on a CUDA failure, SGO_ERR_ARG for bad input. */
SGO_API sgo_status sgo_relax_batch(sgo_batch* b, sgo_relax* const* relax, int max_rounds, int* rounds,
                                   sgo_status* per_item);

SGO_API void sgo_relax_destroy(sgo_relax* r);

/* ---- global search: differential evolution (Sec. II B) --------------------------------
 * A population of np >= 4 structures with the same atoms (species fixed per atom slot) in
 * one cell (9 doubles, rows a_i, bohr); pop is np x natoms x 3 Cartesian bohr, f the np
 * relaxed free energies.  For each individual i, with the SGO_DE_RANDOMS uniforms
 * u[i][0..6] in [0, 1) (the caller draws them):
 *   partners r1, r2, r3: distinct and != i, drawn without replacement by u[i][0..2];
 *   triangle mutation (Eq. 2): V = (X1+X2+X3)/3 + (p2-p1)(X1-X2) + (p3-p2)(X2-X3)
 *     + (p1-p3)(X3-X1), p_k = |f_k| / sum |f|, in fractional coordinates with
 *     minimum-image differences from X1, wrapped into the cell;
 *   cut-and-splice crossover of V (kept side) and X_i (fill): SGO_DE_PLANE keeps V's atoms
 *     above a plane through its centre (normal from u[i][3..4], uniform on the sphere) and
 *     fills each species with X_i's atoms of lowest projection on the normal;
 *     SGO_DE_SPHERE keeps V's atoms within u[i][6] times V's largest distance from its
 *     centre and fills with X_i's atoms farthest from X_i's centre; SGO_DE_RANDOM_SCHEME
 *     picks the plane when u[i][5] < 1/2, else the sphere;
 *   repair: pairs closer than d_min (minimum image) are pushed apart in passes.
 * Children keep the species of each slot. */
enum { SGO_DE_RANDOM_SCHEME = 0, SGO_DE_PLANE = 1, SGO_DE_SPHERE = 2 };
#define SGO_DE_RANDOMS 7
SGO_API sgo_status sgo_de_offspring(int np, int natoms, const double cell[9], const int* species, const double* pop,
                                    const double* f, const double* u, int scheme, double d_min, double* children);

/* Migration between nsub equal subpopulations (consecutive slices of the np individuals;
 * np a multiple of nsub), in ring order: the best individual of subpopulation s replaces the
 * worst of subpopulation (s+1) mod nsub when its energy is lower (pop and f updated in place;
 * ties: the lowest index is best, the lowest index is worst).  Every best and worst is chosen
 * on the population as passed in, before any copy, so a migrant moves one step round the
 * ring; nsub = 1 changes nothing. */
SGO_API sgo_status sgo_de_migrate(int np, int nsub, int natoms, double* pop, double* f);

/* Similarity check between two structures of natoms atoms in one cell (the population's
 * initialisation keeps only dissimilar ones): *similar = 1 when the root-mean-square
 * difference of their sorted minimum-image pair distances is below tol (bohr). */
SGO_API sgo_status sgo_de_similar(int natoms, const double cell[9], const double* a, const double* b, double tol,
                                  int* similar);

/* One DE generation on a batch whose member i evaluates individual i (same atoms, same
 * cell): the offspring above, each relaxed (cold start, then warm) by its own driver with
 * options ro over at most max_rounds batched evaluations, then greedy selection: the
 * lowest-energy configuration of child i's relaxation replaces pop[i], f[i] when lower.
 * replaced (may be NULL) receives 1 where it did; child_f (may be NULL) the children's
 * energies (+inf where a child's evaluation failed).  SGO_ERR_ARG for bad input,
 * SGO_ERR_CUDA on a CUDA failure. */
SGO_API sgo_status sgo_de_generation(sgo_batch* b, const double cell[9], const int* species, double* pop, double* f,
                                     const double* u, int scheme, double d_min, const sgo_relax_opts* ro,
                                     int max_rounds, int* replaced, double* child_f);

SGO_API void sgo_batch_destroy(sgo_batch* b);
SGO_API void sgo_destroy(sgo_ctx* ctx);
SGO_API const char* sgo_status_string(sgo_status s);
SGO_API const char* sgo_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SGO_H */
