// Kernel launch interface between the host engine and the device kernels.
#pragma once

#include "sgo_internal.cuh"

namespace sgo {

// FFT kernel geometry
constexpr int QCP = 8;                 // column pairs per z-column CTA (<= 16 columns)
constexpr int ZCOL_THREADS = 128;
constexpr int QZ = 32;                 // grid columns per z CTA
constexpr int PLANE_THREADS = 256;      // threads of the z-plane kernels
constexpr int PLANE_MIN_BLOCKS = 4;     // register cap (64) for 4+ resident CTAs per SM
constexpr int PLANE_THREADS_MAX = PLANE_THREADS;
constexpr int PLANE_REG_THREADS = 256;  // register-FFT plane kernel (mixed path)
constexpr int PLANE_REG_MAXN = 72;      // longest x / y / z line it transforms
constexpr int PLANE_PAIR_GROUP = 8;     // band pairs per register plane CTA
constexpr int PAIR_REG_MAXN = 128;      // longest line a lane pair transforms
constexpr int ZREG_CP = 64;             // column pairs per register z-column CTA
constexpr int ZREG_THREADS = 2 * ZREG_CP;
// GEMM geometry
constexpr int TN_TILE = 64;
constexpr int TN_KC = 256;             // K chunk of one split-K partial (CUDA-core GEMM)
constexpr int TC_KC = 512;             // K chunk of one split-K partial (tensor-core GEMM)
constexpr int NN_RT = 4;              // row tiles of 64 per NN CTA
constexpr int NN_KP = 128;             // rows of the small matrix staged per pass
constexpr int BAND_THREADS = 256;
constexpr int GRID_CHUNK = 4096;       // grid points per reduction CTA
constexpr int RR_THREADS = 1024;
constexpr int RR_CLUSTER = 8;          // CTAs of the cluster Rayleigh-Ritz (large subspaces)
constexpr int LF_GROUP = 4;            // atoms per local-force CTA

struct KArgs {
  const Prob* probs;
  const int* start;
  int nprob;
  const int* active;
};

struct Launch {
  KArgs ka;
  WorkMap map;
  cudaStream_t stream;
  int max_n1, max_n2, max_n3, max_n12, max_nb;
  int plane_threads;
  long long wait_ns = 2000000000LL;  // bound of the tensor-core kernels' device waits (watchdog)
};

// operands of the subspace GEMMs
enum { OPK_WB = 0, OPK_B = 1, OPK_DB = 2 };
// Up to four (source role, destination role) pairs that one NN launch maps through the same
// small matrix (grid dimension y = pair); also the role pairs one swap kernel exchanges.
struct RolePairs {
  int n;
  int a[4];
  int y[4];
};
inline RolePairs role_pair(int a, int y) { return RolePairs{1, {a, 0, 0, 0}, {y, 0, 0, 0}}; }
enum { DD_S = 0, DD_HS, DD_CM, DD_TM, DD_PROJ, DD_DPROJ, DD_PROJ_D };

// k_fft.cu
template <typename T> void launch_wave_to_cols(const Launch& L, int src);
template <typename T> void launch_cols_to_wave(const Launch& L, int src, int dst);
template <typename T> void launch_plane_vpsi(const Launch& L);
template <typename T> void launch_plane_density(const Launch& L, const double* occ_override);
// grid transforms of the work grids (T = double; T = float views the first half of the
// same memory as single-precision complex)
// T: float (FP32 grids), double (FP64), ff (float-float arithmetic on FP64 grids, ff.cuh)
struct ff;
template <typename T> void launch_grid_plane_fft(const Launch& L, int which, int sign);
template <typename T> void launch_grid_z_fft(const Launch& L, int which, int sign);
template <typename T> void launch_grid_line_fft(const Launch& L, int which, int sign, int axis);  // axis 0: x, 1: y
void fft_set_smem_limits(size_t bytes);
// plane pass by line blocks through a global buffer (planes too large for one CTA)
int big_y_ctas(int npair, int n3, int m1max);
int big_x_ctas(int npair, int n3, int n2);
int big_density_ctas(int n3, int n2);
size_t big_plane_bytes(int npair, int n3, int m1max, int n2, size_t tsize);
template <typename T> void launch_big_y(const Launch& L, int dir, int skip_empty, const double* occ_override);
template <typename T> void launch_big_x(const Launch& L);
template <typename T> void launch_big_density(const Launch& L, const double* occ_override);
// register-FFT plane pass (mixed path): lengths n1, n2 with a register transform
bool plane_reg_ok(int n1, int n2);
// multi-pass plane pass (k_plane_ms.cu): the register lengths' H.psi plane pass as two passes
// of short register DFTs per line over whole planes in shared memory
constexpr bool kPlaneMultiPass = true;
#ifndef PLANE_MS_THREADS
#define PLANE_MS_THREADS 256  // threads of a multi-pass plane CTA
#endif
#ifndef PLANE_MS_MINB
#define PLANE_MS_MINB 3       // CTAs per SM the register budget is sized for
#endif
#ifndef PLANE_MS_BUDGET_KB
#define PLANE_MS_BUDGET_KB 54  // shared memory for the planes of one CTA
#endif
#ifndef PLANE_MS_PAIRS
#define PLANE_MS_PAIRS 8       // band pairs per multi-pass plane CTA (V_eff loaded once for them)
#endif
int plane_ms_ctas(int n1, int n2, int n3, int npair);
size_t plane_ms_smem(int n1, int n2, int n3);
void launch_plane_vpsi_ms(const Launch& L, size_t smem);
bool plane_ms_init();
void plane_ms_set_smem_limits(size_t bytes);
int plane_reg_class(int n1, int n2);          // 0: both <= 40, 1: up to PLANE_REG_MAXN
int plane_reg_ctas(int n2, int n3, int npair);
size_t plane_reg_smem(int n1, int n2, int m1max);
bool fft_reg_init();                          // twiddle tables on the current device
bool plane_vpsi_reg_init();
bool plane_density_reg_init();
void plane_vpsi_reg_set_smem_limits(size_t bytes);
void plane_density_reg_set_smem_limits(size_t bytes);
// register-FFT z-column passes (mixed path), k_cols_reg.cu
int zreg_class(int n3);
bool zreg_ok(int n3);
int zreg_ctas(int ncp, int npair);
size_t zreg_smem(int n3);
void launch_wave_to_cols_reg(const Launch& L, int cls, size_t smem, int src);
void launch_cols_to_wave_reg(const Launch& L, int cls, size_t smem, int src, int dst);
bool zreg_init();
void zreg_set_smem_limits(size_t bytes);
// lane-pair register FFT passes for lengths 96 ... 128 (mixed path), k_pair_reg.cu
bool pair_plane_ok(int n1, int n2);
int pair_plane_ctas(int n2, int n3, int npair);
size_t pair_plane_smem(int n1, int n2, int m1max);
int pair_density_ctas(int n2, int n3);
size_t pair_density_smem(int n1, int n2, int m1max);
bool zpair_ok(int n3);
int zpair_ctas(int ncp, int npair);
size_t zpair_smem(int n3);
void launch_plane_vpsi_pair(const Launch& L, size_t smem);
void launch_plane_density_pair(const Launch& L, size_t smem, const double* occ_override);
void launch_wave_to_cols_pair(const Launch& L, size_t smem, int src);
void launch_cols_to_wave_pair(const Launch& L, size_t smem, int src, int dst);
bool pair_reg_init();
void pair_reg_set_smem_limits(size_t bytes);
void launch_plane_vpsi_reg(const Launch& L, int cls, size_t smem);
size_t plane_density_reg_smem(int n1, int n2, int m1max);
int plane_density_reg_ctas(int n2, int n3);
void launch_plane_density_reg(const Launch& L, int cls, size_t smem, const double* occ_override);

// k_linalg.cu
template <typename T>
void launch_gemm_tn(const Launch& L, int akind, int arole, int bkind, int brole, double* part, size_t stride,
                    int kc = TN_KC);
// sym: the partials are k_gemm_tn's A^T A (same operand twice; tiles below the diagonal mirrored)
void launch_gemm_tn_reduce(const Launch& L, int akind, int bkind, int dst, const double* part, size_t stride,
                           int kc = TN_KC, bool sym = false);
// k_gemm_tc.cu (tcgen05 + TMA, mixed path, operand counts <= 128)
constexpr int TC_NSLOT = NWB + 2;      // tensor maps per problem: wave buffers, B, dB
constexpr int TC_NMAPKIND = 2;         // box 32 x 128 rows (TN), 32 x 32 rows (NN)
constexpr int NN_TPC = 4;              // 128-wave tiles per NN CTA
size_t tc_map_bytes();
bool tc_encode_maps(const Prob& d, void* host_maps);  // TC_NSLOT * TC_NMAPKIND maps of one problem
int nn_tc_image_bytes(int nin, int nb);
int nn_tc_stages(int img_bytes);
void launch_gemm_tn_tc(const Launch& L, const void* maps, int akind, int arole, int bkind, int brole, double* part,
                       size_t stride, int kc = TC_KC);
void launch_nn_image(const Launch& Lprob, int akind, int msel, float* img, size_t img_stride);
void launch_gemm_nn_tc(const Launch& L, const void* maps, const float* img, size_t img_stride, int img_max,
                       int akind, const RolePairs& rp, double alpha, double beta, int tpc = NN_TPC);
void gemm_tc_set_smem_limits();
template <typename T>
void launch_gemm_nn(const Launch& L, int akind, const RolePairs& rp, int msel, double alpha, double beta);
template <typename T> void launch_band_kinetic(const Launch& L, int xrole);
template <typename T> void launch_band_residual(const Launch& L, int xrole, int hxrole);
// rp < 0: no conjugation (P = the preconditioned residual); pp < 0 in normalize: no history copy
template <typename T> void launch_cg_precond(const Launch& L, int x, int hx, int p, int r, int pp, int rp);
template <typename T> void launch_normalize(const Launch& L, int p, int pp);
template <typename T> void launch_line_min(const Launch& L, int x, int hx, int p, int hp);
template <typename T> void launch_random_init(const Launch& L, int xrole, unsigned long long seed);
// rows >= nvec: zero, or (keep_tail) left as they are
template <typename T> void launch_copy_in(const Launch& L, int role, const double* src, int nvec, bool keep_tail = false);
template <typename T> void launch_copy_out(const Launch& L, int role, double* dst, int nvec);
// subspace diagonalisation; max_sweeps caps the Jacobi sweeps (a stop at the cap is counted
// in SC_RRCAP)
// blk = 1: the n_b x n_b subspace (S, Hs -> Tm); blk = 2: the 2 n_b block [X, W] of the block
// Davidson step (S2, H2 -> the lowest n_b Ritz vectors, X coefficients in Tm, W in Cm)
void launch_rr(const Launch& L, int use_smem, size_t smem, double* gscratch, size_t gstride, int max_sweeps = 30,
               int blk = 1);
void launch_rr_f32(const Launch& L, size_t smem, float* gscratch = nullptr, size_t gstride = 0, int max_sweeps = 10,
                   int blk = 1);
void launch_rr2_assemble(const Launch& L, int part);
// Rayleigh-Ritz of large subspaces: one thread-block cluster per problem, matrices in a
// per-problem global scratch of rr_cluster_scratch_bytes(n, sizeof(T)) bytes (T = float:
// deviation-form FP32 as k_rr_f32; T = double: the same in FP64).  False if the launch
// was refused (its shared memory would not fit).
size_t rr_cluster_scratch_bytes(int n, size_t tsize);
size_t rr_cluster_smem(int n);
size_t rr_cluster_smem64(int n);
template <typename T>
bool launch_rr_cluster(const Launch& L, int n_max, unsigned char* scratch, size_t stride, int max_sweeps, int blk = 1);
void launch_occupations(const Launch& L);
void linalg_set_smem_limits(size_t bytes);

// k_grid.cu  (grid sources/destinations: 0 rho_in, 1 rho_out, 2 resid, 3 vion_r)
constexpr int GRID_EW_POINTS = 1024;   // points per elementwise grid CTA
void launch_real_to_grid(const Launch& L, int src, int which);
void launch_grid_real_part(const Launch& L, int which, int dst);
void launch_hartree_g(const Launch& L, int which);
void launch_export_grid(const Launch& L, int sel, double* out);
// in != nullptr: gfft <- in; else out <- gfft (complex, C order (N1, N2, N3))
void launch_grid_copy_c(const Launch& L, const double2* in, double2* out);
template <typename T> void launch_veff(const Launch& L, const double* user_v);
// PBE (grids gfft3 = x + i y, gfft4 = z components): src 0 grad of rho_in(G), 1 of the
// forward-transformed rho_out in gfft2
void launch_gga_grad(const Launch& L, int src);
template <typename T> void launch_gga_point(const Launch& L);
void launch_gga_div(const Launch& L);
template <typename T> void launch_potential_g(const Launch& L);
void launch_vion_g(const Launch& L);
void launch_rho0_g(const Launch& L);
void launch_pulay_store(const Launch& L);
void launch_pulay_mix(const Launch& L, double a, double q0);
template <typename T> void launch_grid_energies(const Launch& Lchunks, double* part, int maxchunk);
void launch_grid_energies_reduce(const Launch& L, const double* part, int maxchunk);
void launch_finish_iteration(const Launch& L, double tol_e, double tol_rho, int count_iter);
void launch_pulay_gram(const Launch& Lchunks, double* part, int maxchunk, int hist);
void launch_pulay_solve(const Launch& L, const double* part, int maxchunk, int hist);
template <typename T> void launch_build_projectors(const Launch& Latoms, int deriv);
void launch_local_forces(const Launch& Latom_chunks, int maxchunk);
void launch_force_total(const Launch& L, int maxchunk);

// k_setup.cu
void launch_basis_count(const Launch& Lcols);
void launch_basis_scan(const Launch& L);
void launch_basis_fill(const Launch& Lcols);
void launch_roots(const Launch& L);
void launch_phases(const Launch& Latoms);
void launch_vloc_table(const Launch& Lew);
void launch_ewald(const Launch& Lsg, const Launch& Latoms, const Launch& Lprob);

}  // namespace sgo
