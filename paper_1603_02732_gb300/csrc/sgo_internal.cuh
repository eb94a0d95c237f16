// Internal declarations shared by the engine's translation units.
//
// Layout conventions (device):
//  * Real-space grids are plane-major: r = (i3 * N1 + i1) * N2 + i2, so one z-plane
//    (fixed i3) is a contiguous N1 x N2 block.  G-space box arrays use the same index
//    with (i1, i2, i3) = (m1 mod N1, m2 mod N2, m3 mod N3).
//  * Band vectors are real-packed Gamma half-sphere coefficients, band-major with
//    leading dimension ld: x[0] = c(0), x[1+2k] = sqrt2 Re c(G_k), x[2+2k] = sqrt2 Im c(G_k).
//    The half sphere is grouped by column pairs (c+, c-) = ((m1,m2), (-m1,-m2)):
//    pair 0 is the (0,0) column (entries m3 > 0), pair p > 0 holds every G of c+.
//  * Compact z-columns: column 0 = (0,0); pair p > 0 owns columns 2p-1 (c+) and 2p (c-).
//    The z-transformed wave buffer Wc is [pair][i3][col] (col fastest).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace sgo {

constexpr int MAX_SPECIES = 8;
constexpr int MAX_HIST = 8;
constexpr int NSCAL = 64;       // per-problem FP64 scalars (see SC_* below)
constexpr int NBANDSCAL = 12;   // per-band FP64 scalars (see BV_* below)
constexpr double SQRT2 = 1.41421356237309504880;
constexpr double PI = 3.14159265358979323846;

// per-problem scalars
enum {
  SC_EKIN = 0, SC_ENL, SC_ELOC, SC_EH, SC_EXC, SC_EEW, SC_MTS, SC_FREE,  // terms, F
  SC_FPREV, SC_RESID, SC_MU, SC_ENTROPY, SC_DF, SC_NELCHK,
  SC_CONV,        // 1 when converged
  SC_ITER,        // SCF iterations done
  SC_PULAY_N,     // history entries stored
  SC_PULAY_POS,   // ring position of the next entry
  SC_STATUS,      // sgo_status of this member
  SC_FIRSTCG,     // 1 while the CG history is empty
  SC_RRSWEEPS,    // Jacobi sweeps accumulated over the run (diagnostic)
  SC_POLISH,      // CG steps after the SCF stopping rule held (residual-controlled loop)
  SC_EIGRES,      // largest |H x - eps x| over the bands with occupation above 1e-6
  SC_RRCAP,       // subspace diagonalisations that stopped at their Jacobi sweep cap
  SC_PULAY_A = 24 // MAX_HIST*MAX_HIST Gram matrix of residuals (24..87 overlaps next; see NSCAL_ALL)
};
constexpr int NSCAL_ALL = SC_PULAY_A + MAX_HIST * MAX_HIST + 8;

// per-band scalars, array [BV_*][nb]
enum {
  BV_EKIN = 0,   // <x|T|x>
  BV_GR,         // <g, r> of this step
  BV_GRP,        // <g, r> of the previous step
  BV_PNORM,      // |P| before normalisation
  BV_THETA,
  BV_A, BV_B, BV_C,
  BV_RES,        // |H x - eps x|
  BV_GAMMA,
  BV_TMP0, BV_TMP1
};

template <typename T>
struct cplx {
  T x, y;
};

template <typename T>
__host__ __device__ __forceinline__ cplx<T> mk(T a, T b) {
  cplx<T> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator+(cplx<T> a, cplx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator-(cplx<T> a, cplx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> operator*(cplx<T> a, cplx<T> b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__host__ __device__ __forceinline__ cplx<T> scale(cplx<T> a, T s) { return mk(a.x * s, a.y * s); }
template <typename T>
__host__ __device__ __forceinline__ cplx<T> conj(cplx<T> a) { return mk(a.x, -a.y); }
// multiply by i*s (s = +1 or -1)
template <typename T>
__host__ __device__ __forceinline__ cplx<T> mul_is(cplx<T> a, T s) { return mk(-s * a.y, s * a.x); }

constexpr int FFT_MAX_STAGES = 10;

// Plan of one 1D FFT length: radices applied in order (see fft.cuh).
struct FftDim {
  int n;
  int nst;
  int rad[FFT_MAX_STAGES];
};

// Factor n into the fewest radices from {16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2} (largest
// first).  False if n has a prime factor other than 2, 3, 5.
inline bool make_fft_dim(int n, FftDim* d) {
  static const int cand[] = {16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};
  d->n = n;
  d->nst = 0;
  for (int i = 0; i < FFT_MAX_STAGES; ++i) d->rad[i] = 0;
  if (n < 1) return false;
  int m = n;
  while (m > 1 && d->nst < FFT_MAX_STAGES) {
    int r = 0;
    for (int c : cand)
      if (m % c == 0) {
        r = c;
        break;
      }
    if (r == 0) return false;
    d->rad[d->nst++] = r;
    m /= r;
  }
  return m == 1;
}

// Wave-buffer roles; the engine keeps one role -> physical map for the whole batch.
enum { WB_X = 0, WB_HX, WB_P, WB_HP, WB_PP, WB_RP, WB_W, WB_W2, NWB };

// Device descriptor of one structure ("problem") of a batch.
struct Prob {
  // geometry
  double cell[9], bvec[9], omega;
  int n1, n2, n3, ngrid;
  int box1, box2, box3;        // Miller enumeration box half-widths
  int m1max, m2max, m3max;
  double ecut;
  FftDim fd[3];                // plans for N1, N2, N3
  double2* roots64;            // [N1 | N2 | N3] exp(-2 pi i t / N_d)
  float2* roots32;             // same, single precision
  // basis
  int nhalf, npw, ld;
  int ncp, ncol;
  int* cp_off;                 // [ncp+1] into half entries
  int* cp_m1;                  // [ncp]
  int* cp_m2;                  // [ncp]
  int* ent_m;                  // [3][nhalf] Miller indices of the half-sphere entries
  int* ent_m3;                 // = ent_m + 2*nhalf
  int* ent_cp;                 // [nhalf] column pair of each half-sphere entry
  double* ekin;                // [ld] |G|^2/2 per packed component (0 in padding)
  float* ekin32;               // [ld] the same in single precision (mixed-path kernels)
  double* gvec;                // [3][ld] Cartesian G per packed component (0 at G = 0 and padding)
  int* colmap;                 // [n1*n2] compact column or -1, index i1*n2 + i2
  int* col_xy;                 // [ncol] i1*n2 + i2
  int* col_sidx;               // [ncol] rho(i1) * (n2 | 1) + i2: the column's slot in the register
                               // plane kernel's compact rows (rho = i1, or i1 - n1 + 2 m1max + 1)
  int* bx_cnt;                 // [(2 box1+1)(2 box2+1)] setup scratch: entries per box column
  int* bx_m3max;               // same: max |m3| in the column
  int* bx_pair;                // same: column pair index or -1
  int* bx_off;                 // same: first entry
  int* setup_out;              // [8]: nhalf, ncp, m1max, m2max, m3max
  // atoms
  int natom, nspecies;
  double* pos;                 // [natom*3]
  int* spec;                   // [natom]
  double sp[MAX_SPECIES * 6];  // z, rc, a, sigma, rp, d
  double nel, kT;
  // bands: nb carried by the eigensolver, of which the lowest nbo (the requested count) are
  // occupied and reported; the nb - nbo above them give the block convergence headroom
  int nb, nbo, npair;
  // wave buffers (element type = engine precision)
  void* wb[NWB];               // each [nb][ld], physical buffers
  int role[NWB];               // role -> physical buffer of this problem (swapped on the device)
  void* B;                     // [nproj][ld] projectors
  void* dB;                    // [3*nproj][ld] projector derivatives (forces)
  // projectors, atom-major (the s projector of each atom, then its p_x, p_y, p_z where the
  // species has a p channel): atom, kind (0 s, 1 + m p_m), strength, width; first of each atom
  int nproj;
  int* pj_atom;                // [nproj]
  int* pj_kind;                // [nproj]
  double* pj_d;                // [nproj]
  double* pj_rp;               // [nproj]
  int* pj_first;               // [natom + 1]
  void* Wc;                    // complex [npair][n3][ncol]
  void* Gp;                    // complex [npair][n3][2 m1max + 1][n2]: occupied x rows of the
                               // planes (big-plane path only, else null)
  void* veff;                  // real [ngrid] (engine precision)
  // FP64 grids
  double* vion_r;              // [ngrid]
  double* vloc_g;              // [nspecies][ngrid] v_s(G) on the box (Nyquist zeroed)
  double* g2box;               // [ngrid] |G|^2 on the box, -1 on Nyquist planes
  double* rho_in;              // [ngrid]
  double* rho_out;             // [ngrid]
  double* resid;               // [ngrid]
  double2* gfft;               // [ngrid]
  double2* gfft2;              // [ngrid]
  double2* gfft3;              // [ngrid] PBE only (else null): grad rho, then 2 de/dsigma grad rho
  double2* gfft4;              // [ngrid] PBE only: the third component, then div of the above
  int xc;                      // 0 LDA, 1 PBE
  double2* rhog_in;            // [ngrid] rho_in(G), the mixed density (SCF state)
  double2* hrho;               // [MAX_HIST][ngrid] Pulay history of rho_in(G)
  double2* hres;               // [MAX_HIST][ngrid] Pulay history of R(G) = rho_out(G) - rho_in(G)
  double2* phase;              // [natom][n1+n2+n3] exp(-i 2pi m s_d), m = -N/2..N/2-1 wrapped
  // small dense FP64
  double* S;                   // [nb*nb]
  double* Hs;                  // [nb*nb]
  double* Tm;                  // [nb*nb]
  double* Cm;                  // [nb*nb]
  double* S2;                  // [4*nb*nb] overlap of the block [X, W] (block Davidson only, else null)
  double* H2;                  // [4*nb*nb] its subspace matrix
  double* proj;                // [nproj*nb]
  double* dproj;               // [3*nproj*nb]
  double* eps;                 // [nb]
  double* occ;                 // [nb]
  double* bv;                  // [NBANDSCAL][nb]
  double* scal;                // [NSCAL_ALL]
  double* forces;              // [natom*3]
  double* ewald_f;             // [natom*3]
  double* fpart;               // force partials [natom][nchunk][3]
  int* status;                 // [4]: Cholesky failure, non-finite energy
  // Ewald
  double ew_eta, ew_rmax, ew_gmax;
  int ew_ng[3], ew_nr[3];
  double2* ew_sg;              // [(2ng1+1)(2ng2+1)(2ng3+1)] S(G)
  double* ew_part;             // [natom] real-space energy per atom, then recip chunks
};

// |G|^2/2 of packed component k in the working precision (no FP64 load or conversion on
// the mixed path)
template <typename T>
__device__ __forceinline__ T ekin_at(const Prob& P, int k);
template <>
__device__ __forceinline__ float ekin_at<float>(const Prob& P, int k) {
  return P.ekin32[k];
}
template <>
__device__ __forceinline__ double ekin_at<double>(const Prob& P, int k) {
  return P.ekin[k];
}

template <typename T>
__device__ __forceinline__ T* wbuf(const Prob& P, int role) {
  return reinterpret_cast<T*>(P.wb[P.role[role]]);
}

// Static CTA -> problem map of one kind of launch: start[p] = first CTA of problem p.
struct WorkMap {
  int* start = nullptr;  // device [nprob+1]
  int total = 0;
  int maxper = 0;
  // largest grid / band dimensions over the problems with work in this map (shared-memory
  // sizes of its launches); -1 = not set (use the batch's)
  int max_n1 = -1, max_n2 = -1, max_n3 = -1, max_n12 = -1, max_nb = -1;
};

__device__ __forceinline__ int locate(const int* __restrict__ start, int nprob, int blk) {
  int lo = 0, hi = nprob;  // find largest p with start[p] <= blk
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(start + mid) <= blk) lo = mid; else hi = mid;
  }
  return lo;
}

// ---- block reductions (deterministic) ----
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block; every thread gets the result.  red: >= 33 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double* red) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double t = lane < nw ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// ---- error helper ----
void set_error(const std::string& msg);
bool cuda_ok(cudaError_t e, const char* what);

}  // namespace sgo
