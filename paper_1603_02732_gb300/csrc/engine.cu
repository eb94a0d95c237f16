// Host engine: context set-up and the lockstep SCF driver (Sec. II D).
//
// One SCF iteration, for every structure still iterating:
//   V_eff[rho_in] -> H Psi -> subspace diagonalisation -> ncg all-band CG steps
//   (Algorithm 1) -> occupations -> rho_out -> energy, convergence -> Pulay mix.
// Every launch covers all active structures; a structure that has converged is masked.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "engine.h"

namespace sgo {

thread_local std::string g_err;
void set_error(const std::string& m) { g_err = m; }
const char* last_error() { return g_err.c_str(); }
bool cuda_ok(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return true;
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return false;
}

// ---- device memory: cudaMalloc, or the caller's allocator (sgo_set_allocator) ----
namespace {
std::mutex g_alloc_mu;
sgo_alloc_fn g_alloc_fn = nullptr;
sgo_free_fn g_free_fn = nullptr;
void* g_alloc_user = nullptr;
struct Hooked {
  sgo_free_fn release;
  void* user;
};
// every block the caller's allocator gave, with the release function it came with (the
// hook may change between a context's creation and its destruction)
std::unordered_map<void*, Hooked>& hooked() {
  static std::unordered_map<void*, Hooked> m;
  return m;
}
}  // namespace

void set_allocator(sgo_alloc_fn a, sgo_free_fn f, void* user) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc_fn = a;
  g_free_fn = f;
  g_alloc_user = user;
}

cudaError_t dev_malloc_bytes(void** p, size_t bytes, cudaStream_t s) {
  sgo_alloc_fn a;
  sgo_free_fn f;
  void* user;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    a = g_alloc_fn;
    f = g_free_fn;
    user = g_alloc_user;
  }
  // every block starts zeroed, whichever allocator gave it (a pool hands back used memory;
  // padding rows of the GEMM images and partial sums are read as zeros)
  if (!a) {
    const cudaError_t e = cudaMalloc(p, bytes);
    return e == cudaSuccess ? cudaMemset(*p, 0, bytes) : e;
  }
  *p = a(bytes ? bytes : 1, s, user);
  if (!*p) return cudaErrorMemoryAllocation;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    hooked()[*p] = Hooked{f, user};
  }
  return cudaMemset(*p, 0, bytes);
}

void dev_free(void* p, bool synced) {
  if (!p) return;
  Hooked h{nullptr, nullptr};
  bool found = false;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    auto it = hooked().find(p);
    if (it != hooked().end()) {
      h = it->second;
      found = true;
      hooked().erase(it);
    }
  }
  if (!found) {
    cudaFree(p);
    return;
  }
  // the caller's pool may hand the block out again at once: no kernel may still use it
  if (!synced) cudaDeviceSynchronize();
  if (h.release) h.release(p, nullptr, h.user);
}

#define CK(x)                                  \
  do {                                         \
    if (!cuda_ok((x), #x)) return SGO_ERR_CUDA; \
  } while (0)

namespace {

// ---- small kernels of the driver ----
__global__ void k_set_scal(KArgs ka, int idx, double v, int only_active) {
  const int p = blockIdx.x;
  if (only_active && !ka.active[p]) return;
  if (threadIdx.x == 0) ka.probs[p].scal[idx] = v;
}
// swap two buffer roles of every active problem
__global__ void k_swap_roles(KArgs ka, RolePairs rp) {
  const int p = blockIdx.x;
  if (!ka.active[p] || threadIdx.x != 0) return;
  Prob* P = const_cast<Prob*>(ka.probs) + p;
  for (int k = 0; k < rp.n; ++k) {
    const int a = rp.a[k], b = rp.y[k];
    const int t = P->role[a];
    P->role[a] = P->role[b];
    P->role[b] = t;
  }
}
// copy the wavefunctions into physical buffer 0 (CTA = (problem, band)), then reset roles
template <typename T>
__global__ void k_x_to_buffer0(KArgs ka) {
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  const Prob& P = ka.probs[p];
  if (P.role[WB_X] == 0) return;
  const int i = blockIdx.x - ka.start[p];
  const T* s = wbuf<T>(P, WB_X) + (size_t)i * P.ld;
  T* d = reinterpret_cast<T*>(P.wb[0]) + (size_t)i * P.ld;
  for (int k = threadIdx.x; k < P.ld; k += blockDim.x) d[k] = s[k];
}
__global__ void k_reset_roles(KArgs ka) {
  Prob* P = const_cast<Prob*>(ka.probs) + blockIdx.x;
  if (threadIdx.x < NWB) P->role[threadIdx.x] = threadIdx.x;
}
__global__ void k_reset(KArgs ka) {
  const int p = blockIdx.x;
  const Prob& P = ka.probs[p];
  for (int i = threadIdx.x; i < NSCAL_ALL; i += blockDim.x) P.scal[i] = 0.0;
  if (threadIdx.x < 4) P.status[threadIdx.x] = 0;
  if (threadIdx.x == 0) P.scal[SC_FIRSTCG] = 1.0;
}
// flags[p] = {converged, cholesky failure, non-finite, resid}
__global__ void k_gather_flags(KArgs ka, double* flags) {
  const int p = blockIdx.x;
  const Prob& P = ka.probs[p];
  if (threadIdx.x == 0) {
    flags[4 * p + 0] = P.scal[SC_CONV];
    flags[4 * p + 1] = (double)(P.status[0] | P.status[2]);
    flags[4 * p + 2] = (double)P.status[1];
    flags[4 * p + 3] = P.scal[SC_RESID];
  }
}
// End of one SCF iteration on the device (graph mode): gather every member's flags as
// k_gather_flags does, retire members that converged or failed (the host loop's test),
// count the iteration, and (set_cond) let the enclosing WHILE node run again while some
// member is active and the iteration cap is not reached.  One CTA.
__global__ void k_scf_control(KArgs ka, int* active, double* flags, int* iter, int max_scf,
                              cudaGraphConditionalHandle cond, int set_cond) {
  __shared__ int nact;
  if (threadIdx.x == 0) nact = 0;
  __syncthreads();
  for (int p = threadIdx.x; p < ka.nprob; p += blockDim.x) {
    const Prob& P = ka.probs[p];
    const double f0 = P.scal[SC_CONV], f1 = (double)(P.status[0] | P.status[2]), f2 = (double)P.status[1];
    flags[4 * p + 0] = f0;
    flags[4 * p + 1] = f1;
    flags[4 * p + 2] = f2;
    flags[4 * p + 3] = P.scal[SC_RESID];
    if (active[p] && (f0 != 0.0 || f1 != 0.0 || f2 != 0.0)) active[p] = 0;
    if (active[p]) atomicAdd(&nact, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int it = ++*iter;
    if (set_cond) cudaGraphSetConditional(cond, (nact > 0 && it < max_scf) ? 1u : 0u);
  }
}
// Entry test of the SCF WHILE node: run the first self-consistent iteration only if some
// member is still active and the cap allows it.
__global__ void k_scf_gate(const int* active, int n, const int* iter, int max_scf, cudaGraphConditionalHandle cond) {
  int nact = 0;
  for (int p = 0; p < n; ++p) nact += active[p] != 0;
  cudaGraphSetConditional(cond, (nact > 0 && *iter < max_scf) ? 1u : 0u);
}
// Algorithm 1's CG loop runs "while not converged".  The SCF iterations take a fixed
// number of CG steps each; once a member's SCF stopping rule holds, further CG steps at its
// final potential refine its bands until every band with occupation above 1e-6 has a
// residual |H x - eps x| below the tolerance.
// mode 0: the members whose stopping rule held (and that have not failed) take part;
// mode 1: of those, the members that took a step (their density and energy are redone).
// Adaptive CG steps: mode 0 keeps the active mask in saved and leaves out of the next step
// the members whose density residual is still above thr; mode 1 restores the mask.  One CTA.
__global__ void k_cg_gate(KArgs ka, int* active, int* saved, double thr, int mode) {
  for (int p = threadIdx.x; p < ka.nprob; p += blockDim.x) {
    if (mode == 0) {
      saved[p] = active[p];
      if (active[p] && ka.probs[p].scal[SC_RESID] > thr) active[p] = 0;
    } else {
      active[p] = saved[p];
    }
  }
}

__global__ void k_polish_activate(KArgs ka, int* active, int mode) {
  for (int p = threadIdx.x; p < ka.nprob; p += blockDim.x) {
    const Prob& P = ka.probs[p];
    const bool ok = P.scal[SC_CONV] != 0.0 && (P.status[0] | P.status[1] | P.status[2]) == 0;
    if (mode == 0) {
      P.scal[SC_POLISH] = 0.0;
      P.scal[SC_EIGRES] = 0.0;
      active[p] = ok ? 1 : 0;
    } else {
      active[p] = (ok && P.scal[SC_POLISH] > 0.0) ? 1 : 0;
    }
  }
}
// The loop's test (one CTA): the largest residual over the bands with occupation above
// 1e-6 (BV_RES, written by k_band_residual for the current bands and eigenvalues); a
// member below tol, or at max_steps, leaves; the others count one more step.  set_cond:
// the enclosing WHILE node runs again while some member is left.
__global__ void k_polish_control(KArgs ka, int* active, int* passes, double tol, int max_steps,
                                 cudaGraphConditionalHandle cond, int set_cond) {
  __shared__ int nact;
  if (threadIdx.x == 0) nact = 0;
  __syncthreads();
  for (int p = threadIdx.x; p < ka.nprob; p += blockDim.x) {
    if (!active[p]) continue;
    const Prob& P = ka.probs[p];
    double mx = 0.0;
    for (int i = 0; i < P.nb; ++i)
      if (P.occ[i] > 1e-6) mx = fmax(mx, P.bv[BV_RES * P.nb + i]);
    P.scal[SC_EIGRES] = mx;
    if (!(mx >= tol) || P.scal[SC_POLISH] >= (double)max_steps) {
      active[p] = 0;
    } else {
      P.scal[SC_POLISH] += 1.0;
      atomicAdd(&nact, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (passes) ++*passes;
    if (set_cond) cudaGraphSetConditional(cond, nact > 0 ? 1u : 0u);
  }
}
// out[p] = F, out_f[off_p + e] = forces (device gather for the device-pointer batch)
__global__ void k_gather_results(KArgs ka, const int* slot, const int* foff, double* energies, double* forces,
                                 int* status) {
  const int p = blockIdx.x;
  const Prob& P = ka.probs[p];
  if (threadIdx.x == 0) {
    energies[slot[p]] = P.scal[SC_FREE];
    status[slot[p]] = P.status[0] ? SGO_ERR_NOT_CONVERGED : (P.scal[SC_CONV] != 0.0 ? SGO_OK : SGO_ERR_NOT_CONVERGED);
  }
  for (int e = threadIdx.x; e < 3 * P.natom; e += blockDim.x) forces[foff[p] + e] = P.forces[e];
}
__global__ void k_scatter_pos(KArgs ka, const int* foff, const double* pos) {
  const int p = blockIdx.x;
  const Prob& P = ka.probs[p];
  for (int e = threadIdx.x; e < 3 * P.natom; e += blockDim.x) P.pos[e] = pos[foff[p] + e];
}

int div_up(long a, long b) { return (int)((a + b - 1) / b); }
double log2d(double x) { return std::log(x) / std::log(2.0); }

bool smooth235(int n) {
  if (n < 1) return false;
  for (int p : {2, 3, 5})
    while (n % p == 0) n /= p;
  return n == 1;
}

}  // namespace

// Which kernels take the plane passes of one structure: the mixed path's register line
// FFTs (single thread per line up to 72, lane pairs 96-128) where their shared memory
// fits, else the shared-memory plane engine (two whole planes per CTA), else line blocks
// through a global buffer (big planes).  vpsi: the H.psi pass; dens: the density pass.
PlanePaths plane_paths(const Prob& d, int precision) {
  const size_t cap = 220 * 1024;
  PlanePaths q;
  q.preg = precision == 1 && plane_reg_ok(d.n1, d.n2) && plane_reg_smem(d.n1, d.n2, d.m1max) <= cap;
  q.dreg = q.preg && plane_density_reg_smem(d.n1, d.n2, d.m1max) <= cap;
  q.ppair = precision == 1 && !q.preg && pair_plane_ok(d.n1, d.n2) && pair_plane_smem(d.n1, d.n2, d.m1max) <= cap;
  q.dpair = q.ppair && pair_density_smem(d.n1, d.n2, d.m1max) <= cap;
  q.psmem = (size_t)(2 * d.n1 * d.n2 + d.n1 + d.n2) * 16 <= cap && d.n1 * d.n2 <= 8192;
  q.pbig = !q.preg && !q.ppair && !q.psmem;
  q.dbig = !q.dreg && !q.dpair && !q.psmem;
  return q;
}

namespace {

// counting arena pass + real pass
template <class A>
void layout(sgo_ctx* c, A& a) {
  Prob& d = c->d;
  const size_t ts = c->tsize;
  const int nb = d.nb, ld = d.ld, na = d.natom, ng = d.ngrid, n12 = d.n1 * d.n2, nt = d.n1 + d.n2 + d.n3;
  d.cp_off = a.template take<int>(d.ncp + 1);
  d.cp_m1 = a.template take<int>(d.ncp);
  d.cp_m2 = a.template take<int>(d.ncp);
  d.ent_m = a.template take<int>(3 * std::max(d.nhalf, 1));
  d.ent_m3 = d.ent_m + 2 * d.nhalf;
  d.ent_cp = a.template take<int>(std::max(d.nhalf, 1));
  d.ekin = a.template take<double>(ld);
  d.ekin32 = a.template take<float>(ld);
  d.gvec = a.template take<double>(3 * (size_t)ld);
  d.colmap = a.template take<int>(n12);
  d.col_xy = a.template take<int>(d.ncol);
  d.col_sidx = a.template take<int>(d.ncol);
  d.roots64 = a.template take<double2>(nt);
  d.roots32 = a.template take<float2>(nt);
  d.pos = a.template take<double>(3 * na);
  d.spec = a.template take<int>(na);
  for (int i = 0; i < NWB; ++i) d.wb[i] = a.template take<char>((size_t)nb * ld * ts);
  const int npj = d.nproj;
  d.B = a.template take<char>((size_t)npj * ld * ts);
  d.dB = a.template take<char>((size_t)3 * npj * ld * ts);
  d.pj_atom = a.template take<int>(npj);
  d.pj_kind = a.template take<int>(npj);
  d.pj_d = a.template take<double>(npj);
  d.pj_rp = a.template take<double>(npj);
  d.pj_first = a.template take<int>(na + 1);
  d.Wc = a.template take<char>((size_t)d.npair * d.n3 * d.ncol * 2 * ts);
  const PlanePaths pp = plane_paths(d, c->precision);
  d.Gp = (pp.pbig || pp.dbig) ? a.template take<char>(big_plane_bytes(d.npair, d.n3, d.m1max, d.n2, ts)) : nullptr;
  d.veff = a.template take<char>((size_t)ng * ts);
  d.vion_r = a.template take<double>(ng);
  d.rho_in = a.template take<double>(ng);
  d.rho_out = a.template take<double>(ng);
  d.resid = a.template take<double>(ng);
  d.vloc_g = a.template take<double>((size_t)d.nspecies * ng);
  d.g2box = a.template take<double>(ng);
  d.gfft = a.template take<double2>(ng);
  d.gfft2 = a.template take<double2>(ng);
  if (c->opts.xc == 1) {
    d.gfft3 = a.template take<double2>(ng);
    d.gfft4 = a.template take<double2>(ng);
  } else {
    d.gfft3 = d.gfft4 = nullptr;
  }
  d.xc = c->opts.xc;
  d.rhog_in = a.template take<double2>(ng);
  d.hrho = a.template take<double2>((size_t)MAX_HIST * ng);
  d.hres = a.template take<double2>((size_t)MAX_HIST * ng);
  d.phase = a.template take<double2>((size_t)na * nt);
  d.S = a.template take<double>((size_t)nb * nb);
  d.Hs = a.template take<double>((size_t)nb * nb);
  d.Tm = a.template take<double>((size_t)nb * nb);
  d.Cm = a.template take<double>((size_t)nb * nb);
  if (c->opts.eigensolver == 1) {
    d.S2 = a.template take<double>((size_t)4 * nb * nb);
    d.H2 = a.template take<double>((size_t)4 * nb * nb);
  } else {
    d.S2 = d.H2 = nullptr;
  }
  d.proj = a.template take<double>((size_t)npj * nb);
  d.dproj = a.template take<double>((size_t)3 * npj * nb);
  d.eps = a.template take<double>(nb);
  d.occ = a.template take<double>(nb);
  d.bv = a.template take<double>((size_t)NBANDSCAL * nb);
  d.scal = a.template take<double>(NSCAL_ALL);
  d.forces = a.template take<double>(3 * na);
  d.ewald_f = a.template take<double>(3 * na);
  d.fpart = a.template take<double>((size_t)na * div_up(ng, GRID_CHUNK) * 3);
  d.status = a.template take<int>(4);
  d.ew_sg = a.template take<double2>(c->ngbox_ew);
  d.ew_part = a.template take<double>(na + div_up(c->ngbox_ew, 256));
}

struct Counter {
  size_t used = 0;
  template <typename P>
  P* take(size_t count, size_t align = 256) {
    used = (used + align - 1) / align * align;
    used += count * sizeof(P);
    return nullptr;
  }
};

sgo_status check_geometry(const sgo_ctx* c, const double* pos) {
  const int n = (int)c->spec.size();
  for (int i = 0; i < 3 * n; ++i)
    if (!std::isfinite(pos[i])) {
      set_error("non-finite atomic position");
      return SGO_ERR_GEOMETRY;
    }
  // minimum-image distances via fractional coordinates
  double inv[9];
  const double* A = c->cell;
  double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) + A[2] * (A[3] * A[7] - A[4] * A[6]);
  inv[0] = (A[4] * A[8] - A[5] * A[7]) / det;
  inv[1] = (A[2] * A[7] - A[1] * A[8]) / det;
  inv[2] = (A[1] * A[5] - A[2] * A[4]) / det;
  inv[3] = (A[5] * A[6] - A[3] * A[8]) / det;
  inv[4] = (A[0] * A[8] - A[2] * A[6]) / det;
  inv[5] = (A[2] * A[3] - A[0] * A[5]) / det;
  inv[6] = (A[3] * A[7] - A[4] * A[6]) / det;
  inv[7] = (A[1] * A[6] - A[0] * A[7]) / det;
  inv[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      double d[3], f[3];
      for (int k = 0; k < 3; ++k) d[k] = pos[3 * i + k] - pos[3 * j + k];
      for (int k = 0; k < 3; ++k) {
        f[k] = d[0] * inv[k] + d[1] * inv[3 + k] + d[2] * inv[6 + k];
        f[k] -= std::nearbyint(f[k]);
      }
      double best = 1e300;
      for (int a = -1; a <= 1; ++a)
        for (int b = -1; b <= 1; ++b)
          for (int e = -1; e <= 1; ++e) {
            double v[3];
            for (int k = 0; k < 3; ++k) v[k] = (f[0] + a) * A[k] + (f[1] + b) * A[3 + k] + (f[2] + e) * A[6 + k];
            best = std::min(best, v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
          }
      if (best < 0.25) {
        set_error("atoms closer than 0.5 bohr");
        return SGO_ERR_GEOMETRY;
      }
    }
  return SGO_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// context set-up
// ---------------------------------------------------------------------------
sgo_status set_positions(sgo_ctx* c, const double* pos) {
  sgo_status s = check_geometry(c, pos);
  if (s != SGO_OK) return s;
  std::copy(pos, pos + c->pos.size(), c->pos.begin());
  CK(cudaMemcpyAsync(c->d.pos, c->pos.data(), c->pos.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  return SGO_OK;
}

sgo_status ctx_setup(sgo_ctx* c) {
  Prob& d = c->d;
  std::memset(&d, 0, sizeof(Prob));
  const double* A = c->cell;
  for (int i = 0; i < 9; ++i) d.cell[i] = A[i];
  double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) + A[2] * (A[3] * A[7] - A[4] * A[6]);
  if (!(std::fabs(det) > 1e-8)) {
    set_error("singular cell");
    return SGO_ERR_ARG;
  }
  d.omega = std::fabs(det);
  // b_j = 2 pi (A^-1)^T rows: b_j[k] = 2 pi inv[k][j]
  double inv[9];
  inv[0] = (A[4] * A[8] - A[5] * A[7]) / det;
  inv[1] = (A[2] * A[7] - A[1] * A[8]) / det;
  inv[2] = (A[1] * A[5] - A[2] * A[4]) / det;
  inv[3] = (A[5] * A[6] - A[3] * A[8]) / det;
  inv[4] = (A[0] * A[8] - A[2] * A[6]) / det;
  inv[5] = (A[2] * A[3] - A[0] * A[5]) / det;
  inv[6] = (A[3] * A[7] - A[4] * A[6]) / det;
  inv[7] = (A[1] * A[6] - A[0] * A[7]) / det;
  inv[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  for (int j = 0; j < 3; ++j)
    for (int k = 0; k < 3; ++k) d.bvec[3 * j + k] = 2.0 * PI * inv[3 * k + j];
  d.ecut = c->ecut;
  const double gmax = std::sqrt(2.0 * c->ecut);
  int nd[3];
  int box[3];
  for (int i = 0; i < 3; ++i) {
    double len = std::sqrt(A[3 * i] * A[3 * i] + A[3 * i + 1] * A[3 * i + 1] + A[3 * i + 2] * A[3 * i + 2]);
    int mb = (int)std::floor(len * gmax / (2.0 * PI));
    box[i] = mb + 1;
    int n = c->opts.fft[i];
    if (n <= 0) {
      n = 4 * mb + 1;
      while (!smooth235(n)) ++n;
    }
    if (!smooth235(n)) {
      set_error("FFT size must have only the factors 2, 3, 5");
      return SGO_ERR_ARG;
    }
    nd[i] = n;
    if (!make_fft_dim(n, &d.fd[i])) return SGO_ERR_ARG;
  }
  d.n1 = nd[0];
  d.n2 = nd[1];
  d.n3 = nd[2];
  d.ngrid = nd[0] * nd[1] * nd[2];
  d.box1 = box[0];
  d.box2 = box[1];
  d.box3 = box[2];
  // planes of any size: register kernels, the shared-memory plane engine or line blocks
  // through a global buffer (see plane_paths); the z lines stay in shared memory
  if ((size_t)(4 * QCP + 1) * d.n3 * 16 > 220 * 1024) {
    set_error("N3 too large");
    return SGO_ERR_ARG;
  }
  d.natom = (int)c->spec.size();
  d.nspecies = (int)c->species.size();
  for (int s = 0; s < d.nspecies; ++s) {
    const sgo_species& q = c->species[s];
    double v[6] = {q.z_val, q.rc, q.a_sr, q.sigma_sr, q.rp, q.d_nl};
    for (int k = 0; k < 6; ++k) d.sp[6 * s + k] = v[k];
  }
  d.nel = 0.0;
  for (int a = 0; a < d.natom; ++a) d.nel += c->species[c->spec[a]].z_val;
  // projector list (atom-major: s, then p_x, p_y, p_z for a species with a p channel)
  c->pj_atom.clear();
  c->pj_kind.clear();
  c->pj_d.clear();
  c->pj_rp.clear();
  c->pj_first.assign(1, 0);
  for (int a = 0; a < d.natom; ++a) {
    const sgo_species& q = c->species[c->spec[a]];
    c->pj_atom.push_back(a);
    c->pj_kind.push_back(0);
    c->pj_d.push_back(q.d_nl);
    c->pj_rp.push_back(q.rp);
    if (q.d_p != 0.0)
      for (int m = 0; m < 3; ++m) {
        c->pj_atom.push_back(a);
        c->pj_kind.push_back(1 + m);
        c->pj_d.push_back(q.d_p);
        c->pj_rp.push_back(q.rp_p);
      }
    c->pj_first.push_back((int)c->pj_atom.size());
  }
  d.nproj = (int)c->pj_atom.size();
  d.kT = c->opts.kT;
  for (int i = 0; i < NWB; ++i) d.role[i] = i;
  d.nb = c->nb_int;
  d.nbo = c->nb;
  d.npair = (d.nb + 1) / 2;
  // Ewald parameters: eta from the volume; sums to a relative tail of 1e-16
  d.ew_eta = 3.0 / std::cbrt(d.omega);
  d.ew_rmax = 5.9 / d.ew_eta;
  d.ew_gmax = 2.0 * d.ew_eta * std::sqrt(-std::log(1e-16));
  for (int i = 0; i < 3; ++i) {
    double len = std::sqrt(A[3 * i] * A[3 * i] + A[3 * i + 1] * A[3 * i + 1] + A[3 * i + 2] * A[3 * i + 2]);
    double bl = std::sqrt(d.bvec[3 * i] * d.bvec[3 * i] + d.bvec[3 * i + 1] * d.bvec[3 * i + 1] +
                          d.bvec[3 * i + 2] * d.bvec[3 * i + 2]);
    d.ew_nr[i] = (int)std::ceil(d.ew_rmax * bl / (2.0 * PI)) + 1;
    d.ew_ng[i] = (int)std::ceil(d.ew_gmax * len / (2.0 * PI)) + 1;
  }
  c->ngbox_ew = (2 * d.ew_ng[0] + 1) * (2 * d.ew_ng[1] + 1) * (2 * d.ew_ng[2] + 1);

  // ---- phase 1: basis enumeration on the device ----
  c->box_cols = (2 * box[0] + 1) * (2 * box[1] + 1);
  const size_t setup_bytes = (size_t)4 * c->box_cols * sizeof(int) + 64 + 4 * 256;
  CK(dev_malloc(&c->arena_setup, setup_bytes));
  {
    Arena a;
    a.base = c->arena_setup;
    d.bx_cnt = a.take<int>(c->box_cols);
    d.bx_m3max = a.take<int>(c->box_cols);
    d.bx_pair = a.take<int>(c->box_cols);
    d.bx_off = a.take<int>(c->box_cols);
    d.setup_out = a.take<int>(8);
  }
  Prob* dprob = nullptr;
  int* dstart = nullptr;
  int* dact = nullptr;
  CK(dev_malloc(&dprob, sizeof(Prob)));
  CK(dev_malloc(&dstart, 2 * sizeof(int)));
  CK(dev_malloc(&dact, sizeof(int)));
  const int one = 1;
  const int nbc = div_up(c->box_cols, 128);
  int st[2] = {0, nbc};
  CK(cudaMemcpy(dstart, st, sizeof(st), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dact, &one, sizeof(int), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(dprob, &d, sizeof(Prob), cudaMemcpyHostToDevice));
  Launch L1;
  L1.ka = KArgs{dprob, dstart, 1, dact};
  L1.map.start = dstart;
  L1.map.total = nbc;
  L1.stream = c->stream;
  launch_basis_count(L1);
  launch_basis_scan(L1);
  int out[8];
  CK(cudaMemcpyAsync(out, d.setup_out, sizeof(out), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  d.nhalf = out[0];
  d.ncp = out[1];
  d.m1max = out[2];
  d.m2max = out[3];
  d.m3max = out[4];
  d.npw = 1 + 2 * d.nhalf;
  d.ld = (d.npw + 31) / 32 * 32;
  d.ncol = 2 * d.ncp - 1;
  if (4 * d.m1max + 1 > d.n1 || 4 * d.m2max + 1 > d.n2 || 4 * d.m3max + 1 > d.n3) {
    dev_free(dprob);
    dev_free(dstart);
    dev_free(dact);
    set_error("FFT grid aliases: need N_i >= 4 m_max,i + 1");
    return SGO_ERR_ARG;
  }
  if (c->nb > d.npw) {
    dev_free(dprob);
    dev_free(dstart);
    dev_free(dact);
    set_error("more bands than plane waves");
    return SGO_ERR_ARG;
  }
  if (c->nb_int > d.npw) {  // the headroom bands are capped by the basis
    c->nb_int = d.npw;
    d.nb = d.npw;
    d.npair = (d.nb + 1) / 2;
  }
  if (c->opts.eigensolver == 1 && 2 * d.nb > d.npw) {
    dev_free(dprob);
    dev_free(dstart);
    dev_free(dact);
    set_error("block Davidson needs 2 n_b (with the headroom bands) <= the number of plane waves");
    return SGO_ERR_ARG;
  }

  // ---- phase 2: allocation ----
  Counter cnt;
  layout(c, cnt);
  cudaError_t e = dev_malloc(&c->arena_main, cnt.used + 256);
  if (e != cudaSuccess) {
    dev_free(dprob);
    dev_free(dstart);
    dev_free(dact);
    set_error(std::string("device allocation failed: ") + cudaGetErrorString(e));
    return SGO_ERR_OOM;
  }
  {
    Arena a;
    a.base = c->arena_main;
    layout(c, a);
  }
  CK(cudaMemsetAsync(c->arena_main, 0, cnt.used, c->stream));
  CK(cudaMemsetAsync(d.colmap, 0xFF, sizeof(int) * d.n1 * d.n2, c->stream));
  std::vector<int> spec(c->spec);
  CK(cudaMemcpyAsync(d.spec, spec.data(), spec.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(d.pos, c->pos.data(), c->pos.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(d.pj_atom, c->pj_atom.data(), sizeof(int) * d.nproj, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(d.pj_kind, c->pj_kind.data(), sizeof(int) * d.nproj, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(d.pj_d, c->pj_d.data(), sizeof(double) * d.nproj, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(d.pj_rp, c->pj_rp.data(), sizeof(double) * d.nproj, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(d.pj_first, c->pj_first.data(), sizeof(int) * (d.natom + 1), cudaMemcpyHostToDevice,
                     c->stream));
  CK(cudaMemcpyAsync(dprob, &d, sizeof(Prob), cudaMemcpyHostToDevice, c->stream));
  launch_basis_fill(L1);
  launch_roots(L1);
  const int nvl = div_up(d.ngrid, 1024);
  st[1] = nvl;
  CK(cudaMemcpyAsync(dstart, st, sizeof(st), cudaMemcpyHostToDevice, c->stream));
  Launch L2 = L1;
  L2.map.total = nvl;
  launch_vloc_table(L2);
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaGetLastError());
  dev_free(dprob);
  dev_free(dstart);
  dev_free(dact);
  c->h_scal.assign(NSCAL_ALL, 0.0);
  c->h_eps.assign(d.nb, 0.0);
  c->h_occ.assign(d.nb, 0.0);
  c->h_forces.assign(3 * d.natom, 0.0);
  return SGO_OK;
}

}  // namespace sgo

sgo_ctx::~sgo_ctx() {
  if (arena_setup) sgo::dev_free(arena_setup);
  if (arena_main) sgo::dev_free(arena_main);
}

namespace sgo {

const char* const kTimerNames[TK_COUNT] = {"plane_vpsi", "wave_to_cols", "cols_to_wave", "plane_density",
                                           "gemm_tn",    "gemm_nn",      "rr",           "grid_fft",
                                           "cg_band",    "grid_other",   "gemm_small"};

// ---------------------------------------------------------------------------
// Engine
// ---------------------------------------------------------------------------
WorkMap Engine::make_map(const std::vector<int>& counts) {
  WorkMap m;
  std::vector<int> st(counts.size() + 1, 0);
  int mx = 0;
  for (size_t i = 0; i < counts.size(); ++i) {
    st[i + 1] = st[i] + counts[i];
    mx = std::max(mx, counts[i]);
  }
  m.total = st.back();
  m.maxper = mx;
  m.max_n1 = m.max_n2 = m.max_n3 = m.max_n12 = m.max_nb = 0;
  for (size_t i = 0; i < counts.size() && i < ctx_.size(); ++i) {
    if (!counts[i]) continue;
    const Prob& d = ctx_[i]->d;
    m.max_n1 = std::max(m.max_n1, d.n1);
    m.max_n2 = std::max(m.max_n2, d.n2);
    m.max_n3 = std::max(m.max_n3, d.n3);
    m.max_n12 = std::max(m.max_n12, d.n1 * d.n2);
    m.max_nb = std::max(m.max_nb, d.nb);
  }
  int* d = nullptr;
  if (!cuda_ok(dev_malloc(&d, st.size() * sizeof(int)), "dev_malloc(map)")) return m;
  cudaMemcpy(d, st.data(), st.size() * sizeof(int), cudaMemcpyHostToDevice);
  allocs_.push_back(d);
  m.start = d;
  return m;
}

// Maps of the GEMMs whose CTA counts follow the tile knobs.
void Engine::build_gemm_maps() {
  std::vector<int> ww, bw, dw, tc, nntc;
  for (auto* c : ctx_) {
    const Prob& d = c->d;
    const int nsplit = div_up(d.npw, tn_kc_);
    const int tw = div_up(d.nb, TN_TILE), ta = div_up(d.nproj, TN_TILE), td = div_up(3 * d.nproj, TN_TILE);
    ww.push_back(tw * tw * nsplit);
    bw.push_back(ta * tw * nsplit);
    dw.push_back(td * tw * nsplit);
    tc.push_back(div_up(d.npw, tc_kc_));
    nntc.push_back(div_up(div_up(d.npw, 128), nn_tpc_));
  }
  m_tn_ww_ = make_map(ww);
  m_tn_bw_ = make_map(bw);
  m_tn_dw_ = make_map(dw);
  m_tc_ = make_map(tc);
  m_nntc_ = make_map(nntc);
}

// Autotuner of the GEMM tile knobs (mixed path): for each knob, every candidate runs its
// GEMM on this batch's own buffers (one warm-up, then three timed launches on the
// engine's stream, CUDA events) and the fastest is kept.  The contents of the scratch
// matrices it overwrites are recomputed by every evaluation.
void Engine::autotune() {
  if (!ok_ || precision_ != 1) return;
  cudaEvent_t a = nullptr, b = nullptr;
  if (!cuda_ok(cudaEventCreate(&a), "autotune event") || !cuda_ok(cudaEventCreate(&b), "autotune event")) return;
  const long long l0 = launches_;
  auto time_of = [&](auto&& fn) {
    fn();
    cudaEventRecord(a, stream_);
    for (int r = 0; r < 3; ++r) fn();
    cudaEventRecord(b, stream_);
    cudaEventSynchronize(b);
    float ms = 1e30f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) ms = 1e30f;
    return ms;
  };
  auto pick = [&](int* knob, std::initializer_list<int> cands, auto&& fn) {
    int best = *knob;
    float tbest = 1e30f;
    for (int v : cands) {
      *knob = v;
      build_gemm_maps();
      const float t = time_of(fn);
      if (t < tbest) {
        tbest = t;
        best = v;
      }
    }
    *knob = best;
    build_gemm_maps();
  };
  if (tc_ok_[OPK_WB]) pick(&tc_kc_, {256, 512, 1024, 2048}, [&] { tn<float>(OPK_WB, WB_X, OPK_WB, WB_HX, DD_HS); });
  pick(&tn_kc_, {128, 256, 512}, [&] { tn<float>(OPK_WB, WB_X, OPK_WB, WB_X, DD_S, false); });
  if (nn_tc_ok_[OPK_WB]) pick(&nn_tpc_, {2, 4, 8, 16}, [&] { nn<float>(OPK_WB, WB_X, DD_TM, WB_W, 1.0, 0.0); });
  cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  launches_ = l0;
}

Launch Engine::L(const WorkMap& m) const {
  if (m.total > 0) ++launches_;  // an empty map launches nothing
  Launch l;
  l.ka = KArgs{d_probs_, m.start ? m.start : m_prob_.start, n_, d_active_};
  l.map = m;
  l.stream = stream_;
  l.max_n1 = m.max_n1 >= 0 ? m.max_n1 : max_n1_;
  l.max_n2 = m.max_n2 >= 0 ? m.max_n2 : max_n2_;
  l.max_n3 = m.max_n3 >= 0 ? m.max_n3 : max_n3_;
  l.max_n12 = m.max_n12 >= 0 ? m.max_n12 : max_n12_;
  l.max_nb = m.max_nb >= 0 ? m.max_nb : max_nb_;
  l.plane_threads = plane_threads_;
  l.wait_ns = wait_ns_;
  return l;
}

Engine::Engine(const std::vector<sgo_ctx*>& ctxs, cudaStream_t stream) : ctx_(ctxs), stream_(stream) {
  n_ = (int)ctxs.size();
  if (n_ == 0) return;
  precision_ = ctxs[0]->precision;
  for (auto* c : ctxs) {
    if (c->precision != precision_) {
      set_error("all members of a batch must use the same precision");
      return;
    }
    if (c->opts.eigensolver != ctxs[0]->opts.eigensolver || c->opts.xc != ctxs[0]->opts.xc) {
      set_error("all members of a batch must use the same eigensolver and exchange-correlation");
      return;
    }
  }
  std::vector<Prob> host(n_);
  std::vector<int> c_zcol, c_plane, c_dens, c_gz, c_gp, c_gew, c_gch, c_bands, c_tnww, c_tnbw, c_tndw, c_rww, c_rbw,
      c_rdw, c_nn, c_atoms, c_projs, c_atomch, c_ewsg, c_prob, c_tc, c_nntc, c_preg[2], c_dreg[2], c_zreg[2], c_ppair,
      c_dpair, c_zpair, c_gx, c_gy, c_bigy, c_bigx, c_bigdy, c_bigd;
  size_t part = 0;
  int max_nproj = 0;
  for (int p = 0; p < n_; ++p) {
    const Prob& d = ctxs[p]->d;
    host[p] = d;
    max_n1_ = std::max(max_n1_, d.n1);
    max_n2_ = std::max(max_n2_, d.n2);
    max_n3_ = std::max(max_n3_, d.n3);
    max_n12_ = std::max(max_n12_, d.n1 * d.n2);
    max_nb_ = std::max(max_nb_, d.nb);
    const int nch = div_up(d.ngrid, GRID_CHUNK);
    maxchunk_ = std::max(maxchunk_, nch);
    const int nsplit = div_up(d.npw, 128);  // the smallest CUDA-core K chunk the autotuner tries
    // z-column passes: register FFTs on the mixed path where n3 has one (single thread or
    // lane pair per line), the shared-memory engine otherwise
    const bool zreg = precision_ == 1 && zreg_ok(d.n3);
    const bool zpair = precision_ == 1 && !zreg && zpair_ok(d.n3);
    c_zcol.push_back(zreg || zpair ? 0 : d.npair * div_up(d.ncp, QCP));
    for (int k = 0; k < 2; ++k) c_zreg[k].push_back(zreg && zreg_class(d.n3) == k ? zreg_ctas(d.ncp, d.npair) : 0);
    if (zreg) zreg_smem_[zreg_class(d.n3)] = std::max(zreg_smem_[zreg_class(d.n3)], zreg_smem(d.n3));
    c_zpair.push_back(zpair ? zpair_ctas(d.ncp, d.npair) : 0);
    if (zpair) zpair_smem_ = std::max(zpair_smem_, zpair_smem(d.n3));
    // FP64 grid transforms: a whole plane per CTA when two planes fit in shared memory,
    // otherwise line blocks along x and y
    const bool gbig = (size_t)(2 * d.n1 * d.n2 + d.n1 + d.n2) * 16 > 220 * 1024;
    c_gx.push_back(gbig ? div_up(d.n3 * d.n2, QZ) : 0);
    c_gy.push_back(gbig ? div_up(d.n3 * d.n1, QZ) : 0);
    // plane passes: register FFTs on the mixed path where both plane lengths have one
    // and the kernels' shared memory fits; the shared-memory engine otherwise
    const PlanePaths pp = plane_paths(d, precision_);
    const bool preg = pp.preg, dreg = pp.dreg, ppair = pp.ppair, dpair = pp.dpair;
    const int pcls = preg ? plane_reg_class(d.n1, d.n2) : -1;
    if ((pp.pbig || pp.dbig) && !d.Gp) {
      set_error("big-plane buffer missing (the context was built for another precision)");
      return;
    }
    c_plane.push_back(preg || ppair || pp.pbig ? 0 : d.npair * d.n3);
    c_dens.push_back(dreg || dpair || pp.dbig ? 0 : d.n3);
    c_bigy.push_back(pp.pbig ? big_y_ctas(d.npair, d.n3, d.m1max) : 0);
    c_bigx.push_back(pp.pbig ? big_x_ctas(d.npair, d.n3, d.n2) : 0);
    c_bigdy.push_back(pp.dbig ? big_y_ctas(d.npair, d.n3, d.m1max) : 0);
    c_bigd.push_back(pp.dbig ? big_density_ctas(d.n3, d.n2) : 0);
    c_ppair.push_back(ppair ? pair_plane_ctas(d.n2, d.n3, d.npair) : 0);
    c_dpair.push_back(dpair ? pair_density_ctas(d.n2, d.n3) : 0);
    if (ppair) ppair_smem_ = std::max(ppair_smem_, pair_plane_smem(d.n1, d.n2, d.m1max));
    if (dpair) dpair_smem_ = std::max(dpair_smem_, pair_density_smem(d.n1, d.n2, d.m1max));
    for (int k = 0; k < 2; ++k) {
      c_preg[k].push_back(pcls != k ? 0
                          : kPlaneMultiPass ? plane_ms_ctas(d.n1, d.n2, d.n3, d.npair)
                                            : plane_reg_ctas(d.n2, d.n3, d.npair));
      c_dreg[k].push_back(dreg && pcls == k ? plane_density_reg_ctas(d.n2, d.n3) : 0);
    }
    if (preg)
      preg_smem_[pcls] = std::max(preg_smem_[pcls], kPlaneMultiPass ? plane_ms_smem(d.n1, d.n2, d.n3)
                                                                    : plane_reg_smem(d.n1, d.n2, d.m1max));
    if (dreg) dreg_smem_[pcls] = std::max(dreg_smem_[pcls], plane_density_reg_smem(d.n1, d.n2, d.m1max));
    c_gz.push_back(div_up(d.n1 * d.n2, QZ));
    c_gp.push_back(gbig ? 0 : d.n3);
    c_gew.push_back(div_up(d.ngrid, GRID_EW_POINTS));
    c_gch.push_back(nch);
    c_bands.push_back(d.nb);
    c_rww.push_back(div_up(d.nb * d.nb, 256));
    c_rbw.push_back(div_up(d.nproj * d.nb, 256));
    c_rdw.push_back(div_up(3 * d.nproj * d.nb, 256));
    c_nn.push_back(div_up(d.npw, 64 * NN_RT) * div_up(d.nb, 64));
    c_atoms.push_back(d.natom);
    c_projs.push_back(d.nproj);
    c_atomch.push_back(div_up(d.natom, LF_GROUP) * nch);
    c_ewsg.push_back(div_up(ctxs[p]->ngbox_ew, 256));
    c_prob.push_back(1);
    max_nproj = std::max(max_nproj, d.nproj);
    size_t need = (size_t)nsplit * std::max({d.nb * d.nb, d.nproj * d.nb, 3 * d.nproj * d.nb});
    part = std::max(part, need);
  }
  plane_threads_ = PLANE_THREADS;
  m_zcol_ = make_map(c_zcol);
  m_plane_ = make_map(c_plane);
  for (int k = 0; k < 2; ++k) m_preg_[k] = make_map(c_preg[k]);
  for (int k = 0; k < 2; ++k) m_dreg_[k] = make_map(c_dreg[k]);
  for (int k = 0; k < 2; ++k) m_zreg_[k] = make_map(c_zreg[k]);
  m_ppair_ = make_map(c_ppair);
  m_dpair_ = make_map(c_dpair);
  m_zpair_ = make_map(c_zpair);
  m_gx_ = make_map(c_gx);
  m_gy_ = make_map(c_gy);
  m_bigy_ = make_map(c_bigy);
  m_bigx_ = make_map(c_bigx);
  m_bigdy_ = make_map(c_bigdy);
  m_bigd_ = make_map(c_bigd);
  m_dens_ = make_map(c_dens);
  m_gz_ = make_map(c_gz);
  m_gp_ = make_map(c_gp);
  m_gew_ = make_map(c_gew);
  m_gch_ = make_map(c_gch);
  m_bands_ = make_map(c_bands);
  m_red_ww_ = make_map(c_rww);
  m_red_bw_ = make_map(c_rbw);
  m_red_dw_ = make_map(c_rdw);
  m_nn_ = make_map(c_nn);
  m_atoms_ = make_map(c_atoms);
  m_projs_ = make_map(c_projs);
  m_atomch_ = make_map(c_atomch);
  m_ewsg_ = make_map(c_ewsg);
  m_prob_ = make_map(c_prob);
  // tensor-core subspace GEMMs: mixed path, every operand count <= 128 (one M tile, one
  // NN image of at most 128 x 128), at least two NN pipeline stages beside the image
  const bool tc = precision_ == 1 && ctxs[0]->opts.gemm_tc != 0;
  tc_ok_[OPK_WB] = tc && max_nb_ <= 128;
  tc_ok_[OPK_B] = tc && max_nb_ <= 128 && max_nproj <= 128;
  tc_ok_[OPK_DB] = tc && max_nb_ <= 128 && 3 * max_nproj <= 128;
  const int nin_max[3] = {max_nb_, max_nproj, 3 * max_nproj};
  for (int k = 0; k < 3; ++k) {
    nnimg_max_[k] = nn_tc_image_bytes(nin_max[k], max_nb_);
    nn_tc_ok_[k] = tc_ok_[k] && nn_tc_stages(nnimg_max_[k]) >= 2;
  }
  part_stride_ = part;
  build_gemm_maps();
  if (!cuda_ok(dev_malloc(&d_probs_, sizeof(Prob) * n_), "dev_malloc(probs)")) return;
  allocs_.push_back(d_probs_);
  cudaMemcpy(d_probs_, host.data(), sizeof(Prob) * n_, cudaMemcpyHostToDevice);
  if (!cuda_ok(dev_malloc(&d_active_, sizeof(int) * n_), "dev_malloc(active)")) return;
  allocs_.push_back(d_active_);
  h_active_.assign(n_, 1);
  cudaMemcpy(d_active_, h_active_.data(), sizeof(int) * n_, cudaMemcpyHostToDevice);
  if (!cuda_ok(dev_malloc(&d_part_, sizeof(double) * part_stride_ * n_), "dev_malloc(part)")) return;
  allocs_.push_back(d_part_);
  if (!cuda_ok(dev_malloc(&d_gpart_, sizeof(double) * (size_t)maxchunk_ * n_ * 8), "dev_malloc(gpart)")) return;
  allocs_.push_back(d_gpart_);
  if (!cuda_ok(dev_malloc(&d_flags_, sizeof(double) * 4 * n_), "dev_malloc(flags)")) return;
  allocs_.push_back(d_flags_);
  if (!cuda_ok(dev_malloc(&d_iter_, 2 * sizeof(int)), "dev_malloc(iter)")) return;
  allocs_.push_back(d_iter_);
  if (!cuda_ok(dev_malloc(&d_saved_, sizeof(int) * n_), "dev_malloc(saved mask)")) return;
  allocs_.push_back(d_saved_);
  if (tc) {
    // TMA descriptors of every operand buffer (fixed for the engine's life; role swaps
    // select among them on the device) and the NN image scratch
    const size_t per = (size_t)TC_NSLOT * TC_NMAPKIND * tc_map_bytes();
    std::vector<unsigned char> hm(per * n_);
    for (int p = 0; p < n_; ++p)
      if (!tc_encode_maps(host[p], hm.data() + per * p)) return;
    if (!cuda_ok(dev_malloc(&d_tmaps_, hm.size()), "dev_malloc(tensor maps)")) return;
    allocs_.push_back(d_tmaps_);
    cudaMemcpy(d_tmaps_, hm.data(), hm.size(), cudaMemcpyHostToDevice);
    nnimg_stride_ = (size_t)(*std::max_element(nnimg_max_, nnimg_max_ + 3) + 1023) / 1024 * 256;  // floats
    if (!cuda_ok(dev_malloc(&d_nnimg_, sizeof(float) * nnimg_stride_ * n_), "dev_malloc(nn image)")) return;
    allocs_.push_back(d_nnimg_);
  }
  {
    // pinned read-back area, and the default slots (the engine is the whole batch)
    size_t nd = 4 * (size_t)n_;
    hp_off_.resize(n_);
    for (int p = 0; p < n_; ++p) {
      hp_off_[p] = nd;
      nd += NSCAL_ALL + 2 * (size_t)ctxs[p]->d.nb + ctxs[p]->h_forces.size();
    }
    if (!cuda_ok(cudaMallocHost(&hp_, sizeof(double) * nd), "cudaMallocHost(read-back)")) return;
    std::memset(hp_, 0, sizeof(double) * nd);
    if (!cuda_ok(cudaMallocHost(&hpi_, sizeof(int) * (2 + 4 * (size_t)n_)), "cudaMallocHost(read-back)")) return;
    std::memset(hpi_, 0, sizeof(int) * (2 + 4 * (size_t)n_));
    if (!cuda_ok(dev_malloc(&d_slot_, sizeof(int) * 2 * n_), "dev_malloc(slots)")) return;
    allocs_.push_back(d_slot_);
    d_foff_ = d_slot_ + n_;
    std::vector<int> slot(n_), foff(n_);
    for (int p = 0, o = 0; p < n_; o += 3 * ctxs[p]->d.natom, ++p) {
      slot[p] = p;
      foff[p] = o;
    }
    if (!set_slots(slot, foff)) return;
  }
  // mixed path: the FP32 eigensolve (its five matrices in shared memory up to nb = 105,
  // else in a per-member global scratch; the Jacobi pair tables allow nb <= 512)
  const sgo_opts& o0 = ctxs[0]->opts;
  wait_ns_ = o0.watchdog_ms > 0.0 ? (long long)(o0.watchdog_ms * 1e6) : 2000000000LL;
  // subspace diagonalisation: one CTA per member with its matrices in shared memory (FP32
  // deviation form up to nb = 105 on the mixed path, FP64 up to nb = 91), else one
  // thread-block cluster per member over a global scratch (k_rr_cluster)
  // (the block Davidson steps diagonalise the 2 n_b block [X, W])
  davidson_ = o0.eigensolver == 1;
  cg_adapt_ = o0.cg_adapt;
  gga_ = o0.xc == 1;
  rr_n_ = (davidson_ ? 2 : 1) * max_nb_;
  rr_f32_ = precision_ == 1 && !o0.rr_fp64;
  rr_smem_bytes_ = (size_t)3 * rr_n_ * rr_n_ * sizeof(double);
  rr_smem_ = rr_f32_ ? (size_t)20 * rr_n_ * (rr_n_ | 1) <= 216 * 1024 : rr_smem_bytes_ <= 200 * 1024;
  // (the one-CTA kernels' pair tables hold 256 pairs: beyond 512 bands the cluster is used)
  rr_cluster_ = o0.rr_cluster > 0 || (o0.rr_cluster < 0 && !rr_smem_) || rr_n_ > 512;
  if (rr_cluster_) {
    rrc_stride_ = (rr_cluster_scratch_bytes(rr_n_, rr_f32_ ? sizeof(float) : sizeof(double)) + 255) / 256 * 256;
    if (!cuda_ok(dev_malloc(&d_rrc_, rrc_stride_ * n_), "dev_malloc(rr cluster scratch)")) return;
    allocs_.push_back(d_rrc_);
  } else if (!rr_smem_) {  // one CTA over a global scratch
    rr1_stride_ = rr_f32_ ? (size_t)5 * rr_n_ * (rr_n_ | 1) * sizeof(float) : (size_t)3 * rr_n_ * rr_n_ * sizeof(double);
    if (!cuda_ok(dev_malloc(&d_rr1_, rr1_stride_ * n_), "dev_malloc(rr scratch)")) return;
    allocs_.push_back(d_rr1_);
  }
  // (a refused shared-memory limit would otherwise surface only as a failed launch later)
  if (!cuda_ok(cudaGetLastError(), "engine set-up")) return;
  fft_set_smem_limits(220 * 1024);
  linalg_set_smem_limits(220 * 1024);
  gemm_tc_set_smem_limits();
  if (!cuda_ok(cudaGetLastError(), "kernel shared-memory limits")) return;
  if (precision_ == 1 && !fft_reg_init()) {
    set_error("register FFT twiddle tables: upload failed");
    return;
  }
  ok_ = cuda_ok(cudaGetLastError(), "engine set-up");
}

Engine::~Engine() {
  if (g_nonscf_) cudaGraphExecDestroy(g_nonscf_);
  if (g_scf_) cudaGraphExecDestroy(g_scf_);
  if (g_polish_) cudaGraphExecDestroy(g_polish_);
  if (g_tail_) cudaGraphExecDestroy(g_tail_);
  if (ev_in_) cudaEventDestroy(ev_in_);
  if (ev_out_) cudaEventDestroy(ev_out_);
  if (own_stream_) cudaStreamDestroy(own_stream_);
  if (hp_) cudaFreeHost(hp_);
  if (hpi_) cudaFreeHost(hpi_);
  for (auto& v : ev_) cudaEventDestroy(v);
  if (!allocs_.empty()) cudaDeviceSynchronize();  // once for all the blocks below
  for (void* p : allocs_) dev_free(p, true);
}

// ---- live kernel timing ----
bool Engine::timer_select(const char* name) {
  timer_kind_ = -1;
  for (int k = 0; k < TK_COUNT; ++k)
    if (name && std::strcmp(name, kTimerNames[k]) == 0) timer_kind_ = k;
  if (timer_kind_ >= 0 && ev_.empty()) {
    ev_.resize(8192);
    for (auto& v : ev_) cudaEventCreate(&v);
    ev_bytes_.resize(ev_.size() / 2);
    ev_flops_.resize(ev_.size() / 2);
  }
  ev_used_ = 0;
  t_ms_ = t_bytes_ = t_flops_ = 0.0;
  t_launches_ = 0;
  return timer_kind_ >= 0 || name == nullptr;
}

void Engine::tbeg(int kind) {
  if (kind != timer_kind_ || ev_used_ + 2 > (int)ev_.size()) return;
  cudaEventRecord(ev_[ev_used_], stream_);
}

void Engine::tend(int kind) {
  if (kind != timer_kind_ || ev_used_ + 2 > (int)ev_.size()) return;
  cudaEventRecord(ev_[ev_used_ + 1], stream_);
  work_of(kind, &ev_bytes_[ev_used_ / 2], &ev_flops_[ev_used_ / 2]);
  ev_used_ += 2;
}

// Harvest the recorded pairs (the stream is synchronised at the end of every run).
void Engine::timer_read(double* ms, int* launches, double* bytes, double* flops) {
  for (int i = 0; i + 1 < ev_used_; i += 2) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, ev_[i], ev_[i + 1]) == cudaSuccess) {
      t_ms_ += t;
      t_bytes_ += ev_bytes_[i / 2];
      t_flops_ += ev_flops_[i / 2];
      ++t_launches_;
    }
  }
  ev_used_ = 0;
  if (ms) *ms = t_ms_;
  if (launches) *launches = t_launches_;
  if (bytes) *bytes = t_bytes_;
  if (flops) *flops = t_flops_;
}

// Algorithmic work of one launch over the active members: the bytes each kernel must move
// to and from device memory at least once and its arithmetic (5 N log2 N per complex FFT
// of length N; 2 m n k per GEMM).
void Engine::work_of(int kind, double* bytes, double* flops) const {
  double b = 0.0, f = 0.0;
  const double ts = precision_ ? 4.0 : 8.0;
  for (int p = 0; p < n_; ++p) {
    if (!h_active_[p]) continue;
    const Prob& d = ctx_[p]->d;
    const double n1 = d.n1, n2 = d.n2, n3 = d.n3, np = d.npair, nc = d.ncol, nb = d.nb, npw = d.npw;
    const double rows = 2.0 * d.m1max + 1.0;
    switch (kind) {
      case TK_PLANE_VPSI:
        f += np * n3 * (2.0 * rows * 5.0 * n2 * log2d(n2) + 2.0 * n2 * 5.0 * n1 * log2d(n1) + 2.0 * n1 * n2);
        b += np * n3 * (2.0 * nc * 2.0 * ts + n1 * n2 * ts);
        break;
      case TK_PLANE_DENSITY:
        f += np * n3 * (rows * 5.0 * n2 * log2d(n2) + n2 * 5.0 * n1 * log2d(n1) + 4.0 * n1 * n2);
        b += np * n3 * nc * 2.0 * ts + n1 * n2 * n3 * 8.0;
        break;
      case TK_WAVE_TO_COLS:
        f += np * nc * 5.0 * n3 * log2d(n3);
        b += 2.0 * np * npw * ts + np * nc * n3 * 2.0 * ts;
        break;
      case TK_COLS_TO_WAVE:
        f += np * nc * 5.0 * n3 * log2d(n3);
        b += np * nc * n3 * 2.0 * ts + 4.0 * np * npw * ts + npw * 8.0;
        break;
      case TK_GEMM_TN:
        f += 2.0 * nb * nb * npw;
        b += 2.0 * nb * npw * ts;
        break;
      case TK_GEMM_NN:
        f += 2.0 * npw * nb * nb * work_mult_;
        b += 2.0 * nb * npw * ts * work_mult_;
        break;
      case TK_RR:  // (work_mult_ = 8 for the 2 n_b block)
        f += 4.0 * nb * nb * nb * work_mult_;
        b += 3.0 * nb * nb * 8.0 * work_mult_;
        break;
    }
  }
  *bytes = b;
  *flops = f;
}

void Engine::swap_roles(int a, int b) { k_swap_roles<<<n_, 32, 0, stream_>>>(L(m_prob_).ka, role_pair(a, b)); }

void Engine::set_scal(int idx, double v, bool only_active) {
  k_set_scal<<<n_, 32, 0, stream_>>>(L(m_prob_).ka, idx, v, only_active ? 1 : 0);
}

void Engine::grid_fft(int which, int sign, bool fp32) {
  tbeg(TK_GRID_FFT);
  // the mixed path's FP64 grids are transformed in float-float arithmetic (FP64 runs at
  // about 1/64 of the FP32 rate on this GPU); the plain path stays FP64 throughout
  if (fp32) grid_fft_raw<float>(which, sign);
  else if (precision_) grid_fft_raw<ff>(which, sign);
  else grid_fft_raw<double>(which, sign);
  tend(TK_GRID_FFT);
}

template <typename T>
void Engine::grid_fft_raw(int which, int sign) {
  // forward: planes (y, x), then z; inverse: z, then planes.  Large planes go by line
  // blocks along y and x.
  auto planes = [&](int sg) {
    launch_grid_plane_fft<T>(L(m_gp_), which, sg);
    launch_grid_line_fft<T>(L(m_gy_), which, sg, 1);
    launch_grid_line_fft<T>(L(m_gx_), which, sg, 0);
  };
  if (sign < 0) {
    planes(-1);
    launch_grid_z_fft<T>(L(m_gz_), which, -1);
  } else {
    launch_grid_z_fft<T>(L(m_gz_), which, 1);
    planes(1);
  }
}

// allow_tc = false keeps a product off the tensor cores: the energy and force overlaps
// feed F and the forces directly, where 3xTF32 noise would exceed the SCF tolerance.
template <typename T>
void Engine::tn(int akind, int arole, int bkind, int brole, int dst, bool allow_tc) {
  const WorkMap* m = &m_tn_ww_;
  const WorkMap* r = &m_red_ww_;
  if (akind == OPK_B) { m = &m_tn_bw_; r = &m_red_bw_; }
  if (akind == OPK_DB) { m = &m_tn_dw_; r = &m_red_dw_; }
  const int kind = akind == OPK_WB ? TK_GEMM_TN : TK_GEMM_SMALL;
  tbeg(kind);
  if (sizeof(T) == 4 && allow_tc && tc_ok_[akind]) {
    launch_gemm_tn_tc(L(m_tc_), d_tmaps_, akind, arole, bkind, brole, d_part_, part_stride_, tc_kc_);
    launch_gemm_tn_reduce(L(*r), akind, bkind, dst, d_part_, part_stride_, tc_kc_);
  } else {
    launch_gemm_tn<T>(L(*m), akind, arole, bkind, brole, d_part_, part_stride_, tn_kc_);
    launch_gemm_tn_reduce(L(*r), akind, bkind, dst, d_part_, part_stride_, tn_kc_, akind == bkind && arole == brole);
  }
  tend(kind);
}

// image_ready: the previous NN call built the tensor-core image of the same matrix.
template <typename T>
void Engine::nn(int akind, int arole, int msel, int yrole, double alpha, double beta, bool image_ready) {
  nn_pairs<T>(akind, role_pair(arole, yrole), msel, alpha, beta, image_ready);
}

// One launch maps every (source, destination) role pair of rp through the same matrix.
template <typename T>
void Engine::nn_pairs(int akind, const RolePairs& rp, int msel, double alpha, double beta, bool image_ready) {
  const int kind = akind == OPK_WB ? TK_GEMM_NN : TK_GEMM_SMALL;
  tbeg(kind);
  if (sizeof(T) == 4 && nn_tc_ok_[akind]) {
    if (!image_ready) launch_nn_image(L(m_prob_), akind, msel, d_nnimg_, nnimg_stride_);
    launch_gemm_nn_tc(L(m_nntc_), d_tmaps_, d_nnimg_, nnimg_stride_, nnimg_max_[akind], akind, rp, alpha, beta,
                      nn_tpc_);
  } else {
    launch_gemm_nn<T>(L(m_nn_), akind, rp, msel, alpha, beta);
  }
  work_mult_ = rp.n;
  tend(kind);
  work_mult_ = 1;
}

// Psi <- Psi Tm for the block and its companions in one NN launch: every source role of
// rp is rotated into its destination role (a buffer whose contents are dead), then the
// pairs listed in swap exchange roles, so that each rotated block sits under its source's
// role again (a pair left out of swap keeps the rotated block under the destination).
template <typename T>
void Engine::rotate_pairs(const RolePairs& rp, const RolePairs& swap) {
  nn_pairs<T>(OPK_WB, rp, DD_TM, 1.0, 0.0, false);
  if (swap.n > 0) k_swap_roles<<<n_, 32, 0, stream_>>>(L(m_prob_).ka, swap);
}

// z-column passes: shared-memory engine for the members without a register transform of
// n3 (or on the FP64 path), register kernels for the others.
template <typename T>
void Engine::wave_to_cols(int src) {
  launch_wave_to_cols<T>(L(m_zcol_), src);
  if (sizeof(T) == 4) {
    for (int k = 0; k < 2; ++k) launch_wave_to_cols_reg(L(m_zreg_[k]), k, zreg_smem_[k], src);
    launch_wave_to_cols_pair(L(m_zpair_), zpair_smem_, src);
  }
}

template <typename T>
void Engine::cols_to_wave(int src, int dst) {
  launch_cols_to_wave<T>(L(m_zcol_), src, dst);
  if (sizeof(T) == 4) {
    for (int k = 0; k < 2; ++k) launch_cols_to_wave_reg(L(m_zreg_[k]), k, zreg_smem_[k], src, dst);
    launch_cols_to_wave_pair(L(m_zpair_), zpair_smem_, src, dst);
  }
}

// H applied to every band of src: FFT local + kinetic, then nonlocal B (D o B^T src).
template <typename T>
void Engine::hpsi(int src, int dst) {
  tbeg(TK_WAVE_TO_COLS);
  wave_to_cols<T>(src);
  tend(TK_WAVE_TO_COLS);
  tbeg(TK_PLANE_VPSI);
  launch_plane_vpsi<T>(L(m_plane_));
  for (int k = 0; k < 2; ++k) {
    if (kPlaneMultiPass) launch_plane_vpsi_ms(L(m_preg_[k]), preg_smem_[k]);
    else launch_plane_vpsi_reg(L(m_preg_[k]), k, preg_smem_[k]);
  }
  launch_plane_vpsi_pair(L(m_ppair_), ppair_smem_);
  launch_big_y<T>(L(m_bigy_), 1, 0, nullptr);
  launch_big_x<T>(L(m_bigx_));
  launch_big_y<T>(L(m_bigy_), -1, 0, nullptr);
  tend(TK_PLANE_VPSI);
  tbeg(TK_COLS_TO_WAVE);
  cols_to_wave<T>(src, dst);
  tend(TK_COLS_TO_WAVE);
  tn<T>(OPK_B, 0, OPK_WB, src, DD_PROJ);
  nn<T>(OPK_B, 0, DD_PROJ_D, dst, 1.0, 1.0);
}

// Overlap + subspace matrix, FP64 Cholesky/eigensolve, rotation of the block.
template <typename T>
void Engine::rayleigh_ritz(bool rotate_history) {
  // the overlap sets the norms of the bands and hence rho and F: CUDA-core FP32 (about 1e-7
  // relative); the tensor cores' 3xTF32 (about 5e-7) would leave F drifting above tol_e
  tn<T>(OPK_WB, WB_X, OPK_WB, WB_X, DD_S, false);
  tn<T>(OPK_WB, WB_X, OPK_WB, WB_HX, DD_HS);
  rr_solve(1);
  // P and HP (the last search direction and its H image) and W are dead here; so is RP
  // (after a CG step the new residual waits in W2 and the old one in RP is done with): one
  // launch rotates X -> P, HX -> HP and, with the CG history, PP -> W and the new residual
  // W2 -> RP; the role swaps put the rotated blocks under X, HX and PP.
  if (rotate_history)
    rotate_pairs<T>(RolePairs{4, {WB_X, WB_HX, WB_PP, WB_W2}, {WB_P, WB_HP, WB_W, WB_RP}},
                    RolePairs{3, {WB_X, WB_HX, WB_PP, 0}, {WB_P, WB_HP, WB_W, 0}});
  else
    rotate_pairs<T>(RolePairs{2, {WB_X, WB_HX, 0, 0}, {WB_P, WB_HP, 0, 0}},
                    RolePairs{2, {WB_X, WB_HX, 0, 0}, {WB_P, WB_HP, 0, 0}});
}

// Cholesky, congruence and eigensolve of the blk n_b subspace (blk = 2: the block [X, W]).
void Engine::rr_solve(int blk) {
  tbeg(TK_RR);
  work_mult_ = blk * blk * blk;
  // (the 2 n_b block is far from diagonal: its FP32 Jacobi gets the full sweep cap)
  const int cap = blk == 2 ? 30 : rr_cap_;
  if (rr_cluster_) {
    const Launch l = L(m_prob_);
    const bool launched = rr_f32_ ? launch_rr_cluster<float>(l, rr_n_, d_rrc_, rrc_stride_, cap, blk)
                                  : launch_rr_cluster<double>(l, rr_n_, d_rrc_, rrc_stride_, 30, blk);
    if (!launched) set_error("cluster Rayleigh-Ritz launch refused");
  } else if (rr_f32_) {  // 5 FP32 n x (n|1) matrices in shared memory or a global scratch
    launch_rr_f32(L(m_prob_), (size_t)20 * rr_n_ * (rr_n_ | 1), reinterpret_cast<float*>(d_rr1_),
                  rr1_stride_ / sizeof(float), cap, blk);
  } else {
    launch_rr(L(m_prob_), rr_smem_ ? 1 : 0, rr_smem_bytes_, reinterpret_cast<double*>(d_rr1_),
              rr1_stride_ / sizeof(double), 30, blk);
  }
  tend(TK_RR);
  work_mult_ = 1;
}

// Block Davidson step (the eigensolver alternative to Algorithm 1's CG step): the
// preconditioned residuals W = K (H X - X eps) of every band, without conjugation, projected
// on the complement of X and normalised; H W; then one Rayleigh-Ritz over the 2 n_b block
// [X, W] that keeps its lowest n_b Ritz pairs: X <- X C_X + W C_W, HX <- HX C_X + HW C_W.
// Its eigensolve is 8x the n_b one (and on the FP64 path runs at the FP64 rate).
template <typename T>
void Engine::davidson_step() {
  tbeg(TK_CG_BAND);
  launch_cg_precond<T>(L(m_bands_), WB_X, WB_HX, WB_P, WB_W2, WB_PP, -1);
  tend(TK_CG_BAND);
  tn<T>(OPK_WB, WB_X, OPK_WB, WB_P, DD_CM);
  nn<T>(OPK_WB, WB_X, DD_CM, WB_P, -1.0, 1.0);
  tbeg(TK_CG_BAND);
  launch_normalize<T>(L(m_bands_), WB_P, -1);
  tend(TK_CG_BAND);
  hpsi<T>(WB_P, WB_HP);
  // the blocks of S2 = [X W]^T [X W] and H2 = [X W]^T [HX HW] (overlaps on CUDA cores)
  tn<T>(OPK_WB, WB_X, OPK_WB, WB_X, DD_S, false);
  tn<T>(OPK_WB, WB_X, OPK_WB, WB_HX, DD_HS);
  tn<T>(OPK_WB, WB_X, OPK_WB, WB_P, DD_TM, false);
  tn<T>(OPK_WB, WB_X, OPK_WB, WB_HP, DD_CM);
  launch_rr2_assemble(L(m_red_ww_), 0);
  tn<T>(OPK_WB, WB_P, OPK_WB, WB_P, DD_S, false);
  tn<T>(OPK_WB, WB_P, OPK_WB, WB_HP, DD_HS);
  launch_rr2_assemble(L(m_red_ww_), 1);
  rr_solve(2);
  // the Ritz vectors and their H images into the dead W, W2, which then take the roles of
  // X and HX
  nn_pairs<T>(OPK_WB, RolePairs{2, {WB_X, WB_HX, 0, 0}, {WB_W, WB_W2, 0, 0}}, DD_TM, 1.0, 0.0, false);
  nn_pairs<T>(OPK_WB, RolePairs{2, {WB_P, WB_HP, 0, 0}, {WB_W, WB_W2, 0, 0}}, DD_CM, 1.0, 1.0, false);
  k_swap_roles<<<n_, 32, 0, stream_>>>(L(m_prob_).ka, RolePairs{2, {WB_X, WB_HX, 0, 0}, {WB_W, WB_W2, 0, 0}});
}

// One all-band CG step of Algorithm 1: search directions, projection, line minimisation,
// Rayleigh-Ritz.
template <typename T>
void Engine::cg_step() {
  tbeg(TK_CG_BAND);
  launch_cg_precond<T>(L(m_bands_), WB_X, WB_HX, WB_P, WB_W2, WB_PP, WB_RP);
  tend(TK_CG_BAND);
  tn<T>(OPK_WB, WB_X, OPK_WB, WB_P, DD_CM);        // C = Psi^T P
  nn<T>(OPK_WB, WB_X, DD_CM, WB_P, -1.0, 1.0);     // P -= Psi C  (projection)
  tbeg(TK_CG_BAND);
  launch_normalize<T>(L(m_bands_), WB_P, WB_PP);
  tend(TK_CG_BAND);
  hpsi<T>(WB_P, WB_HP);
  tbeg(TK_CG_BAND);
  launch_line_min<T>(L(m_bands_), WB_X, WB_HX, WB_P, WB_HP);  // line minimisation
  tend(TK_CG_BAND);
  // orthonormalise + subspace diagonalisation; the residual of this step (in W2) becomes
  // the history RP, rotated with the bands (k_normalize has already moved <g, r> on)
  rayleigh_ritz<T>(true);
}

void Engine::sync_active() {
  k_gather_flags<<<n_, 32, 0, stream_>>>(L(m_prob_).ka, d_flags_);
  cudaMemcpyAsync(hp_, d_flags_, sizeof(double) * 4 * n_, cudaMemcpyDeviceToHost, stream_);
  cudaStreamSynchronize(stream_);
  for (int p = 0; p < n_; ++p) {
    if (!h_active_[p]) continue;
    if (hp_[4 * p] != 0.0 || hp_[4 * p + 1] != 0.0 || hp_[4 * p + 2] != 0.0) h_active_[p] = 0;
  }
  cudaMemcpyAsync(d_active_, h_active_.data(), sizeof(int) * n_, cudaMemcpyHostToDevice, stream_);
}

sgo_status Engine::structure_terms() {
  const Launch la = L(m_atoms_);
  launch_phases(la);
  launch_vion_g(L(m_gew_));
  grid_fft(0, 1);
  launch_grid_real_part(L(m_gew_), 0, 3);
  if (precision_) launch_build_projectors<float>(L(m_projs_), 0);
  else launch_build_projectors<double>(L(m_projs_), 0);
  launch_ewald(L(m_ewsg_), la, L(m_prob_));
  return cuda_ok(cudaGetLastError(), "structure terms") ? SGO_OK : SGO_ERR_CUDA;
}

// One SCF iteration up to the convergence test (Sec. II D): V_eff from rho_in, H Psi and
// the subspace diagonalisation that start Algorithm 1, ncg all-band CG steps, occupations,
// rho_out, the energy at (Psi, rho_out) and the per-member convergence test.
template <typename T>
void Engine::scf_iteration(int ncg, bool count_iter) {
  // V_eff from rho_in(G): one inverse transform of rho_in(G) + i V_H(G) gives
  // rho_in(r) + i V_H(r); LDA in real space
  // (in FP64 on both paths: an FP32 transform, measured, slows the SCF of some members:
  // its absolute error swamps rho_in(r) where the density is small, and v_xc follows it)
  tbeg(TK_GRID_OTHER);
  launch_potential_g<double>(L(m_gew_));
  if (gga_) launch_gga_grad(L(m_gew_), 0);
  tend(TK_GRID_OTHER);
  grid_fft(0, 1);
  if (gga_) {
    // PBE: grad rho_in (x + i y, z), then h = 2 de/dsigma grad rho to G space, div h back
    grid_fft(2, 1);
    grid_fft(3, 1);
    tbeg(TK_GRID_OTHER);
    launch_gga_point<T>(L(m_gew_));
    tend(TK_GRID_OTHER);
    grid_fft(2, -1);
    grid_fft(3, -1);
    tbeg(TK_GRID_OTHER);
    launch_gga_div(L(m_gew_));
    tend(TK_GRID_OTHER);
    grid_fft(3, 1);
  }
  tbeg(TK_GRID_OTHER);
  launch_veff<T>(L(m_gew_), nullptr);
  tend(TK_GRID_OTHER);
  hpsi<T>(WB_X, WB_HX);
  rayleigh_ritz<T>(false);
  set_scal(SC_FIRSTCG, 1.0, true);
  for (int k = 0; k < ncg; ++k) {
    // (cg_adapt: the last step only for members whose density residual is below it)
    const bool gate = count_iter && cg_adapt_ > 0.0 && ncg > 1 && k == ncg - 1;
    if (gate) k_cg_gate<<<1, 256, 0, stream_>>>(L(m_prob_).ka, d_active_, d_saved_, cg_adapt_, 0);
    eig_step<T>();
    if (gate) k_cg_gate<<<1, 256, 0, stream_>>>(L(m_prob_).ka, d_active_, d_saved_, cg_adapt_, 1);
  }
  density_energy<T>(count_iter ? 1 : 0);
}

// Occupations, rho_out, the energy at (Psi, rho_out) and (mode 1) the convergence test;
// mode 2 recomputes the energy of bands refined after the stopping rule held.
template <typename T>
void Engine::density_energy(int mode) {
  const sgo_opts& o = ctx_[0]->opts;
  // occupations and rho_out
  launch_occupations(L(m_prob_));
  wave_to_cols<T>(WB_X);
  tbeg(TK_PLANE_DENSITY);
  launch_plane_density<T>(L(m_dens_), nullptr);
  for (int k = 0; k < 2; ++k) launch_plane_density_reg(L(m_dreg_[k]), k, dreg_smem_[k], nullptr);
  launch_plane_density_pair(L(m_dpair_), dpair_smem_, nullptr);
  launch_big_y<T>(L(m_bigdy_), 1, 1, nullptr);
  launch_big_density<T>(L(m_bigd_), nullptr);
  tend(TK_PLANE_DENSITY);
  // energy at (Psi, rho_out) and the convergence test
  launch_band_kinetic<T>(L(m_bands_), WB_X);
  tn<T>(OPK_B, 0, OPK_WB, WB_X, DD_PROJ, false);
  tbeg(TK_GRID_OTHER);
  launch_real_to_grid(L(m_gew_), 1, 1);
  tend(TK_GRID_OTHER);
  grid_fft(1, -1);
  if (gga_) {  // PBE energy: grad rho_out
    tbeg(TK_GRID_OTHER);
    launch_gga_grad(L(m_gew_), 1);
    tend(TK_GRID_OTHER);
    grid_fft(2, 1);
    grid_fft(3, 1);
  }
  tbeg(TK_GRID_OTHER);
  launch_grid_energies<T>(L(m_gch_), d_gpart_, maxchunk_);
  launch_grid_energies_reduce(L(m_prob_), d_gpart_, maxchunk_);
  launch_finish_iteration(L(m_prob_), o.scf_tol_e, o.scf_tol_rho, mode);
  tend(TK_GRID_OTHER);
}

bool Engine::read_active() {
  cudaMemcpyAsync(h_active_.data(), d_active_, sizeof(int) * n_, cudaMemcpyDeviceToHost, stream_);
  cudaStreamSynchronize(stream_);
  for (int p = 0; p < n_; ++p)
    if (h_active_[p]) return true;
  return false;
}

// Host-driven form of the residual-controlled CG steps that follow the SCF loop (see
// k_polish_activate), then the density and energy of the refined bands.
template <typename T>
void Engine::polish() {
  const sgo_opts& o = ctx_[0]->opts;
  const int maxs = o.eig_tol > 0.0 ? std::max(0, o.max_polish) : 0;
  k_polish_activate<<<1, 256, 0, stream_>>>(L(m_prob_).ka, d_active_, 0);
  rr_cap_ = 30;
  for (int step = 0; step <= maxs; ++step) {
    tbeg(TK_CG_BAND);
    launch_band_residual<T>(L(m_bands_), WB_X, WB_HX);
    tend(TK_CG_BAND);
    k_polish_control<<<1, 256, 0, stream_>>>(L(m_prob_).ka, d_active_, nullptr, o.eig_tol, maxs, 0, 0);
    if (!read_active()) break;
    eig_step<T>();
  }
  rr_cap_ = 10;
  k_polish_activate<<<1, 256, 0, stream_>>>(L(m_prob_).ka, d_active_, 1);
  if (read_active()) density_energy<T>(2);
}

// Graph form: g_polish_ is one WHILE node (its condition starts at 1 on every launch)
// whose body tests the residuals (k_polish_control ends the loop when no member is left)
// and takes one all-band CG step for the members left (a pass in which none is left
// launches the step's kernels with every CTA masked out); g_tail_ picks the members that
// took a step and recomputes their density and energy.  k_polish_activate(mode 0) runs
// as a plain launch before g_polish_.
template <typename T>
bool Engine::build_polish_graphs() {
  const sgo_opts& o = ctx_[0]->opts;
  const int maxs = o.eig_tol > 0.0 ? std::max(0, o.max_polish) : 0;
  cudaGraph_t gp = nullptr, gt = nullptr, body = nullptr;
  cudaGraphConditionalHandle cond = 0;
  cudaGraphNode_t loop = nullptr;
  bool ok = cuda_ok(cudaGraphCreate(&gp, 0), "graph create") &&
            cuda_ok(cudaGraphConditionalHandleCreate(&cond, gp, 1, cudaGraphCondAssignDefault), "conditional handle");
  if (ok) {
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    ok = cuda_ok(cudaGraphAddNode(&loop, gp, nullptr, nullptr, 0, &cp), "polish while node");
    if (ok) body = cp.conditional.phGraph_out[0];
  }
  const long long l0 = launches_;
  ok = ok && cuda_ok(cudaStreamBeginCaptureToGraph(stream_, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
                     "capture polish body");
  if (ok) {
    rr_cap_ = 30;
    launch_band_residual<T>(L(m_bands_), WB_X, WB_HX);
    k_polish_control<<<1, 256, 0, stream_>>>(L(m_prob_).ka, d_active_, d_iter_ + 1, o.eig_tol, maxs, cond, 1);
    eig_step<T>();
    rr_cap_ = 10;
    cudaGraph_t got = nullptr;
    ok = cuda_ok(cudaStreamEndCapture(stream_, &got), "capture polish body end");
  }
  graph_launches_[2] = launches_ - l0;
  ok = ok && cuda_ok(cudaGraphInstantiate(&g_polish_, gp, 0), "graph instantiate (polish)");
  const long long l1 = launches_;
  ok = ok && cuda_ok(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal), "capture tail");
  if (ok) {
    k_polish_activate<<<1, 256, 0, stream_>>>(L(m_prob_).ka, d_active_, 1);
    density_energy<T>(2);
    ok = cuda_ok(cudaStreamEndCapture(stream_, &gt), "capture tail end");
  }
  graph_launches_[3] = launches_ - l1;
  launches_ = l0;
  ok = ok && cuda_ok(cudaGraphInstantiate(&g_tail_, gt, 0), "graph instantiate (tail)");
  if (gp) cudaGraphDestroy(gp);
  if (gt) cudaGraphDestroy(gt);
  if (!ok) {
    cudaGetLastError();
    if (g_polish_) cudaGraphExecDestroy(g_polish_);
    if (g_tail_) cudaGraphExecDestroy(g_tail_);
    g_polish_ = g_tail_ = nullptr;
  }
  return ok;
}

// Pulay mixing of rho_out with rho_in (members still iterating).
void Engine::pulay_step() {
  const sgo_opts& o = ctx_[0]->opts;
  const int hist = std::min(std::max(o.pulay_hist, 1), MAX_HIST);
  tbeg(TK_GRID_OTHER);
  launch_pulay_store(L(m_gew_));
  launch_pulay_gram(L(m_gch_), d_gpart_, maxchunk_, hist);
  launch_pulay_solve(L(m_prob_), d_gpart_, maxchunk_, hist);
  launch_pulay_mix(L(m_gew_), o.mix_alpha, o.kerker_q0);
  tend(TK_GRID_OTHER);
}

// Graph mode: the iteration sequence captured once per engine.
//   g_nonscf_: one iteration at the fixed initial potential (ncg_first CG steps, no count)
//              followed by k_scf_control; the host replays it n_nonscf times.
//   g_scf_:    k_scf_gate -> WHILE node whose body is one self-consistent iteration,
//              k_scf_control (which sets the loop condition) and the Pulay step.
// Kernel arguments (descriptor tables, maps, buffers) are fixed for the engine's life; the
// per-member state they point to (active masks, roles, scalars) is read at replay time.
template <typename T>
bool Engine::build_graphs() {
  const sgo_opts& o = ctx_[0]->opts;
  cudaGraph_t ga = nullptr, gb = nullptr, body = nullptr;
  const long long l0 = launches_;
  bool ok = cuda_ok(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal), "capture begin");
  if (ok) {
    scf_iteration<T>(o.ncg_first, false);
    k_scf_control<<<1, 256, 0, stream_>>>(L(m_prob_).ka, d_active_, d_flags_, d_iter_, o.max_scf, 0, 0);
    ok = cuda_ok(cudaStreamEndCapture(stream_, &ga), "capture end");
  }
  graph_launches_[0] = launches_ - l0;
  ok = ok && cuda_ok(cudaGraphInstantiate(&g_nonscf_, ga, 0), "graph instantiate");
  cudaGraphConditionalHandle cond = 0;
  cudaGraphNode_t gate = nullptr, loop = nullptr;
  ok = ok && cuda_ok(cudaGraphCreate(&gb, 0), "graph create") &&
       cuda_ok(cudaGraphConditionalHandleCreate(&cond, gb, 0, 0), "conditional handle");
  if (ok) {
    const int* act = d_active_;
    int n = n_;
    const int* itp = d_iter_;
    int mx = o.max_scf;
    void* args[] = {&act, &n, &itp, &mx, &cond};
    cudaKernelNodeParams kp = {};
    kp.func = reinterpret_cast<void*>(k_scf_gate);
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.kernelParams = args;
    ok = cuda_ok(cudaGraphAddKernelNode(&gate, gb, nullptr, 0, &kp), "gate node");
  }
  if (ok) {
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    ok = cuda_ok(cudaGraphAddNode(&loop, gb, &gate, nullptr, 1, &cp), "while node");
    if (ok) body = cp.conditional.phGraph_out[0];
  }
  const long long l1 = launches_;
  ok = ok && cuda_ok(cudaStreamBeginCaptureToGraph(stream_, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal),
                     "capture body begin");
  if (ok) {
    scf_iteration<T>(o.ncg, true);
    k_scf_control<<<1, 256, 0, stream_>>>(L(m_prob_).ka, d_active_, d_flags_, d_iter_, o.max_scf, cond, 1);
    pulay_step();
    cudaGraph_t got = nullptr;
    ok = cuda_ok(cudaStreamEndCapture(stream_, &got), "capture body end");
  }
  graph_launches_[1] = launches_ - l1;
  launches_ = l0;
  ok = ok && cuda_ok(cudaGraphInstantiate(&g_scf_, gb, 0), "graph instantiate (while)");
  if (ga) cudaGraphDestroy(ga);
  if (gb) cudaGraphDestroy(gb);
  if (!ok) {
    cudaGetLastError();
    if (g_nonscf_) cudaGraphExecDestroy(g_nonscf_);
    if (g_scf_) cudaGraphExecDestroy(g_scf_);
    g_nonscf_ = g_scf_ = nullptr;
  }
  return ok;
}

template <typename T>
sgo_status Engine::launch_t(bool want_forces) {
  const sgo_opts& o = ctx_[0]->opts;
  h_active_.assign(n_, 1);
  CK(cudaMemcpyAsync(d_active_, h_active_.data(), sizeof(int) * n_, cudaMemcpyHostToDevice, stream_));
  bool warm = true;
  for (auto* c : ctx_) warm = warm && c->warm && c->have_state;
  for (auto* c : ctx_) c->last_warm = warm;
  k_reset<<<n_, 128, 0, stream_>>>(L(m_prob_).ka);
  sgo_status s = structure_terms();
  if (s != SGO_OK) return s;
  if (!warm) {
    launch_rho0_g(L(m_gew_));
    launch_random_init<T>(L(m_bands_), WB_X, o.seed);
  }
  const int nonsc = warm ? 0 : std::max(0, o.n_nonscf);
  run_nonsc_ = nonsc;
  run_forces_ = want_forces;
  // graph mode: batch engines, no live kernel timer (its events are host bookkeeping)
  run_graph_ = use_graph_ && timer_kind_ < 0;
  if (run_graph_ && !g_scf_) run_graph_ = build_graphs<T>();
  if (run_graph_ && !g_polish_) run_graph_ = build_polish_graphs<T>();
  if (run_graph_) {
    // the iteration counts and the flags are read back by finish(), after the one wait
    CK(cudaMemsetAsync(d_iter_, 0, 2 * sizeof(int), stream_));
    run_na_ = std::min(nonsc, o.max_scf);
    for (int i = 0; i < run_na_; ++i) CK(cudaGraphLaunch(g_nonscf_, stream_));
    if (o.max_scf > nonsc) CK(cudaGraphLaunch(g_scf_, stream_));
    CK(cudaMemcpyAsync(hp_, d_flags_, sizeof(double) * 4 * n_, cudaMemcpyDeviceToHost, stream_));
    k_polish_activate<<<1, 256, 0, stream_>>>(L(m_prob_).ka, d_active_, 0);
    CK(cudaGraphLaunch(g_polish_, stream_));
    CK(cudaGraphLaunch(g_tail_, stream_));
    CK(cudaMemcpyAsync(hpi_, d_iter_, 2 * sizeof(int), cudaMemcpyDeviceToHost, stream_));
  } else {
    int it = 0;
    for (it = 1; it <= o.max_scf; ++it) {
      scf_iteration<T>(it <= nonsc ? o.ncg_first : o.ncg, it > nonsc);
      CK(cudaGetLastError());
      sync_active();
      int nact = 0;
      for (int p = 0; p < n_; ++p) nact += h_active_[p];
      if (nact == 0) break;
      if (it > nonsc) pulay_step();
    }
    run_it_ = it;
    polish<T>();
  }
  // forces on every member
  h_active_.assign(n_, 1);
  CK(cudaMemcpyAsync(d_active_, h_active_.data(), sizeof(int) * n_, cudaMemcpyHostToDevice, stream_));
  if (want_forces) {
    launch_build_projectors<T>(L(m_projs_), 1);
    tn<T>(OPK_DB, 0, OPK_WB, WB_X, DD_DPROJ, false);
    tn<T>(OPK_B, 0, OPK_WB, WB_X, DD_PROJ, false);
    launch_real_to_grid(L(m_gew_), 1, 0);
    grid_fft(0, -1);
    launch_local_forces(L(m_atomch_), maxchunk_);
    launch_force_total(L(m_prob_), maxchunk_);
  }
  // X back to physical buffer 0 so that the next run (warm or component call) finds it there
  k_x_to_buffer0<T><<<m_bands_.total, 256, 0, stream_>>>(L(m_bands_).ka);
  k_reset_roles<<<n_, 32, 0, stream_>>>(L(m_prob_).ka);
  for (int p = 0; p < n_; ++p) {
    const sgo_ctx* c = ctx_[p];
    double* h = hp_ + hp_off_[p];
    CK(cudaMemcpyAsync(h, c->d.scal, sizeof(double) * NSCAL_ALL, cudaMemcpyDeviceToHost, stream_));
    h += NSCAL_ALL;
    CK(cudaMemcpyAsync(h, c->d.eps, sizeof(double) * c->d.nb, cudaMemcpyDeviceToHost, stream_));
    h += c->d.nb;
    CK(cudaMemcpyAsync(h, c->d.occ, sizeof(double) * c->d.nb, cudaMemcpyDeviceToHost, stream_));
    h += c->d.nb;
    CK(cudaMemcpyAsync(h, c->d.forces, sizeof(double) * c->h_forces.size(), cudaMemcpyDeviceToHost, stream_));
    CK(cudaMemcpyAsync(hpi_ + 2 + 4 * p, c->d.status, sizeof(int) * 4, cudaMemcpyDeviceToHost, stream_));
  }
  CK(cudaGetLastError());
  return SGO_OK;
}

sgo_status Engine::enter() {
  run_status_ = ok_ ? SGO_OK : SGO_ERR_CUDA;
  user_stream_ = run_stream_ = stream_;
  if (!ok_ || !use_graph_ || timer_kind_ >= 0) return run_status_;
  // graph mode runs on a private stream (the caller's may be the legacy default stream,
  // which cannot be captured), ordered after the caller's stream and before anything the
  // caller enqueues after leave()
  if (!own_stream_) {
    if (!cuda_ok(cudaStreamCreateWithFlags(&own_stream_, cudaStreamNonBlocking), "graph stream") ||
        !cuda_ok(cudaEventCreateWithFlags(&ev_in_, cudaEventDisableTiming), "graph event") ||
        !cuda_ok(cudaEventCreateWithFlags(&ev_out_, cudaEventDisableTiming), "graph event"))
      return run_status_ = SGO_ERR_CUDA;
  }
  if (!cuda_ok(cudaEventRecord(ev_in_, user_stream_), "graph event") ||
      !cuda_ok(cudaStreamWaitEvent(own_stream_, ev_in_, 0), "graph event"))
    return run_status_ = SGO_ERR_CUDA;
  stream_ = run_stream_ = own_stream_;
  return SGO_OK;
}

sgo_status Engine::launch(bool want_forces, const DeviceIO* io) {
  if (run_status_ != SGO_OK) return run_status_;
  if (io && io->pos) k_scatter_pos<<<n_, 128, 0, stream_>>>(L(m_prob_).ka, d_foff_, io->pos);
  run_status_ = precision_ ? launch_t<float>(want_forces) : launch_t<double>(want_forces);
  if (run_status_ == SGO_OK && io)
    k_gather_results<<<n_, 128, 0, stream_>>>(L(m_prob_).ka, d_slot_, d_foff_, io->energies, io->forces,
                                               io->status);
  return run_status_;
}

void Engine::leave() {
  if (run_stream_ != user_stream_) {
    cudaEventRecord(ev_out_, run_stream_);
    cudaStreamWaitEvent(user_stream_, ev_out_, 0);
  }
  stream_ = user_stream_;
}

sgo_status Engine::finish(std::vector<sgo_status>* per_item) {
  CK(cudaStreamSynchronize(run_stream_));  // (a null stream is the caller's legacy default stream)
  if (run_status_ != SGO_OK) return run_status_;
  CK(cudaGetLastError());
  const sgo_opts& o = ctx_[0]->opts;
  int it = run_it_;
  if (run_graph_) {
    it = hpi_[0];
    launches_ += (long long)run_na_ * graph_launches_[0] + (long long)std::max(0, it - run_na_) * graph_launches_[1] +
                 1 + (long long)hpi_[1] * graph_launches_[2] + graph_launches_[3];
  }
  const int niter = std::min(it, o.max_scf);
  sgo_status all = SGO_OK;
  for (int p = 0; p < n_; ++p) {
    sgo_ctx* c = ctx_[p];
    const double* h = hp_ + hp_off_[p];
    std::memcpy(c->h_scal.data(), h, sizeof(double) * NSCAL_ALL);
    h += NSCAL_ALL;
    std::memcpy(c->h_eps.data(), h, sizeof(double) * c->d.nb);
    h += c->d.nb;
    std::memcpy(c->h_occ.data(), h, sizeof(double) * c->d.nb);
    h += c->d.nb;
    std::memcpy(c->h_forces.data(), h, sizeof(double) * c->h_forces.size());
    std::memcpy(c->h_status, hpi_ + 2 + 4 * p, sizeof(int) * 4);
    c->have_state = true;
    c->last_iter = (int)c->h_scal[SC_ITER] + run_nonsc_;  // this member's iterations (until it converged)
    if (c->last_iter > niter) c->last_iter = niter;
    c->last_resid = c->h_scal[SC_RESID];
    sgo_status st = SGO_OK;
    if (hp_[4 * p + 1] != 0.0) st = SGO_ERR_NOT_CONVERGED;
    if (c->h_status[2] != 0) st = SGO_ERR_TIMEOUT;
    else if (hp_[4 * p + 2] != 0.0 || !std::isfinite(c->h_scal[SC_FREE])) st = SGO_ERR_NAN;
    else if (c->h_scal[SC_CONV] == 0.0) st = SGO_ERR_NOT_CONVERGED;
    if (run_forces_)
      for (double f : c->h_forces)
        if (!std::isfinite(f)) st = SGO_ERR_NAN;
    c->last_status = st;
    if (per_item) (*per_item)[p] = st;
    if (st != SGO_OK && all == SGO_OK) all = st;
  }
  return all;
}

sgo_status Engine::run(bool want_forces, std::vector<sgo_status>* per_item) {
  enter();
  launch(want_forces, nullptr);
  leave();
  return finish(per_item);
}

bool Engine::set_slots(const std::vector<int>& slot, const std::vector<int>& foff) {
  if ((int)slot.size() != n_ || (int)foff.size() != n_ || !d_slot_) return false;
  std::vector<int> h(slot);
  h.insert(h.end(), foff.begin(), foff.end());
  return cuda_ok(cudaMemcpy(d_slot_, h.data(), sizeof(int) * 2 * n_, cudaMemcpyHostToDevice), "slots");
}

// ---- component entry points (problem 0) ----
sgo_status Engine::apply_h(const double* veff_c, int nvec, const double* psi, double* hpsi_out) {
  sgo_ctx* c = ctx_[0];
  const Prob& d = c->d;
  double *dv = nullptr, *dpsi = nullptr, *dout = nullptr;
  CK(dev_malloc(&dv, sizeof(double) * d.ngrid));
  CK(dev_malloc(&dpsi, sizeof(double) * (size_t)nvec * d.npw));
  CK(dev_malloc(&dout, sizeof(double) * (size_t)nvec * d.npw));
  CK(cudaMemcpyAsync(dv, veff_c, sizeof(double) * d.ngrid, cudaMemcpyHostToDevice, stream_));
  CK(cudaMemcpyAsync(dpsi, psi, sizeof(double) * (size_t)nvec * d.npw, cudaMemcpyHostToDevice, stream_));
  h_active_.assign(n_, 1);
  CK(cudaMemcpyAsync(d_active_, h_active_.data(), sizeof(int) * n_, cudaMemcpyHostToDevice, stream_));
  if (structure_terms() != SGO_OK) return SGO_ERR_CUDA;
  if (precision_) {
    launch_veff<float>(L(m_gew_), dv);
    launch_copy_in<float>(L(m_bands_), WB_W, dpsi, nvec);
    hpsi<float>(WB_W, WB_W2);
    launch_copy_out<float>(L(m_bands_), WB_W2, dout, nvec);
  } else {
    launch_veff<double>(L(m_gew_), dv);
    launch_copy_in<double>(L(m_bands_), WB_W, dpsi, nvec);
    hpsi<double>(WB_W, WB_W2);
    launch_copy_out<double>(L(m_bands_), WB_W2, dout, nvec);
  }
  CK(cudaMemcpyAsync(hpsi_out, dout, sizeof(double) * (size_t)nvec * d.npw, cudaMemcpyDeviceToHost, stream_));
  CK(cudaStreamSynchronize(stream_));
  CK(cudaGetLastError());
  dev_free(dv);
  dev_free(dpsi);
  dev_free(dout);
  return SGO_OK;
}

sgo_status Engine::density(int nvec, const double* psi, const double* occ, double* rho) {
  sgo_ctx* c = ctx_[0];
  const Prob& d = c->d;
  double *dpsi = nullptr, *docc = nullptr, *dr = nullptr;
  CK(dev_malloc(&dpsi, sizeof(double) * (size_t)nvec * d.npw));
  CK(dev_malloc(&docc, sizeof(double) * d.nb));
  CK(dev_malloc(&dr, sizeof(double) * d.ngrid));
  std::vector<double> o(d.nb, 0.0);
  for (int i = 0; i < nvec; ++i) o[i] = occ[i];
  CK(cudaMemcpyAsync(dpsi, psi, sizeof(double) * (size_t)nvec * d.npw, cudaMemcpyHostToDevice, stream_));
  CK(cudaMemcpyAsync(docc, o.data(), sizeof(double) * d.nb, cudaMemcpyHostToDevice, stream_));
  h_active_.assign(n_, 1);
  CK(cudaMemcpyAsync(d_active_, h_active_.data(), sizeof(int) * n_, cudaMemcpyHostToDevice, stream_));
  if (precision_) {
    launch_copy_in<float>(L(m_bands_), WB_W, dpsi, nvec);
    wave_to_cols<float>(WB_W);
    launch_plane_density<float>(L(m_dens_), docc);
    for (int k = 0; k < 2; ++k) launch_plane_density_reg(L(m_dreg_[k]), k, dreg_smem_[k], docc);
    launch_plane_density_pair(L(m_dpair_), dpair_smem_, docc);
    launch_big_y<float>(L(m_bigdy_), 1, 1, docc);
    launch_big_density<float>(L(m_bigd_), docc);
  } else {
    launch_copy_in<double>(L(m_bands_), WB_W, dpsi, nvec);
    wave_to_cols<double>(WB_W);
    launch_plane_density<double>(L(m_dens_), docc);
    launch_big_y<double>(L(m_bigdy_), 1, 1, docc);
    launch_big_density<double>(L(m_bigd_), docc);
  }
  launch_export_grid(L(m_gew_), 1, dr);
  CK(cudaMemcpyAsync(rho, dr, sizeof(double) * d.ngrid, cudaMemcpyDeviceToHost, stream_));
  CK(cudaStreamSynchronize(stream_));
  CK(cudaGetLastError());
  dev_free(dpsi);
  dev_free(docc);
  dev_free(dr);
  return SGO_OK;
}

sgo_status Engine::subspace(int nvec, const double* x, const double* y, double* c_out) {
  sgo_ctx* c = ctx_[0];
  const Prob& d = c->d;
  double *dx = nullptr, *dy = nullptr;
  CK(dev_malloc(&dx, sizeof(double) * (size_t)nvec * d.npw));
  CK(dev_malloc(&dy, sizeof(double) * (size_t)nvec * d.npw));
  CK(cudaMemcpyAsync(dx, x, sizeof(double) * (size_t)nvec * d.npw, cudaMemcpyHostToDevice, stream_));
  CK(cudaMemcpyAsync(dy, y, sizeof(double) * (size_t)nvec * d.npw, cudaMemcpyHostToDevice, stream_));
  h_active_.assign(n_, 1);
  CK(cudaMemcpyAsync(d_active_, h_active_.data(), sizeof(int) * n_, cudaMemcpyHostToDevice, stream_));
  if (precision_) {
    launch_copy_in<float>(L(m_bands_), WB_W, dx, nvec);
    launch_copy_in<float>(L(m_bands_), WB_W2, dy, nvec);
    tn<float>(OPK_WB, WB_W, OPK_WB, WB_W2, DD_S);
  } else {
    launch_copy_in<double>(L(m_bands_), WB_W, dx, nvec);
    launch_copy_in<double>(L(m_bands_), WB_W2, dy, nvec);
    tn<double>(OPK_WB, WB_W, OPK_WB, WB_W2, DD_S);
  }
  std::vector<double> s((size_t)d.nb * d.nb);
  CK(cudaMemcpyAsync(s.data(), d.S, sizeof(double) * s.size(), cudaMemcpyDeviceToHost, stream_));
  CK(cudaStreamSynchronize(stream_));
  CK(cudaGetLastError());
  for (int i = 0; i < nvec; ++i)
    for (int j = 0; j < nvec; ++j) c_out[(size_t)i * nvec + j] = s[(size_t)i * d.nb + j];
  dev_free(dx);
  dev_free(dy);
  return SGO_OK;
}

sgo_status Engine::block_update(int nvec, const double* x, const double* m, double alpha, double beta, double* y) {
  sgo_ctx* c = ctx_[0];
  const Prob& d = c->d;
  const size_t nbytes = sizeof(double) * (size_t)nvec * d.npw;
  double *dx = nullptr, *dy = nullptr;
  CK(dev_malloc(&dx, nbytes));
  CK(dev_malloc(&dy, nbytes));
  std::vector<double> tm((size_t)d.nb * d.nb, 0.0);
  for (int i = 0; i < nvec; ++i)
    for (int j = 0; j < nvec; ++j) tm[(size_t)i * d.nb + j] = m[(size_t)i * nvec + j];
  CK(cudaMemcpyAsync(dx, x, nbytes, cudaMemcpyHostToDevice, stream_));
  CK(cudaMemcpyAsync(dy, y, nbytes, cudaMemcpyHostToDevice, stream_));
  CK(cudaMemcpyAsync(d.Tm, tm.data(), sizeof(double) * tm.size(), cudaMemcpyHostToDevice, stream_));
  h_active_.assign(n_, 1);
  CK(cudaMemcpyAsync(d_active_, h_active_.data(), sizeof(int) * n_, cudaMemcpyHostToDevice, stream_));
  if (precision_) {
    launch_copy_in<float>(L(m_bands_), WB_W, dx, nvec);
    launch_copy_in<float>(L(m_bands_), WB_W2, dy, nvec);
    nn<float>(OPK_WB, WB_W, DD_TM, WB_W2, alpha, beta);
    launch_copy_out<float>(L(m_bands_), WB_W2, dy, nvec);
  } else {
    launch_copy_in<double>(L(m_bands_), WB_W, dx, nvec);
    launch_copy_in<double>(L(m_bands_), WB_W2, dy, nvec);
    nn<double>(OPK_WB, WB_W, DD_TM, WB_W2, alpha, beta);
    launch_copy_out<double>(L(m_bands_), WB_W2, dy, nvec);
  }
  CK(cudaMemcpyAsync(y, dy, nbytes, cudaMemcpyDeviceToHost, stream_));
  CK(cudaStreamSynchronize(stream_));
  CK(cudaGetLastError());
  dev_free(dx);
  dev_free(dy);
  return SGO_OK;
}

sgo_status Engine::export_density(double* rho) {
  const Prob& d = ctx_[0]->d;
  double* dr = nullptr;
  CK(dev_malloc(&dr, sizeof(double) * d.ngrid));
  h_active_.assign(n_, 1);
  CK(cudaMemcpyAsync(d_active_, h_active_.data(), sizeof(int) * n_, cudaMemcpyHostToDevice, stream_));
  launch_export_grid(L(m_gew_), 1, dr);
  CK(cudaMemcpyAsync(rho, dr, sizeof(double) * d.ngrid, cudaMemcpyDeviceToHost, stream_));
  CK(cudaStreamSynchronize(stream_));
  dev_free(dr);
  return SGO_OK;
}

sgo_status Engine::export_state(double* rho_g, double* psi) {
  const Prob& d = ctx_[0]->d;
  const size_t gbytes = sizeof(double2) * (size_t)d.ngrid, pbytes = sizeof(double) * (size_t)d.nbo * d.npw;
  h_active_.assign(n_, 1);
  CK(cudaMemcpyAsync(d_active_, h_active_.data(), sizeof(int) * n_, cudaMemcpyHostToDevice, stream_));
  char* dbuf = nullptr;
  CK(dev_malloc(&dbuf, gbytes + pbytes));
  double2* dg = reinterpret_cast<double2*>(dbuf);
  double* dp = reinterpret_cast<double*>(dbuf + gbytes);
  if (rho_g) {
    CK(cudaMemcpyAsync(d.gfft, d.rhog_in, gbytes, cudaMemcpyDeviceToDevice, stream_));
    launch_grid_copy_c(L(m_gew_), nullptr, dg);
    CK(cudaMemcpyAsync(rho_g, dg, gbytes, cudaMemcpyDeviceToHost, stream_));
  }
  if (psi) {
    if (precision_) launch_copy_out<float>(L(m_bands_), WB_X, dp, d.nbo);
    else launch_copy_out<double>(L(m_bands_), WB_X, dp, d.nbo);
    CK(cudaMemcpyAsync(psi, dp, pbytes, cudaMemcpyDeviceToHost, stream_));
  }
  CK(cudaStreamSynchronize(stream_));
  dev_free(dbuf);
  return cuda_ok(cudaGetLastError(), "export state") ? SGO_OK : SGO_ERR_CUDA;
}

sgo_status Engine::import_state(const double* rho_g, const double* psi) {
  const Prob& d = ctx_[0]->d;
  const size_t gbytes = sizeof(double2) * (size_t)d.ngrid, pbytes = sizeof(double) * (size_t)d.nbo * d.npw;
  h_active_.assign(n_, 1);
  CK(cudaMemcpyAsync(d_active_, h_active_.data(), sizeof(int) * n_, cudaMemcpyHostToDevice, stream_));
  char* dbuf = nullptr;
  CK(dev_malloc(&dbuf, gbytes + pbytes));
  double2* dg = reinterpret_cast<double2*>(dbuf);
  double* dp = reinterpret_cast<double*>(dbuf + gbytes);
  CK(cudaMemcpyAsync(dg, rho_g, gbytes, cudaMemcpyHostToDevice, stream_));
  CK(cudaMemcpyAsync(dp, psi, pbytes, cudaMemcpyHostToDevice, stream_));
  launch_grid_copy_c(L(m_gew_), dg, nullptr);
  CK(cudaMemcpyAsync(d.rhog_in, d.gfft, gbytes, cudaMemcpyDeviceToDevice, stream_));
  // the requested bands from the caller; the headroom bands above them start random
  const unsigned long long seed = ctx_[0]->opts.seed;
  if (precision_) {
    launch_random_init<float>(L(m_bands_), WB_X, seed);
    launch_copy_in<float>(L(m_bands_), WB_X, dp, d.nbo, true);
  } else {
    launch_random_init<double>(L(m_bands_), WB_X, seed);
    launch_copy_in<double>(L(m_bands_), WB_X, dp, d.nbo, true);
  }
  CK(cudaStreamSynchronize(stream_));
  dev_free(dbuf);
  return cuda_ok(cudaGetLastError(), "import state") ? SGO_OK : SGO_ERR_CUDA;
}

sgo_status Engine::grid_transform(int sign, const double* in, double* out) {
  const Prob& d = ctx_[0]->d;
  const size_t bytes = sizeof(double2) * (size_t)d.ngrid;
  double2* dg = nullptr;
  CK(dev_malloc(&dg, bytes));
  h_active_.assign(n_, 1);
  CK(cudaMemcpyAsync(d_active_, h_active_.data(), sizeof(int) * n_, cudaMemcpyHostToDevice, stream_));
  CK(cudaMemcpyAsync(dg, in, bytes, cudaMemcpyHostToDevice, stream_));
  launch_grid_copy_c(L(m_gew_), dg, nullptr);
  grid_fft(0, sign);
  launch_grid_copy_c(L(m_gew_), nullptr, dg);
  CK(cudaMemcpyAsync(out, dg, bytes, cudaMemcpyDeviceToHost, stream_));
  CK(cudaStreamSynchronize(stream_));
  dev_free(dg);
  return cuda_ok(cudaGetLastError(), "grid transform") ? SGO_OK : SGO_ERR_CUDA;
}

sgo_status Engine::run_device(const double* pos, double* energies, double* forces, int* status) {
  const DeviceIO io{pos, energies, forces, status};
  enter();
  launch(true, &io);
  leave();
  const sgo_status s = finish(nullptr);
  return s == SGO_ERR_CUDA ? s : SGO_OK;
}

}  // namespace sgo
