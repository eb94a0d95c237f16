// Grid-level kernels of one SCF step (Sec. II D: rho_in -> V_eff; rho_out -> energy;
// rho_out mixed with rho_in), the structure-dependent terms (local ionic potential,
// projectors, initial density) and the Hellmann-Feynman forces.
//
// Fields on the FFT box follow f(G) = (1/N) sum_r f(r) exp(-iG.r); the unnormalised
// forward transform leaves N f(G) in the complex work grid.  Nyquist planes (m_i =
// -N_i/2 for even N_i) are zeroed in every field defined by a formula in G.
#include "kernels.h"

namespace sgo {

namespace {

struct GPt {
  int m1, m2, m3;
  bool nyq;
};

__device__ __forceinline__ int wrapm(int i, int n, bool* nyq) {
  if ((n & 1) == 0 && i == n / 2) *nyq = true;
  return i < (n + 1) / 2 ? i : i - n;
}

// box point of plane-major index idx = (i3*N1 + i1)*N2 + i2
__device__ __forceinline__ GPt grid_pt(const Prob& P, int idx, int* i1o = nullptr, int* i2o = nullptr,
                                       int* i3o = nullptr) {
  GPt g;
  g.nyq = false;
  int i2 = idx % P.n2;
  int t = idx / P.n2;
  int i1 = t % P.n1;
  int i3 = t / P.n1;
  g.m1 = wrapm(i1, P.n1, &g.nyq);
  g.m2 = wrapm(i2, P.n2, &g.nyq);
  g.m3 = wrapm(i3, P.n3, &g.nyq);
  if (i1o) *i1o = i1;
  if (i2o) *i2o = i2;
  if (i3o) *i3o = i3;
  return g;
}

__device__ __forceinline__ void gcart(const Prob& P, int m1, int m2, int m3, double* G) {
  for (int d = 0; d < 3; ++d) G[d] = m1 * P.bvec[d] + m2 * P.bvec[3 + d] + m3 * P.bvec[6 + d];
}

__device__ __forceinline__ double* grid_sel(const Prob& P, int sel) {
  switch (sel) {
    case 0: return P.rho_in;
    case 1: return P.rho_out;
    case 2: return P.resid;
    default: return P.vion_r;
  }
}

// exp(-i G.R_I) from the atom's 1D tables (indexed by grid index per axis).
__device__ __forceinline__ cplx<double> phase_at(const Prob& P, int atom, int i1, int i2, int i3) {
  const cplx<double>* ph = reinterpret_cast<const cplx<double>*>(P.phase) + (size_t)atom * (P.n1 + P.n2 + P.n3);
  return ph[i1] * ph[P.n1 + i2] * ph[P.n1 + P.n2 + i3];
}

__device__ __forceinline__ float cbrt_t(float x) { return cbrtf(x); }
__device__ __forceinline__ double cbrt_t(double x) { return cbrt(x); }
__device__ __forceinline__ float sqrt_t(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_t(double x) { return sqrt(x); }
__device__ __forceinline__ float log_t(float x) { return logf(x); }
__device__ __forceinline__ double log_t(double x) { return log(x); }

// Perdew-Zunger 1981 correlation + Slater exchange (unpolarised); rho clipped at 0.
// R = double on the FP64 path.  R = float on the mixed path: v_xc enters the FP32 V_eff
// there anyway, and eps_xc (relative error ~1e-7 per point) is summed in FP64.  One cube
// root per point: (3 rho/pi)^(1/3) = (3/pi)^(1/3) rho^(1/3), r_s = (3/(4 pi))^(1/3) / rho^(1/3).
template <typename R>
__device__ __forceinline__ void lda_pz81(R rho, R* exc, R* vxc) {
  if (!(rho > R(1e-30))) {
    *exc = R(0);
    *vxc = R(0);
    return;
  }
  const R c = cbrt_t(rho);
  const R ex = R(-0.75 * 0.98474502184269641) * c;  // (3/pi)^(1/3)
  const R rs = R(0.62035049089940009) / c;          // (3/(4 pi))^(1/3)
  R ec, vc;
  if (rs >= R(1)) {
    const R g = R(-0.1423), b1 = R(1.0529), b2 = R(0.3334);
    const R sr = sqrt_t(rs);
    const R den = R(1) + b1 * sr + b2 * rs;
    ec = g / den;
    vc = ec * (R(1) + R(7.0 / 6.0) * b1 * sr + R(4.0 / 3.0) * b2 * rs) / den;
  } else {
    const R A = R(0.0311), B = R(-0.048), C = R(0.0020), D = R(-0.0116);
    const R lr = log_t(rs);
    ec = A * lr + B + C * rs * lr + D * rs;
    vc = A * lr + (B - A / R(3)) + R(2.0 / 3.0) * C * rs * lr + (R(2) * D - C) / R(3) * rs;
  }
  *exc = ex + ec;
  *vxc = R(4.0 / 3.0) * ex + vc;
}

}  // namespace

// ---------------------------------------------------------------------------
// elementwise grid kernels: CTA = (problem, chunk of GRID_EW points)
// ---------------------------------------------------------------------------
constexpr int GRID_EW = GRID_EW_POINTS;

#define GRID_EW_PROLOGUE                                           \
  const int p = locate(ka.start, ka.nprob, blockIdx.x);            \
  if (!ka.active[p]) return;                                       \
  const Prob& P = ka.probs[p];                                     \
  const int base = (blockIdx.x - ka.start[p]) * GRID_EW;           \
  const int end = min(P.ngrid, base + GRID_EW);

__global__ void k_real_to_grid(KArgs ka, int src, int which) {
  GRID_EW_PROLOGUE
  const double* s = grid_sel(P, src);
  double2* g = which ? P.gfft2 : P.gfft;
  for (int i = base + threadIdx.x; i < end; i += blockDim.x) g[i] = make_double2(s[i], 0.0);
}

__global__ void k_grid_real_part(KArgs ka, int which, int dst) {
  GRID_EW_PROLOGUE
  const double2* g = which ? P.gfft2 : P.gfft;
  double* d = grid_sel(P, dst);
  for (int i = base + threadIdx.x; i < end; i += blockDim.x) d[i] = g[i].x;
}

// V_H(G) = 4 pi rho(G) / |G|^2 (G != 0), from N rho(G) in the work grid.
__global__ void k_hartree_g(KArgs ka, int which) {
  GRID_EW_PROLOGUE
  double2* g = which ? P.gfft2 : P.gfft;
  const double inv_n = 1.0 / P.ngrid;
  for (int i = base + threadIdx.x; i < end; i += blockDim.x) {
    GPt q = grid_pt(P, i);
    double G[3];
    gcart(P, q.m1, q.m2, q.m3, G);
    double g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
    double2 v = g[i];
    double f = (q.nyq || g2 < 1e-14) ? 0.0 : 4.0 * PI * inv_n / g2;
    g[i] = make_double2(v.x * f, v.y * f);
  }
}

// V_eff(r) = V_ion(r) + V_H(r) + v_xc(rho_in(r)), stored divided by N in the wave
// precision for the H.psi plane kernel; the work grid holds rho_in(r) + i V_H(r) (one
// inverse transform of rho_in(G) + i V_H(G), both fields real).  rho_in(r) is kept.
// With user_v: the caller's C-order grid instead.
template <typename T>
__global__ void k_veff(KArgs ka, const double* user_v) {
  GRID_EW_PROLOGUE
  T* v = reinterpret_cast<T*>(P.veff);
  const double inv_n = 1.0 / P.ngrid;
  for (int i = base + threadIdx.x; i < end; i += blockDim.x) {
    double val;
    if (user_v) {
      int i1, i2, i3;
      grid_pt(P, i, &i1, &i2, &i3);
      val = user_v[((size_t)i1 * P.n2 + i2) * P.n3 + i3];
    } else {
      const double2 c = P.gfft[i];
      T exc, vxc;
      lda_pz81<T>((T)c.x, &exc, &vxc);
      P.rho_in[i] = c.x;
      val = P.vion_r[i] + c.y + (double)vxc;
    }
    v[i] = (T)(val * inv_n);
  }
}

// Work grid := rho_in(G) + i V_H(G), V_H(G) = 4 pi rho_in(G) / |G|^2 (0 at G = 0), in the
// precision of the transform that follows (T = float: the grid's single-precision view).
template <typename T>
__global__ void k_potential_g(KArgs ka) {
  GRID_EW_PROLOGUE
  cplx<T>* g = reinterpret_cast<cplx<T>*>(P.gfft);
  for (int i = base + threadIdx.x; i < end; i += blockDim.x) {
    const double g2 = P.g2box[i];  // -1 on Nyquist planes
    double2 r = P.rhog_in[i];
    double f = g2 < 1e-14 ? 0.0 : 4.0 * PI / g2;
    // (r.x + i r.y) + i f (r.x + i r.y)
    g[i] = mk((T)(r.x - f * r.y), (T)(r.y + f * r.x));
  }
}

// V_ion(G) = sum_I v_s(G) exp(-iG.R_I) (work grid gfft).
__global__ void k_vion_g(KArgs ka) {
  GRID_EW_PROLOGUE
  for (int i = base + threadIdx.x; i < end; i += blockDim.x) {
    int i1, i2, i3;
    grid_pt(P, i, &i1, &i2, &i3);
    cplx<double> acc = mk(0.0, 0.0);
    double v[MAX_SPECIES];
    for (int s = 0; s < P.nspecies; ++s) v[s] = P.vloc_g[(size_t)s * P.ngrid + i];
    for (int a = 0; a < P.natom; ++a) acc = acc + scale(phase_at(P, a, i1, i2, i3), v[P.spec[a]]);
    P.gfft[i] = make_double2(acc.x, acc.y);
  }
}

// Initial density: neutral atomic Gaussians (Z/Omega) exp(-G^2 rc^2/4) exp(-iG.R_I),
// band-limited to |G|^2/2 <= 4 Ecut, written as rho_in(G).
__global__ void k_rho0_g(KArgs ka) {
  GRID_EW_PROLOGUE
  for (int i = base + threadIdx.x; i < end; i += blockDim.x) {
    int i1, i2, i3;
    grid_pt(P, i, &i1, &i2, &i3);
    const double g2 = P.g2box[i];  // -1 on Nyquist planes
    cplx<double> acc = mk(0.0, 0.0);
    if (g2 >= 0.0 && 0.5 * g2 <= 4.0 * P.ecut) {
      double amp[MAX_SPECIES];
      for (int s = 0; s < P.nspecies; ++s) {
        const double* sp = P.sp + s * 6;
        amp[s] = sp[0] / P.omega * exp(-g2 * sp[1] * sp[1] * 0.25);
      }
      for (int a = 0; a < P.natom; ++a) acc = acc + scale(phase_at(P, a, i1, i2, i3), amp[P.spec[a]]);
    }
    P.rhog_in[i] = make_double2(acc.x, acc.y);
  }
}

// ---------------------------------------------------------------------------
// Grid reductions for the energy at rho_out (work grid gfft2 = N rho_out(G)):
// part[p][chunk][0..4] = sum V_ion rho, sum rho eps_xc, sum rho, sum |rho_out - rho_in|,
// sum_{G!=0} |rho(G)|^2 / G^2.
// ---------------------------------------------------------------------------
constexpr int NGE = 5;

template <typename T>
__global__ void k_grid_energies(KArgs ka, double* part, int maxchunk) {
  __shared__ double red[33];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int chunk = blockIdx.x - ka.start[p];
  const int base = chunk * GRID_CHUNK, end = min(P.ngrid, base + GRID_CHUNK);
  const double inv_n = 1.0 / P.ngrid;
  double s[NGE] = {0, 0, 0, 0, 0};
  for (int i = base + threadIdx.x; i < end; i += blockDim.x) {
    double r = P.rho_out[i];
    T exc, vxc;
    lda_pz81<T>((T)r, &exc, &vxc);
    s[0] += P.vion_r[i] * r;
    s[1] += fmax(r, 0.0) * (double)exc;
    s[2] += r;
    s[3] += fabs(r - P.rho_in[i]);
    const double g2 = P.g2box[i];  // -1 on Nyquist planes
    if (g2 > 1e-14) {
      double2 v = P.gfft2[i];
      s[4] += (v.x * v.x + v.y * v.y) * inv_n * inv_n / g2;
    }
  }
  for (int k = 0; k < NGE; ++k) {
    double t = block_sum(s[k], red);
    if (threadIdx.x == 0) part[((size_t)p * maxchunk + chunk) * NGE + k] = t;
  }
}

__global__ void k_grid_energies_reduce(KArgs ka, const double* part, int maxchunk) {
  const int p = blockIdx.x;
  if (!ka.active[p] || threadIdx.x != 0) return;
  const Prob& P = ka.probs[p];
  const int nch = (P.ngrid + GRID_CHUNK - 1) / GRID_CHUNK;
  double s[NGE] = {0, 0, 0, 0, 0};
  for (int c = 0; c < nch; ++c)
    for (int k = 0; k < NGE; ++k) s[k] += part[((size_t)p * maxchunk + c) * NGE + k];
  const double dv = P.omega / P.ngrid;
  P.scal[SC_ELOC] = dv * s[0];
  P.scal[SC_EXC] = dv * s[1];
  P.scal[SC_NELCHK] = dv * s[2];
  P.scal[SC_RESID] = dv * s[3] / P.nel;
  P.scal[SC_EH] = 0.5 * P.omega * 4.0 * PI * s[4];
}

// Band terms, total free energy, convergence test.  One CTA per problem.
__global__ void k_finish_iteration(KArgs ka, double tol_e, double tol_rho, int count_iter) {
  __shared__ double red[33];
  const int p = blockIdx.x;
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  double ek = 0.0, en = 0.0;
  for (int i = threadIdx.x; i < P.nb; i += blockDim.x) {
    const double f = P.occ[i];
    ek += f * P.bv[BV_EKIN * P.nb + i];
    double s = 0.0;
    for (int a = 0; a < P.natom; ++a) {
      double pr = P.proj[(size_t)a * P.nb + i];
      s += P.sp[P.spec[a] * 6 + 5] * pr * pr;
    }
    en += f * s;
  }
  ek = block_sum(ek, red);
  en = block_sum(en, red);
  if (threadIdx.x == 0) {
    double* sc = P.scal;
    sc[SC_EKIN] = ek;
    sc[SC_ENL] = en;
    sc[SC_MTS] = -P.kT * sc[SC_ENTROPY];
    double F = ek + en + sc[SC_ELOC] + sc[SC_EH] + sc[SC_EXC] + sc[SC_EEW] + sc[SC_MTS];
    sc[SC_FREE] = F;
    if (!isfinite(F)) P.status[1] = 1;
    // count_iter 2: the energy of the bands refined after the stopping rule held (the
    // convergence state and the iteration count stay)
    if (count_iter == 2) return;
    const int it = (int)sc[SC_ITER];
    sc[SC_DF] = it > 0 ? F - sc[SC_FPREV] : 1e300;
    bool conv = count_iter && it > 0 && fabs(sc[SC_DF]) < tol_e && sc[SC_RESID] < tol_rho;
    sc[SC_FPREV] = F;
    if (count_iter) sc[SC_ITER] = it + 1;
    sc[SC_CONV] = conv ? 1.0 : 0.0;
  }
}

// ---------------------------------------------------------------------------
// Pulay (DIIS) mixing on R = rho_out - rho_in with a ring history.
// ---------------------------------------------------------------------------
__global__ void k_pulay_store(KArgs ka) {
  GRID_EW_PROLOGUE
  const int pos = (int)P.scal[SC_PULAY_POS];
  double2* hr = P.hrho + (size_t)pos * P.ngrid;
  double2* hs = P.hres + (size_t)pos * P.ngrid;
  const double inv_n = 1.0 / P.ngrid;
  for (int i = base + threadIdx.x; i < end; i += blockDim.x) {
    double2 ri = P.rhog_in[i], ro = P.gfft2[i];
    hr[i] = ri;
    hs[i] = make_double2(ro.x * inv_n - ri.x, ro.y * inv_n - ri.y);
  }
}

// part[p][chunk][j] = <R_pos, R_j> over a chunk, for every ring slot j.
__global__ void k_pulay_gram(KArgs ka, double* part, int maxchunk, int hist) {
  __shared__ double red[33];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int chunk = blockIdx.x - ka.start[p];
  const int base = chunk * GRID_CHUNK, end = min(P.ngrid, base + GRID_CHUNK);
  const int pos = (int)P.scal[SC_PULAY_POS];
  const int cnt = min((int)P.scal[SC_PULAY_N] + 1, hist);
  const double2* rp = P.hres + (size_t)pos * P.ngrid;
  for (int j = 0; j < cnt; ++j) {
    const double2* rj = P.hres + (size_t)j * P.ngrid;
    double s = 0.0;
    for (int i = base + threadIdx.x; i < end; i += blockDim.x) s += rp[i].x * rj[i].x + rp[i].y * rj[i].y;
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[((size_t)p * maxchunk + chunk) * MAX_HIST + j] = s;
  }
}

// Gram row update and the DIIS system [A 1; 1 0][c; l] = [0; 1] (partial pivoting).
__global__ void k_pulay_solve(KArgs ka, const double* part, int maxchunk, int hist) {
  const int p = blockIdx.x;
  if (!ka.active[p] || threadIdx.x != 0) return;
  const Prob& P = ka.probs[p];
  double* sc = P.scal;
  double* A = sc + SC_PULAY_A;
  double* alpha = sc + SC_PULAY_A + MAX_HIST * MAX_HIST;
  const int pos = (int)sc[SC_PULAY_POS];
  const int cnt = min((int)sc[SC_PULAY_N] + 1, hist);
  const int nch = (P.ngrid + GRID_CHUNK - 1) / GRID_CHUNK;
  for (int j = 0; j < cnt; ++j) {
    double s = 0.0;
    for (int c = 0; c < nch; ++c) s += part[((size_t)p * maxchunk + c) * MAX_HIST + j];
    A[pos * MAX_HIST + j] = s;
    A[j * MAX_HIST + pos] = s;
  }
  const int m = cnt + 1;
  double M[(MAX_HIST + 1) * (MAX_HIST + 2)];
  const double scl = A[pos * MAX_HIST + pos] > 0.0 ? 1.0 / A[pos * MAX_HIST + pos] : 1.0;
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < m; ++j) {
      double v;
      if (i < cnt && j < cnt) v = A[i * MAX_HIST + j] * scl;
      else if (i == cnt && j == cnt) v = 0.0;
      else v = 1.0;
      M[i * (m + 1) + j] = v;
    }
    M[i * (m + 1) + m] = (i == cnt) ? 1.0 : 0.0;
  }
  bool ok = true;
  for (int k = 0; k < m && ok; ++k) {
    int piv = k;
    for (int i = k + 1; i < m; ++i)
      if (fabs(M[i * (m + 1) + k]) > fabs(M[piv * (m + 1) + k])) piv = i;
    if (fabs(M[piv * (m + 1) + k]) < 1e-300) { ok = false; break; }
    if (piv != k)
      for (int j = 0; j <= m; ++j) {
        double t = M[k * (m + 1) + j];
        M[k * (m + 1) + j] = M[piv * (m + 1) + j];
        M[piv * (m + 1) + j] = t;
      }
    for (int i = k + 1; i < m; ++i) {
      double f = M[i * (m + 1) + k] / M[k * (m + 1) + k];
      for (int j = k; j <= m; ++j) M[i * (m + 1) + j] -= f * M[k * (m + 1) + j];
    }
  }
  double x[MAX_HIST + 1];
  if (ok) {
    for (int i = m - 1; i >= 0; --i) {
      double s = M[i * (m + 1) + m];
      for (int j = i + 1; j < m; ++j) s -= M[i * (m + 1) + j] * x[j];
      x[i] = s / M[i * (m + 1) + i];
      if (!isfinite(x[i])) ok = false;
    }
  }
  for (int j = 0; j < MAX_HIST; ++j) alpha[j] = 0.0;
  if (ok) {
    for (int j = 0; j < cnt; ++j) alpha[j] = x[j];
  } else {
    alpha[pos] = 1.0;
  }
  sc[SC_PULAY_N] = cnt;
  sc[SC_PULAY_POS] = (pos + 1) % hist;
}

// rho_in(G) = sum_j c_j rho_j(G) + a K(G) sum_j c_j R_j(G), K = G^2/(G^2 + q0^2) (1 if q0 = 0),
// zero on Nyquist planes.
__global__ void k_pulay_mix(KArgs ka, double a, double q0) {
  GRID_EW_PROLOGUE
  const double* alpha = P.scal + SC_PULAY_A + MAX_HIST * MAX_HIST;
  const int cnt = (int)P.scal[SC_PULAY_N];
  for (int i = base + threadIdx.x; i < end; i += blockDim.x) {
    const double g2 = P.g2box[i];  // -1 on Nyquist planes
    double rx = 0.0, ry = 0.0, sx = 0.0, sy = 0.0;
    for (int j = 0; j < cnt; ++j) {
      const double2 h = P.hrho[(size_t)j * P.ngrid + i], r = P.hres[(size_t)j * P.ngrid + i];
      rx += alpha[j] * h.x;
      ry += alpha[j] * h.y;
      sx += alpha[j] * r.x;
      sy += alpha[j] * r.y;
    }
    double k = 1.0;
    if (q0 > 0.0) k = g2 < 1e-14 ? 0.0 : g2 / (g2 + q0 * q0);
    if (g2 < 0.0) k = 0.0, rx = ry = 0.0;
    P.rhog_in[i] = make_double2(rx + a * k * sx, ry + a * k * sy);
  }
}

// ---------------------------------------------------------------------------
// Projectors (packed real form): B[I] = pack(beta_s(G) exp(-iG.R_I)) and, for the
// forces, dB[3I+a] = pack(-i G_a beta_I(G)) = (G_a b_im, -G_a b_re).
// beta_s(G) = Omega^{-1/2} N (2 pi)^{3/2} rp^3 exp(-G^2 rp^2/2), N^2 = 1/(pi^{3/2} rp^3).
// CTA = (problem, atom).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_build_projectors(KArgs ka, int deriv) {
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int a = blockIdx.x - ka.start[p];
  const double* sp = P.sp + P.spec[a] * 6;
  const double rp = sp[4];
  const double nrm = 1.0 / sqrt(pow(PI, 1.5) * rp * rp * rp);
  const double amp = nrm * pow(2.0 * PI, 1.5) * rp * rp * rp / sqrt(P.omega);
  T* b = reinterpret_cast<T*>(P.B) + (size_t)a * P.ld;
  T* d0 = deriv ? reinterpret_cast<T*>(P.dB) + (size_t)(3 * a) * P.ld : nullptr;
  const int* em1 = P.ent_m3 - 2 * P.nhalf;
  const int* em2 = P.ent_m3 - P.nhalf;
  for (int k = threadIdx.x; k <= P.nhalf; k += blockDim.x) {
    if (k == 0) {
      if (!deriv) b[0] = (T)amp;
      else for (int c = 0; c < 3; ++c) d0[(size_t)c * P.ld] = T(0);
      continue;
    }
    const int e = k - 1;
    const double g2 = 2.0 * P.ekin[1 + 2 * e];
    const double bg = amp * exp(-0.5 * g2 * rp * rp);
    const int m1 = em1[e], m2 = em2[e], m3 = P.ent_m3[e];
    const int i1 = m1 < 0 ? m1 + P.n1 : m1, i2 = m2 < 0 ? m2 + P.n2 : m2, i3 = m3 < 0 ? m3 + P.n3 : m3;
    cplx<double> ph = phase_at(P, a, i1, i2, i3);
    const double bre = SQRT2 * bg * ph.x, bim = SQRT2 * bg * ph.y;
    if (!deriv) {
      b[1 + 2 * e] = (T)bre;
      b[2 + 2 * e] = (T)bim;
    } else {
      for (int c = 0; c < 3; ++c) {
        const double gc = P.gvec[(size_t)c * P.ld + 1 + 2 * e];
        d0[(size_t)c * P.ld + 1 + 2 * e] = (T)(gc * bim);
        d0[(size_t)c * P.ld + 2 + 2 * e] = (T)(-gc * bre);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Forces.  Local: dE/dR_Ia = Omega sum_G v_s(G) G_a Im[exp(-iG.R_I) rho(G)^*] over the
// box (work grid gfft = N rho_out(G)).  CTA = (problem, group of LF_AG atoms, chunk):
// the point's G, rho(G) and v_s(G) are fetched once for the group -> partials.
// ---------------------------------------------------------------------------
constexpr int LF_AG = LF_GROUP;

__global__ void k_local_forces(KArgs ka, int maxchunk) {
  __shared__ double red[33];
  (void)maxchunk;
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int nch = (P.ngrid + GRID_CHUNK - 1) / GRID_CHUNK;  // fpart is [natom][nch][3]
  const int local = blockIdx.x - ka.start[p];
  const int g = local / nch, chunk = local - g * nch;
  const int a0 = g * LF_AG, na = min(LF_AG, P.natom - a0);
  const int base = chunk * GRID_CHUNK, end = min(P.ngrid, base + GRID_CHUNK);
  const double inv_n = 1.0 / P.ngrid;
  double f[LF_AG][3];
#pragma unroll
  for (int k = 0; k < LF_AG; ++k) f[k][0] = f[k][1] = f[k][2] = 0.0;
  for (int i = base + threadIdx.x; i < end; i += blockDim.x) {
    int i1, i2, i3;
    GPt q = grid_pt(P, i, &i1, &i2, &i3);
    if (q.nyq) continue;
    double vs[MAX_SPECIES];
    for (int s = 0; s < P.nspecies; ++s) vs[s] = P.vloc_g[(size_t)s * P.ngrid + i];
    const double2 rg = P.gfft[i];
    const cplx<double> rc = mk(rg.x * inv_n, -rg.y * inv_n);
    double G[3];
    gcart(P, q.m1, q.m2, q.m3, G);
#pragma unroll
    for (int k = 0; k < LF_AG; ++k) {
      if (k >= na) break;
      const double v = vs[P.spec[a0 + k]];
      if (v == 0.0) continue;
      const double t = v * (phase_at(P, a0 + k, i1, i2, i3) * rc).y;
      f[k][0] += t * G[0];
      f[k][1] += t * G[1];
      f[k][2] += t * G[2];
    }
  }
#pragma unroll
  for (int k = 0; k < LF_AG; ++k) {
    if (k >= na) break;  // uniform across the block
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double t = block_sum(f[k][c], red);
      if (threadIdx.x == 0) P.fpart[((size_t)(a0 + k) * nch + chunk) * 3 + c] = -P.omega * t;
    }
  }
}

// Total: local partials + nonlocal -2 D sum_n f_n p_nI dp_nIa + Ewald.  CTA per problem.
__global__ void k_force_total(KArgs ka, int maxchunk) {
  (void)maxchunk;
  const int p = blockIdx.x;
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int nch = (P.ngrid + GRID_CHUNK - 1) / GRID_CHUNK;
  for (int e = threadIdx.x; e < 3 * P.natom; e += blockDim.x) {
    const int a = e / 3, c = e % 3;
    double s = 0.0;
    for (int k = 0; k < nch; ++k) s += P.fpart[((size_t)a * nch + k) * 3 + c];
    const double D = P.sp[P.spec[a] * 6 + 5];
    double nl = 0.0;
    for (int n = 0; n < P.nb; ++n)
      nl += P.occ[n] * P.proj[(size_t)a * P.nb + n] * P.dproj[(size_t)(3 * a + c) * P.nb + n];
    P.forces[e] = s - 2.0 * D * nl + P.ewald_f[e];
  }
}

// Copy a grid (sel as in grid_sel) to C order (i1, i2, i3) for the caller.
__global__ void k_export_grid(KArgs ka, int sel, double* out) {
  GRID_EW_PROLOGUE
  const double* s = grid_sel(P, sel);
  for (int i = base + threadIdx.x; i < end; i += blockDim.x) {
    int i1, i2, i3;
    grid_pt(P, i, &i1, &i2, &i3);
    out[((size_t)i1 * P.n2 + i2) * P.n3 + i3] = s[i];
  }
}

// complex grid (C order (N1, N2, N3), interleaved) <-> the transform buffer gfft
__global__ void k_grid_copy_c(KArgs ka, const double2* in, double2* out) {
  GRID_EW_PROLOGUE
  for (int i = base + threadIdx.x; i < end; i += blockDim.x) {
    int i1, i2, i3;
    grid_pt(P, i, &i1, &i2, &i3);
    const size_t e = ((size_t)i1 * P.n2 + i2) * P.n3 + i3;
    if (in) P.gfft[i] = in[e];
    else out[e] = P.gfft[i];
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline int ew_blocks(const Launch& L) { return L.map.total; }
void launch_grid_copy_c(const Launch& L, const double2* in, double2* out) {
  if (ew_blocks(L)) k_grid_copy_c<<<L.map.total, 256, 0, L.stream>>>(L.ka, in, out);
}

void launch_real_to_grid(const Launch& L, int src, int which) {
  if (ew_blocks(L)) k_real_to_grid<<<L.map.total, 256, 0, L.stream>>>(L.ka, src, which);
}
void launch_grid_real_part(const Launch& L, int which, int dst) {
  if (ew_blocks(L)) k_grid_real_part<<<L.map.total, 256, 0, L.stream>>>(L.ka, which, dst);
}
void launch_export_grid(const Launch& L, int sel, double* out) {
  if (ew_blocks(L)) k_export_grid<<<L.map.total, 256, 0, L.stream>>>(L.ka, sel, out);
}
void launch_hartree_g(const Launch& L, int which) {
  if (ew_blocks(L)) k_hartree_g<<<L.map.total, 256, 0, L.stream>>>(L.ka, which);
}
template <typename T>
void launch_veff(const Launch& L, const double* user_v) {
  if (ew_blocks(L)) k_veff<T><<<L.map.total, 256, 0, L.stream>>>(L.ka, user_v);
}
template <typename T>
void launch_potential_g(const Launch& L) {
  if (ew_blocks(L)) k_potential_g<T><<<L.map.total, 256, 0, L.stream>>>(L.ka);
}
template void launch_potential_g<float>(const Launch&);
template void launch_potential_g<double>(const Launch&);
void launch_vion_g(const Launch& L) {
  if (ew_blocks(L)) k_vion_g<<<L.map.total, 256, 0, L.stream>>>(L.ka);
}
void launch_rho0_g(const Launch& L) {
  if (ew_blocks(L)) k_rho0_g<<<L.map.total, 256, 0, L.stream>>>(L.ka);
}
void launch_pulay_store(const Launch& L) {
  if (ew_blocks(L)) k_pulay_store<<<L.map.total, 256, 0, L.stream>>>(L.ka);
}
void launch_pulay_mix(const Launch& L, double a, double q0) {
  if (ew_blocks(L)) k_pulay_mix<<<L.map.total, 256, 0, L.stream>>>(L.ka, a, q0);
}
template <typename T>
void launch_grid_energies(const Launch& Lchunks, double* part, int maxchunk) {
  if (Lchunks.map.total) k_grid_energies<T><<<Lchunks.map.total, 256, 0, Lchunks.stream>>>(Lchunks.ka, part, maxchunk);
}
void launch_grid_energies_reduce(const Launch& L, const double* part, int maxchunk) {
  k_grid_energies_reduce<<<L.ka.nprob, 32, 0, L.stream>>>(L.ka, part, maxchunk);
}
void launch_finish_iteration(const Launch& L, double tol_e, double tol_rho, int count_iter) {
  k_finish_iteration<<<L.ka.nprob, 128, 0, L.stream>>>(L.ka, tol_e, tol_rho, count_iter);
}
void launch_pulay_gram(const Launch& Lchunks, double* part, int maxchunk, int hist) {
  if (Lchunks.map.total) k_pulay_gram<<<Lchunks.map.total, 256, 0, Lchunks.stream>>>(Lchunks.ka, part, maxchunk, hist);
}
void launch_pulay_solve(const Launch& L, const double* part, int maxchunk, int hist) {
  k_pulay_solve<<<L.ka.nprob, 32, 0, L.stream>>>(L.ka, part, maxchunk, hist);
}
template <typename T>
void launch_build_projectors(const Launch& Latoms, int deriv) {
  if (Latoms.map.total) k_build_projectors<T><<<Latoms.map.total, 256, 0, Latoms.stream>>>(Latoms.ka, deriv);
}
void launch_local_forces(const Launch& Lac, int maxchunk) {
  if (Lac.map.total) k_local_forces<<<Lac.map.total, 256, 0, Lac.stream>>>(Lac.ka, maxchunk);
}
void launch_force_total(const Launch& L, int maxchunk) {
  k_force_total<<<L.ka.nprob, 128, 0, L.stream>>>(L.ka, maxchunk);
}

template void launch_grid_energies<float>(const Launch&, double*, int);
template void launch_grid_energies<double>(const Launch&, double*, int);
template void launch_veff<float>(const Launch&, const double*);
template void launch_veff<double>(const Launch&, const double*);
template void launch_build_projectors<float>(const Launch&, int);
template void launch_build_projectors<double>(const Launch&, int);

}  // namespace sgo
