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
__device__ __forceinline__ float exp_t(float x) { return expf(x); }
__device__ __forceinline__ double exp_t(double x) { return exp(x); }
__device__ __forceinline__ float expm1_t(float x) { return expm1f(x); }
__device__ __forceinline__ double expm1_t(double x) { return expm1(x); }

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

// ---- PBE (Perdew, Burke & Ernzerhof 1996; uniform-gas correlation of Perdew & Wang 1992) ----
// e(rho, sigma) = rho eps_xc with sigma = |grad rho|^2, and its two partial derivatives,
// carried through the formula as first-order dual numbers (value, d/drho, d/dsigma).
template <typename R>
struct Dual {
  R v, r, s;
};
template <typename R>
__device__ __forceinline__ Dual<R> dmk(R v, R r, R s) {
  Dual<R> d;
  d.v = v;
  d.r = r;
  d.s = s;
  return d;
}
template <typename R>
__device__ __forceinline__ Dual<R> operator+(Dual<R> a, Dual<R> b) { return dmk(a.v + b.v, a.r + b.r, a.s + b.s); }
template <typename R>
__device__ __forceinline__ Dual<R> operator-(Dual<R> a, Dual<R> b) { return dmk(a.v - b.v, a.r - b.r, a.s - b.s); }
template <typename R>
__device__ __forceinline__ Dual<R> operator*(Dual<R> a, Dual<R> b) {
  return dmk(a.v * b.v, a.r * b.v + a.v * b.r, a.s * b.v + a.v * b.s);
}
template <typename R>
__device__ __forceinline__ Dual<R> operator/(Dual<R> a, Dual<R> b) {
  const R q = a.v / b.v, ib = R(1) / b.v;
  return dmk(q, (a.r - q * b.r) * ib, (a.s - q * b.s) * ib);
}
template <typename R>
__device__ __forceinline__ Dual<R> operator+(Dual<R> a, R c) { return dmk(a.v + c, a.r, a.s); }
template <typename R>
__device__ __forceinline__ Dual<R> operator*(R c, Dual<R> a) { return dmk(c * a.v, c * a.r, c * a.s); }
template <typename R>
__device__ __forceinline__ Dual<R> dlog(Dual<R> a) {
  const R ia = R(1) / a.v;
  return dmk(log_t(a.v), a.r * ia, a.s * ia);
}
template <typename R>
__device__ __forceinline__ Dual<R> dexpm1(Dual<R> a) {  // exp(a) - 1
  const R e = exp_t(a.v);
  return dmk(expm1_t(a.v), e * a.r, e * a.s);
}
template <typename R>
__device__ __forceinline__ Dual<R> dsqrt(Dual<R> a) {
  const R q = sqrt_t(a.v), h = R(0.5) / q;
  return dmk(q, h * a.r, h * a.s);
}
template <typename R>
__device__ __forceinline__ Dual<R> dcbrt(Dual<R> a) {
  const R c = cbrt_t(a.v), h = c / (R(3) * a.v);
  return dmk(c, h * a.r, h * a.s);
}
template <typename R>
__device__ __forceinline__ Dual<R> dmin(Dual<R> a, R cap) { return a.v > cap ? dmk(cap, R(0), R(0)) : a; }

constexpr double PBE_RHO_CUT = 1e-10;  // points below: e = 0 (near-empty regions)
// Reduced gradients beyond this bound leave F_x and H saturated to 3e-8 relative: capped,
// so that the FP32 path's intermediate products stay finite.
constexpr double PBE_S2_CAP = 1e8;

// (e, de/drho, de/dsigma) at one point; rho <= PBE_RHO_CUT gives zeros.
template <typename R>
__device__ __forceinline__ void pbe_point(R rho_v, R sigma_v, R* e, R* dr, R* ds) {
  if (!(rho_v > R(PBE_RHO_CUT))) {
    *e = *dr = *ds = R(0);
    return;
  }
  const R kappa = R(0.804), beta = R(0.06672455060314922);
  const R mu = R(0.06672455060314922 * 9.8696044010893586 / 3.0);  // beta pi^2 / 3
  const R gamma = R(0.031090690869654895);                          // (1 - ln 2) / pi^2
  const Dual<R> rho = dmk(rho_v, R(1), R(0));
  const Dual<R> sig = dmk(sigma_v > R(0) ? sigma_v : R(0), R(0), R(1));
  const Dual<R> c = dcbrt(rho);                          // rho^(1/3)
  const Dual<R> kf = R(3.0936677262801355) * c;          // (3 pi^2)^(1/3) rho^(1/3)
  const Dual<R> rho2 = rho * rho;
  // exchange: -(3/4) (3/pi)^(1/3) rho^(4/3) F_x(s^2)
  const Dual<R> s2 = dmin(sig / (R(4) * (kf * kf * rho2)), R(PBE_S2_CAP));
  const Dual<R> fx = dmk(R(1) + kappa, R(0), R(0)) - kappa * (dmk(R(1), R(0), R(0)) / ((mu / kappa) * s2 + R(1)));
  const Dual<R> ex = R(-0.75 * 0.98474502184269641) * (rho * c) * fx;
  // correlation: rho (eps_c^PW92(r_s) + H(r_s, t^2))
  const Dual<R> rs = R(0.62035049089940009) * (dmk(R(1), R(0), R(0)) / c);  // (3/(4 pi))^(1/3) / rho^(1/3)
  const Dual<R> srs = dsqrt(rs);
  const Dual<R> den = R(2 * 0.031091) *
                      (R(7.5957) * srs + R(3.5876) * rs + R(1.6382) * (rs * srs) + R(0.49294) * (rs * rs));
  const Dual<R> ec = R(-2 * 0.031091) * (R(0.21370) * rs + R(1)) * dlog(dmk(R(1), R(0), R(0)) / den + R(1));
  const Dual<R> t2 = dmin(sig / ((R(16 / 3.14159265358979324) * kf) * rho2), R(PBE_S2_CAP));  // 4 k_s^2 rho^2
  const Dual<R> a = (beta / gamma) * (dmk(R(1), R(0), R(0)) / dexpm1(R(-1) / gamma * ec));
  const Dual<R> at2 = a * t2;
  const Dual<R> h = gamma * dlog((beta / gamma) * (t2 * (at2 + R(1))) / (at2 + at2 * at2 + R(1)) + R(1));
  const Dual<R> tot = ex + rho * (ec + h);
  *e = tot.v;
  *dr = tot.r;
  *ds = tot.s;
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
    } else if (P.xc == 1) {  // PBE: gfft = rho + i (V_H + de/drho), gfft4 = div(2 de/dsigma grad rho)
      const double2 c = P.gfft[i];
      P.rho_in[i] = c.x;
      val = P.vion_r[i] + c.y - P.gfft4[i].x;
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

// PBE gradient: gfft3 := (i G_x - G_y) rho(G), gfft4 := i G_z rho(G) (zero on Nyquist planes),
// so that one inverse transform gives d_x rho + i d_y rho and another d_z rho.  src 0:
// rho_in(G); src 1: N rho_out(G) in gfft2 (scaled by 1/N).
__global__ void k_gga_grad(KArgs ka, int src) {
  GRID_EW_PROLOGUE
  const double sc = src ? 1.0 / P.ngrid : 1.0;
  const double2* rg = src ? P.gfft2 : P.rhog_in;
  for (int i = base + threadIdx.x; i < end; i += blockDim.x) {
    const GPt q = grid_pt(P, i);
    double G[3];
    gcart(P, q.m1, q.m2, q.m3, G);
    const double2 r = rg[i];
    const double a = q.nyq ? 0.0 : r.x * sc, b = q.nyq ? 0.0 : r.y * sc;
    P.gfft3[i] = make_double2(-G[0] * b - G[1] * a, G[0] * a - G[1] * b);
    P.gfft4[i] = make_double2(-G[2] * b, G[2] * a);
  }
}

// PBE at each point of rho_in(r) (real part of gfft) with grad rho_in (gfft3 = d_x + i d_y,
// gfft4 = d_z): de/drho joins V_H in the imaginary part of gfft, and h = 2 de/dsigma grad rho
// replaces the gradient (gfft3 = h_x + i h_y, gfft4 = h_z).
template <typename T>
__global__ void k_gga_point(KArgs ka) {
  GRID_EW_PROLOGUE
  for (int i = base + threadIdx.x; i < end; i += blockDim.x) {
    const double2 c = P.gfft[i], gxy = P.gfft3[i];
    const double gz = P.gfft4[i].x;
    T e, dr, ds;
    pbe_point<T>((T)fmax(c.x, 0.0), (T)(gxy.x * gxy.x + gxy.y * gxy.y + gz * gz), &e, &dr, &ds);
    const double two_ds = 2.0 * (double)ds;
    P.gfft[i] = make_double2(c.x, c.y + (double)dr);
    P.gfft3[i] = make_double2(two_ds * gxy.x, two_ds * gxy.y);
    P.gfft4[i] = make_double2(two_ds * gz, 0.0);
  }
}

// div h in G space from the forward transforms F = N (h_x + i h_y)(G) (gfft3) and
// N h_z(G) (gfft4): h_x(G) = (F(G) + F(-G)^*) / 2N, h_y(G) = (F(G) - F(-G)^*) / 2iN;
// gfft4 := i G.h(G) (zero on Nyquist planes), whose inverse transform is div h.
__global__ void k_gga_div(KArgs ka) {
  GRID_EW_PROLOGUE
  const double inv_n = 1.0 / P.ngrid;
  for (int i = base + threadIdx.x; i < end; i += blockDim.x) {
    int i1, i2, i3;
    const GPt q = grid_pt(P, i, &i1, &i2, &i3);
    double G[3];
    gcart(P, q.m1, q.m2, q.m3, G);
    const int j1 = i1 ? P.n1 - i1 : 0, j2 = i2 ? P.n2 - i2 : 0, j3 = i3 ? P.n3 - i3 : 0;
    const int j = (j3 * P.n1 + j1) * P.n2 + j2;  // -G (plane-major index)
    const double2 f = P.gfft3[i], fm = P.gfft3[j], hz = P.gfft4[i];
    // h_x = (f + conj fm)/2, h_y = (f - conj fm)/(2i)
    const double hxr = 0.5 * (f.x + fm.x), hxi = 0.5 * (f.y - fm.y);
    const double hyr = 0.5 * (f.y + fm.y), hyi = -0.5 * (f.x - fm.x);
    const double sr = G[0] * hxr + G[1] * hyr + G[2] * hz.x;  // G.h
    const double si = G[0] * hxi + G[1] * hyi + G[2] * hz.y;
    P.gfft4[i] = q.nyq ? make_double2(0.0, 0.0) : make_double2(-si * inv_n, sr * inv_n);  // i G.h / N
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
    if (P.xc == 1) {  // PBE with grad rho_out in gfft3 (x + i y) and gfft4 (z)
      const double2 gxy = P.gfft3[i];
      const double gz = P.gfft4[i].x;
      T e, dr, ds;
      pbe_point<T>((T)fmax(r, 0.0), (T)(gxy.x * gxy.x + gxy.y * gxy.y + gz * gz), &e, &dr, &ds);
      s[1] += (double)e;
    } else {
      T exc, vxc;
      lda_pz81<T>((T)r, &exc, &vxc);
      s[1] += fmax(r, 0.0) * (double)exc;
    }
    s[0] += P.vion_r[i] * r;
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
    for (int k = 0; k < P.nproj; ++k) {
      double pr = P.proj[(size_t)k * P.nb + i];
      s += P.pj_d[k] * pr * pr;
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
// Projectors (packed real form): B[k] = pack(beta_k(G) exp(-iG.R_I)) for projector k of atom
// I and, for the forces, dB[3k+a] = pack(-i G_a B[k](G)) = (G_a b_im, -G_a b_re).
//   s: beta(G) = Omega^{-1/2} N (2 pi)^{3/2} rp^3 exp(-G^2 rp^2/2), N^2 = 1/(pi^{3/2} rp^3);
//   p_m: beta(G) = -i G_m Omega^{-1/2} N_p (2 pi)^{3/2} s^5 exp(-G^2 s^2/2), N_p^2 = 2/(pi^{3/2} s^5)
//        (the transform of N_p x_m exp(-r^2/(2 s^2)), zero at G = 0).
// CTA = (problem, projector).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_build_projectors(KArgs ka, int deriv) {
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int k = blockIdx.x - ka.start[p];
  const int a = P.pj_atom[k], kind = P.pj_kind[k];
  const double rp = P.pj_rp[k];
  const double r3 = rp * rp * rp;
  // radial amplitude: s N (2 pi)^{3/2} rp^3; p N_p (2 pi)^{3/2} s^5 (times -i G_m below)
  const double amp = kind == 0 ? (1.0 / sqrt(pow(PI, 1.5) * r3)) * pow(2.0 * PI, 1.5) * r3 / sqrt(P.omega)
                               : sqrt(2.0 / (pow(PI, 1.5) * r3 * rp * rp)) * pow(2.0 * PI, 1.5) * r3 * rp * rp /
                                     sqrt(P.omega);
  T* b = reinterpret_cast<T*>(P.B) + (size_t)k * P.ld;
  T* d0 = deriv ? reinterpret_cast<T*>(P.dB) + (size_t)(3 * k) * P.ld : nullptr;
  const int* em1 = P.ent_m3 - 2 * P.nhalf;
  const int* em2 = P.ent_m3 - P.nhalf;
  for (int t = threadIdx.x; t <= P.nhalf; t += blockDim.x) {
    if (t == 0) {  // G = 0: the s amplitude; a p projector has none
      if (!deriv) b[0] = (T)(kind == 0 ? amp : 0.0);
      else for (int c = 0; c < 3; ++c) d0[(size_t)c * P.ld] = T(0);
      continue;
    }
    const int e = t - 1;
    const double g2 = 2.0 * P.ekin[1 + 2 * e];
    const double bg = amp * exp(-0.5 * g2 * rp * rp);
    const int m1 = em1[e], m2 = em2[e], m3 = P.ent_m3[e];
    const int i1 = m1 < 0 ? m1 + P.n1 : m1, i2 = m2 < 0 ? m2 + P.n2 : m2, i3 = m3 < 0 ? m3 + P.n3 : m3;
    cplx<double> ph = phase_at(P, a, i1, i2, i3);
    double bre, bim;
    if (kind == 0) {
      bre = SQRT2 * bg * ph.x;
      bim = SQRT2 * bg * ph.y;
    } else {  // -i c ph with c = G_m bg: (c ph.y, -c ph.x)
      const double cm = P.gvec[(size_t)(kind - 1) * P.ld + 1 + 2 * e] * bg;
      bre = SQRT2 * cm * ph.y;
      bim = -SQRT2 * cm * ph.x;
    }
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

// Total: local partials + nonlocal -2 sum_k D_k sum_n f_n p_nk dp_nka over the atom's
// projectors k + Ewald.  CTA per problem.
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
    double nl = 0.0;  // sum over the atom's projectors k of D_k sum_n f_n p_nk dp_nka
    for (int k = P.pj_first[a]; k < P.pj_first[a + 1]; ++k) {
      double t = 0.0;
      for (int n = 0; n < P.nb; ++n)
        t += P.occ[n] * P.proj[(size_t)k * P.nb + n] * P.dproj[(size_t)(3 * k + c) * P.nb + n];
      nl += P.pj_d[k] * t;
    }
    P.forces[e] = s - 2.0 * nl + P.ewald_f[e];
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
void launch_gga_grad(const Launch& L, int src) {
  if (ew_blocks(L)) k_gga_grad<<<L.map.total, 256, 0, L.stream>>>(L.ka, src);
}
template <typename T>
void launch_gga_point(const Launch& L) {
  if (ew_blocks(L)) k_gga_point<T><<<L.map.total, 256, 0, L.stream>>>(L.ka);
}
template void launch_gga_point<float>(const Launch&);
template void launch_gga_point<double>(const Launch&);
void launch_gga_div(const Launch& L) {
  if (ew_blocks(L)) k_gga_div<<<L.map.total, 256, 0, L.stream>>>(L.ka);
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
