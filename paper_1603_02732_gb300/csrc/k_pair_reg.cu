// Register-FFT passes for line lengths N = 2M (96 ... 128) transformed by a pair of lanes
// (mixed path): each lane of the pair holds M elements, one radix-2 exchange by shuffles
// joins the halves (fft_reg.cuh: pair_inv).  The plane kernels follow k_plane_vpsi.cu and
// k_plane_density.cu (compact occupied rows, cp.async scatter, V_eff prefetch), the
// z-column kernels follow k_cols_reg.cu, with one lane pair per line.  Loops over lines are
// warp-uniform (every lane runs every transform, lanes without a line on zeros) because
// the pair exchange needs the whole warp.
#include "fft_reg.cuh"
#include "kernels.h"

namespace sgo {

namespace {

constexpr int PP = PLANE_REG_THREADS / 2;  // lane pairs of a plane CTA
constexpr int ZP_CP = ZREG_THREADS / 4;     // column pairs of a z-column CTA (one lane pair per column)

// Column of length N = 2M of the H.psi plane pass: inverse x transform, times v, forward
// x transform (as conj o inverse o conj), one M-point body run twice.  Lane h loads rows
// e = h M + j; after the inverse the lane holds times h + 2 q (q = dif_freq<M>(p)), which
// is the even/odd split that the forward transform starts from (decimation in time:
// Z[k] = E[k] + W^k O[k], Z[k + M] = E[k] - W^k O[k], E/O the M-point transforms of the
// even/odd samples); after it the lane holds Z[h M + dif_freq<M>(p)].
template <int M>
__device__ __forceinline__ void col_vpsi_pair(cplx<float>* col, int stride, const float* v, int vstride, int mx,
                                              int h, bool act) {
  constexpr int N = 2 * M;
  const int R = 2 * mx + 1;
  const cplx<float>* tn = twf<N>();
  cplx<float> x[M];
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const int e = h * M + j;
    const bool lo = e <= mx, hi = e >= N - mx;
    x[j] = (act && (lo || hi)) ? col[(lo ? e : e - N + R) * stride] : mk(0.f, 0.f);
  }
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 0) {
#pragma unroll
      for (int j = 0; j < M; ++j) {  // radix-2 decimation-in-frequency step of the inverse
        const cplx<float> o = shfl_pair(x[j]);
        if (h == 0) {
          x[j] = x[j] + o;
        } else {
          cplx<float> w = tn[j];
          w.y = -w.y;
          x[j] = (o - x[j]) * w;
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < M; ++j) x[j].y = -x[j].y;
    }
    reg_fft<float, M, 1>(x, twf<M>());
    if (pass == 0) {
      cplx<float> y[M];  // times h + 2q in natural q, times v
#pragma unroll
      for (int p = 0; p < M; ++p) {
        const int q = dif_freq<M>(p);
        y[q] = scale(x[p], act ? v[(h + 2 * q) * vstride] : 0.f);
      }
#pragma unroll
      for (int j = 0; j < M; ++j) x[j] = y[j];
    } else {
#pragma unroll
      for (int p = 0; p < M; ++p) {  // E or O at k = dif_freq<M>(p); join across the pair
        const cplx<float> own = mk(x[p].x, -x[p].y);
        const cplx<float> o = shfl_pair(own);
        const cplx<float> w = tn[dif_freq<M>(p)];
        x[p] = h == 0 ? own + w * o : o - w * own;
      }
    }
  }
  if (act) {
#pragma unroll
    for (int p = 0; p < M; ++p) {
      const int e = h * M + dif_freq<M>(p);
      const bool lo = e <= mx, hi = e >= N - mx;
      if (lo || hi) col[(lo ? e : e - N + R) * stride] = x[p];
    }
  }
}

// Column of the density pass: inverse x transform of the occupied rows, then
// acc[e] += fa Re^2 + fb Im^2 for every x row e (times h + 2 dif_freq<M>(p) of the lane).
template <int M>
__device__ __forceinline__ void col_density_pair(const cplx<float>* col, int stride, double* acc, int astride,
                                                 int mx, float fa, float fb, int h, bool act) {
  constexpr int N = 2 * M;
  const int R = 2 * mx + 1;
  cplx<float> x[M];
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const int e = h * M + j;
    const bool lo = e <= mx, hi = e >= N - mx;
    x[j] = (act && (lo || hi)) ? col[(lo ? e : e - N + R) * stride] : mk(0.f, 0.f);
  }
  pair_inv<M>(x, h);
  if (act) {
#pragma unroll
    for (int p = 0; p < M; ++p) {
      const int e = h + 2 * dif_freq<M>(p);
      acc[e * astride] += (double)(fa * x[p].x * x[p].x + fb * x[p].y * x[p].y);
    }
  }
}

#define SGO_PAIRS(X) X(96) X(100) X(108) X(120) X(128)

__device__ __forceinline__ void col_vpsi_pair_n(int n, cplx<float>* col, int stride, const float* v, int vstride,
                                                int mx, int h, bool act) {
  switch (n) {
#define SGO_CASE(N)                                                   \
  case N:                                                             \
    col_vpsi_pair<N / 2>(col, stride, v, vstride, mx, h, act);        \
    break;
    SGO_PAIRS(SGO_CASE)
#undef SGO_CASE
    default: break;
  }
}

__device__ __forceinline__ void col_density_pair_n(int n, const cplx<float>* col, int stride, double* acc,
                                                   int astride, int mx, float fa, float fb, int h, bool act) {
  switch (n) {
#define SGO_CASE(N)                                                            \
  case N:                                                                      \
    col_density_pair<N / 2>(col, stride, acc, astride, mx, fa, fb, h, act);    \
    break;
    SGO_PAIRS(SGO_CASE)
#undef SGO_CASE
    default: break;
  }
}

template <int M>
__device__ __forceinline__ void zline_inv_pair(const cplx<float>* line, cplx<float>* out, size_t zstride, int h,
                                               bool act) {
  cplx<float> x[M];
#pragma unroll
  for (int j = 0; j < M; ++j) x[j] = act ? line[h * M + j] : mk(0.f, 0.f);
  pair_inv<M>(x, h);
  if (act) {
#pragma unroll
    for (int p = 0; p < M; ++p) out[(size_t)(h + 2 * dif_freq<M>(p)) * zstride] = x[p];
  }
}

template <int M>
__device__ __forceinline__ void zline_fwd_pair(const cplx<float>* in, size_t zstride, cplx<float>* line, int h,
                                               bool act) {
  cplx<float> x[M];
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const cplx<float> v = act ? in[(size_t)(h * M + j) * zstride] : mk(0.f, 0.f);
    x[j] = mk(v.x, -v.y);
  }
  pair_inv<M>(x, h);
  if (act) {
#pragma unroll
    for (int p = 0; p < M; ++p) line[h + 2 * dif_freq<M>(p)] = mk(x[p].x, -x[p].y);
  }
}

__device__ __forceinline__ void zline_inv_pair_n(int n, const cplx<float>* line, cplx<float>* out, size_t zs, int h,
                                                 bool act) {
  switch (n) {
#define SGO_CASE(N)                                    \
  case N:                                              \
    zline_inv_pair<N / 2>(line, out, zs, h, act);      \
    break;
    SGO_PAIRS(SGO_CASE)
#undef SGO_CASE
    default: break;
  }
}

__device__ __forceinline__ void zline_fwd_pair_n(int n, const cplx<float>* in, size_t zs, cplx<float>* line, int h,
                                                 bool act) {
  switch (n) {
#define SGO_CASE(N)                                    \
  case N:                                              \
    zline_fwd_pair<N / 2>(in, zs, line, h, act);       \
    break;
    SGO_PAIRS(SGO_CASE)
#undef SGO_CASE
    default: break;
  }
}

__device__ __forceinline__ void zp_cols(int cp0, int cp1, int* col0, int* col1) {
  *col0 = cp0 == 0 ? 0 : 2 * cp0 - 1;
  *col1 = 2 * cp1 - 1;
}

}  // namespace

// H.psi plane pass, lengths N1, N2 of pair size.  CTA = (problem, band pair, block of Q
// z-planes), Q = max(1, PP / N2).
__global__ void __launch_bounds__(PLANE_REG_THREADS, 1) k_plane_vpsi_pair(KArgs ka) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int n1 = P.n1, n2 = P.n2, n3 = P.n3, mx = P.m1max, ncol = P.ncol, n12 = n1 * n2;
  const int R = 2 * mx + 1, P2 = n2 | 1, plane = R * P2;
  const int Q = max(1, PP / n2);
  const int nzb = (n3 + Q - 1) / Q;
  const int local = blockIdx.x - ka.start[p];
  const int pair = local / nzb, zb = local - pair * nzb;
  const int z0 = zb * Q, nq = min(Q, n3 - z0);
  const int h = threadIdx.x & 1, lp = threadIdx.x >> 1;
  cplx<float>* S = reinterpret_cast<cplx<float>*>(smem_raw);
  float* Vs = reinterpret_cast<float*>(S + Q * plane);
  cplx<float>* wc = reinterpret_cast<cplx<float>*>(P.Wc) + ((size_t)pair * n3 + z0) * ncol;
  const int* __restrict__ sidx = P.col_sidx;
  for (int t = threadIdx.x; t < nq * plane; t += blockDim.x) S[t] = mk(0.f, 0.f);
  __syncthreads();
  for (int q = 0; q < nq; ++q)
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) cp_async8(S + q * plane + sidx[c], wc + q * ncol + c);
  cp_async_commit();
  const float* veff = reinterpret_cast<const float*>(P.veff) + (size_t)z0 * n12;
  for (int t = threadIdx.x; t < nq * n12; t += blockDim.x) cp_async4(Vs + t, veff + t);
  cp_async_commit();
  cp_async_wait<1>();
  __syncthreads();
#pragma unroll 1
  for (int ph = 0; ph < 2; ++ph) {
    for (int b = 0; b < nq * R; b += PP) {
      const int l = b + lp;
      const bool act = l < nq * R;
      row_pair_n<PAIR_REG_MAXN>(n2, S + (act ? l : 0) * P2, ph == 1, h, act);
    }
    if (ph == 0) cp_async_wait<0>();
    __syncthreads();
    if (ph == 1) break;
    for (int b = 0; b < nq * n2; b += PP) {
      const int l = b + lp;
      const bool act = l < nq * n2;
      const int q = act ? l / n2 : 0, i2 = act ? l - q * n2 : 0;
      col_vpsi_pair_n(n1, S + q * plane + i2, P2, Vs + q * n12 + i2, n2, mx, h, act);
    }
    __syncthreads();
  }
  for (int q = 0; q < nq; ++q)
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) wc[q * ncol + c] = S[q * plane + sidx[c]];
}

// Density pass, lengths N1, N2 of pair size.  CTA = (problem, block of Q z-planes).
__global__ void __launch_bounds__(PLANE_REG_THREADS, 1) k_plane_density_pair(KArgs ka, const double* occ_override) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int n1 = P.n1, n2 = P.n2, n3 = P.n3, mx = P.m1max, ncol = P.ncol, n12 = n1 * n2;
  const int R = 2 * mx + 1, P2 = n2 | 1, plane = R * P2;
  const int Q = max(1, PP / n2);
  const int z0 = (blockIdx.x - ka.start[p]) * Q, nq = min(Q, n3 - z0);
  const int h = threadIdx.x & 1, lp = threadIdx.x >> 1;
  double* acc = reinterpret_cast<double*>(smem_raw);
  cplx<float>* S = reinterpret_cast<cplx<float>*>(acc + Q * n12);
  const int* __restrict__ sidx = P.col_sidx;
  const double* occ = occ_override ? occ_override : P.occ;
  for (int t = threadIdx.x; t < nq * n12; t += blockDim.x) acc[t] = 0.0;
  for (int pair = 0; pair < P.npair; ++pair) {
    const double fa = occ[2 * pair];
    const double fb = (2 * pair + 1 < P.nb) ? occ[2 * pair + 1] : 0.0;
    if (fa == 0.0 && fb == 0.0) continue;  // uniform across the block
    const cplx<float>* wc = reinterpret_cast<const cplx<float>*>(P.Wc) + ((size_t)pair * n3 + z0) * ncol;
    for (int t = threadIdx.x; t < nq * plane; t += blockDim.x) S[t] = mk(0.f, 0.f);
    __syncthreads();
    for (int q = 0; q < nq; ++q)
      for (int c = threadIdx.x; c < ncol; c += blockDim.x) cp_async8(S + q * plane + sidx[c], wc + q * ncol + c);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    for (int b = 0; b < nq * R; b += PP) {
      const int l = b + lp;
      const bool act = l < nq * R;
      row_pair_n<PAIR_REG_MAXN>(n2, S + (act ? l : 0) * P2, false, h, act);
    }
    __syncthreads();
    for (int b = 0; b < nq * n2; b += PP) {
      const int l = b + lp;
      const bool act = l < nq * n2;
      const int q = act ? l / n2 : 0, i2 = act ? l - q * n2 : 0;
      col_density_pair_n(n1, S + q * plane + i2, P2, acc + q * n12 + i2, n2, mx, (float)fa, (float)fb, h, act);
    }
    __syncthreads();
  }
  __syncthreads();
  const double io = 1.0 / P.omega;
  double* rho = P.rho_out + (size_t)z0 * n12;
  for (int t = threadIdx.x; t < nq * n12; t += blockDim.x) rho[t] = acc[t] * io;
}

// sphere -> z columns, N3 of pair size.  CTA = (problem, band pair, chunk of ZP_CP column
// pairs), one lane pair per compact column.
__global__ void __launch_bounds__(ZREG_THREADS) k_wave_to_cols_pair(KArgs ka, int src) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int nchunk = (P.ncp + ZP_CP - 1) / ZP_CP;
  const int local = blockIdx.x - ka.start[p];
  const int pair = local / nchunk, chunk = local - pair * nchunk;
  const int n3 = P.n3, L3 = n3 | 1;
  const int cp0 = chunk * ZP_CP, cp1 = min(cp0 + ZP_CP, P.ncp);
  int col0, col1;
  zp_cols(cp0, cp1, &col0, &col1);
  const int ncl = col1 - col0;
  cplx<float>* lines = reinterpret_cast<cplx<float>*>(smem_raw);
  for (int t = threadIdx.x; t < ncl * L3; t += blockDim.x) lines[t] = mk(0.f, 0.f);
  __syncthreads();
  const int ia = 2 * pair, ib = 2 * pair + 1;
  const bool hasb = ib < P.nb;
  const float* xa = wbuf<float>(P, src) + (size_t)ia * P.ld;
  const float* xb = wbuf<float>(P, src) + (size_t)(hasb ? ib : ia) * P.ld;
  const float rs2 = (float)(1.0 / SQRT2);
  const int e0 = P.cp_off[cp0], e1 = P.cp_off[cp1];
  for (int k = e0 + threadIdx.x; k < e1; k += blockDim.x) {
    const int cp = P.ent_cp[k];
    const int m3 = P.ent_m3[k];
    const cplx<float> ca = mk(xa[1 + 2 * k] * rs2, xa[2 + 2 * k] * rs2);
    const cplx<float> cb = hasb ? mk(xb[1 + 2 * k] * rs2, xb[2 + 2 * k] * rs2) : mk(0.f, 0.f);
    const int lp = cp == 0 ? 0 : 2 * cp - 1 - col0, lm = cp == 0 ? 0 : 2 * cp - col0;
    lines[lp * L3 + (m3 < 0 ? m3 + n3 : m3)] = mk(ca.x - cb.y, ca.y + cb.x);   // c_a(G) + i c_b(G)
    lines[lm * L3 + (m3 > 0 ? n3 - m3 : -m3)] = mk(ca.x + cb.y, cb.x - ca.y);  // c_a^* + i c_b^* at -G
  }
  if (cp0 == 0 && threadIdx.x == 0) lines[0] = mk(xa[0], hasb ? xb[0] : 0.f);
  __syncthreads();
  const int c = threadIdx.x >> 1, h = threadIdx.x & 1;
  const bool act = c < ncl;
  cplx<float>* wc = reinterpret_cast<cplx<float>*>(P.Wc) + (size_t)pair * n3 * P.ncol + col0 + (act ? c : 0);
  zline_inv_pair_n(n3, lines + (act ? c : 0) * L3, wc, (size_t)P.ncol, h, act);
}

// z columns -> sphere, N3 of pair size (band separation and kinetic term as in
// k_cols_to_wave_reg).
__global__ void __launch_bounds__(ZREG_THREADS) k_cols_to_wave_pair(KArgs ka, int src, int dst) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int nchunk = (P.ncp + ZP_CP - 1) / ZP_CP;
  const int local = blockIdx.x - ka.start[p];
  const int pair = local / nchunk, chunk = local - pair * nchunk;
  const int n3 = P.n3, L3 = n3 | 1;
  const int cp0 = chunk * ZP_CP, cp1 = min(cp0 + ZP_CP, P.ncp);
  int col0, col1;
  zp_cols(cp0, cp1, &col0, &col1);
  const int ncl = col1 - col0;
  cplx<float>* lines = reinterpret_cast<cplx<float>*>(smem_raw);
  {
    const int c = threadIdx.x >> 1, h = threadIdx.x & 1;
    const bool act = c < ncl;
    const cplx<float>* wc =
        reinterpret_cast<const cplx<float>*>(P.Wc) + (size_t)pair * n3 * P.ncol + col0 + (act ? c : 0);
    zline_fwd_pair_n(n3, wc, (size_t)P.ncol, lines + (act ? c : 0) * L3, h, act);
  }
  __syncthreads();
  const int ia = 2 * pair, ib = 2 * pair + 1;
  const bool hasb = ib < P.nb;
  const float* xa = wbuf<float>(P, src) + (size_t)ia * P.ld;
  const float* xb = wbuf<float>(P, src) + (size_t)(hasb ? ib : ia) * P.ld;
  float* ya = wbuf<float>(P, dst) + (size_t)ia * P.ld;
  float* yb = wbuf<float>(P, dst) + (size_t)(hasb ? ib : ia) * P.ld;
  const float hs2 = (float)(0.5 * SQRT2);
  const int e0 = P.cp_off[cp0], e1 = P.cp_off[cp1];
  for (int k = e0 + threadIdx.x; k < e1; k += blockDim.x) {
    const int cp = P.ent_cp[k];
    const int m3 = P.ent_m3[k];
    const int lp = cp == 0 ? 0 : 2 * cp - 1 - col0, lm = cp == 0 ? 0 : 2 * cp - col0;
    const cplx<float> fp = lines[lp * L3 + (m3 < 0 ? m3 + n3 : m3)];
    const cplx<float> fm = lines[lm * L3 + (m3 > 0 ? n3 - m3 : -m3)];
    const float ek = P.ekin32[1 + 2 * k];
    ya[1 + 2 * k] = (fp.x + fm.x) * hs2 + ek * xa[1 + 2 * k];
    ya[2 + 2 * k] = (fp.y - fm.y) * hs2 + ek * xa[2 + 2 * k];
    if (hasb) {
      yb[1 + 2 * k] = (fp.y + fm.y) * hs2 + ek * xb[1 + 2 * k];
      yb[2 + 2 * k] = (fm.x - fp.x) * hs2 + ek * xb[2 + 2 * k];
    }
  }
  if (cp0 == 0 && threadIdx.x == 0) {
    const cplx<float> f0 = lines[0];
    ya[0] = f0.x;
    if (hasb) yb[0] = f0.y;
  }
}

bool pair_plane_ok(int n1, int n2) { return pair_supported(n1) && pair_supported(n2); }
int pair_plane_ctas(int n2, int n3, int npair) {
  const int q = std::max(1, PP / n2);
  return npair * ((n3 + q - 1) / q);
}
size_t pair_plane_smem(int n1, int n2, int m1max) {
  const size_t q = std::max(1, PP / n2);
  return q * (2 * m1max + 1) * (n2 | 1) * sizeof(cplx<float>) + q * n1 * n2 * sizeof(float);
}
int pair_density_ctas(int n2, int n3) {
  const int q = std::max(1, PP / n2);
  return (n3 + q - 1) / q;
}
size_t pair_density_smem(int n1, int n2, int m1max) {
  const size_t q = std::max(1, PP / n2);
  return q * n1 * n2 * sizeof(double) + q * (2 * m1max + 1) * (n2 | 1) * sizeof(cplx<float>);
}
bool zpair_ok(int n3) { return pair_supported(n3); }
int zpair_ctas(int ncp, int npair) { return npair * ((ncp + ZP_CP - 1) / ZP_CP); }
size_t zpair_smem(int n3) { return (size_t)2 * ZP_CP * (n3 | 1) * sizeof(cplx<float>); }

void launch_plane_vpsi_pair(const Launch& L, size_t smem) {
  if (L.map.total) k_plane_vpsi_pair<<<L.map.total, PLANE_REG_THREADS, smem, L.stream>>>(L.ka);
}
void launch_plane_density_pair(const Launch& L, size_t smem, const double* occ_override) {
  if (L.map.total) k_plane_density_pair<<<L.map.total, PLANE_REG_THREADS, smem, L.stream>>>(L.ka, occ_override);
}
void launch_wave_to_cols_pair(const Launch& L, size_t smem, int src) {
  if (L.map.total) k_wave_to_cols_pair<<<L.map.total, ZREG_THREADS, smem, L.stream>>>(L.ka, src);
}
void launch_cols_to_wave_pair(const Launch& L, size_t smem, int src, int dst) {
  if (L.map.total) k_cols_to_wave_pair<<<L.map.total, ZREG_THREADS, smem, L.stream>>>(L.ka, src, dst);
}

bool pair_reg_init() { return upload_twiddles(); }

void pair_reg_set_smem_limits(size_t bytes) {
  cudaFuncSetAttribute(k_plane_vpsi_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_plane_density_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_wave_to_cols_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_cols_to_wave_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace sgo
