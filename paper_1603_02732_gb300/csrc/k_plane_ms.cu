// Multi-pass plane pass of H.psi (mixed path, the line lengths with a register transform).
//
// Every line transform of length N = A B runs as two passes of short DFTs held in registers
// (Cooley-Tukey in the Gentleman-Sande form), the line itself staying in shared memory:
//   inverse (G -> r), natural order in, "transposed" order out:
//     pass 1, group g < B:  Y[B k1 + g] = W_N^(+g k1) sum_{n1 < A} x[B n1 + g] W_A^(+n1 k1)
//     pass 2, group k1 < A: position B k1 + k2 receives sum_{g < B} Y[B k1 + g] W_B^(+g k2),
//                           the sample at k1 + A k2
//   forward (r -> G), transposed order in, natural order out:
//     pass 1, group k1 < A: Z[B k1 + m2] = W_N^(-k1 m2) sum_{k2 < B} v[B k1 + k2] W_B^(-k2 m2)
//     pass 2, group m2 < B: F[m2 + B m1] = sum_{k1 < A} Z[B k1 + m2] W_A^(-k1 m1)
// (W_N = exp(2 pi i / N); the products of the indices reduce mod N to the twiddles shown).
// A thread holds at most max(A, B) <= 10 complex values, so a CTA of 256 threads needs few
// registers and several CTAs share an SM, where one thread per whole line (k_plane_vpsi_reg)
// holds up to 72 and leaves one CTA per SM.  The cost is shared-memory traffic: the planes are
// stored whole (all n1 x rows) while the x lines are transformed.
//
// CTA = (problem, group of PLANE_MS_PAIRS band pairs, block of Q z-planes).  Per band pair:
// the compact columns land in the occupied x rows (|m1| <= m1max) of the CTA's planes; y
// inverse over the occupied rows (natural -> transposed y order); per column: x inverse (only
// the occupied rows are read), times V_eff/N at (x, y), x forward (only the occupied rows are
// written); y forward (transposed -> natural); the compact columns go back.  Rows are padded
// to n2 | 1 entries so that threads walking down columns or across rows hit distinct banks.
#include "fft_reg.cuh"
#include "kernels.h"

namespace sgo {

namespace {

// Factorisation N = A B of every register length (A, B <= 10).
__host__ __device__ constexpr int ms_a(int n) {
  switch (n) {
    case 10: return 2;
    case 12: return 3;
    case 15: return 3;
    case 16: return 4;
    case 18: return 3;
    case 20: return 4;
    case 24: return 4;
    case 25: return 5;
    case 27: return 3;
    case 30: return 5;
    case 32: return 4;
    case 36: return 6;
    case 40: return 5;
    case 45: return 5;
    case 48: return 6;
    case 50: return 5;
    case 54: return 6;
    case 60: return 6;
    case 64: return 8;
    case 72: return 8;
    default: return 0;
  }
}

// Shared memory of one plane (whole rows plus V_eff / N) and of the CTA's tables.
__host__ __device__ inline size_t ms_plane_bytes(int n1, int n2) {
  return (size_t)n1 * (n2 | 1) * 8 + (size_t)n1 * n2 * 4;
}
__host__ __device__ inline size_t ms_table_bytes(int n1, int n2) { return (size_t)(n1 + n2) * 8; }
constexpr size_t kMsPlaneBudget = PLANE_MS_BUDGET_KB * 1024;  // planes per CTA: as many as fit (at least one)
__host__ __device__ inline int ms_q(int n1, int n2, int n3) {
  int q = (int)(kMsPlaneBudget / ms_plane_bytes(n1, n2));
  q = q < 1 ? 1 : (q > 8 ? 8 : q);
  return q < n3 ? q : n3;
}

// quotient of small non-negative integers by the reciprocal (exact for t < 2^16, d <= 1024)
__device__ __forceinline__ int qdiv(int t, float inv) { return __float2int_rz(((float)t + 0.5f) * inv); }

struct MsPlanes {
  cplx<float>* S;            // plane q at S + q * pstride, x row e at + e * P2
  const float* V;            // V_eff / N: plane q at V + q * n12, [x * n2 + c], the column
                             // positions c in the transposed y order of the y inverse
  const cplx<float>* twx;    // exp(-2 pi i t / n1)
  const cplx<float>* twy;    // exp(-2 pi i t / n2)
  int n1, n2, P2, pstride, n12, nq, mx, R;
  float inv_R, inv_n2;
};

// occupied x row rho (0 .. R-1) of the CTA's line l = q R + rho
__device__ __forceinline__ cplx<float>* ms_row(const MsPlanes& p, int l) {
  const int q = qdiv(l, p.inv_R), rho = l - q * p.R;
  const int e = rho <= p.mx ? rho : rho + p.n1 - p.R;
  return p.S + q * p.pstride + e * p.P2;
}
__device__ __forceinline__ bool ms_occ(const MsPlanes& p, int e) { return e <= p.mx || e >= p.n1 - p.mx; }

template <int R>
__device__ __forceinline__ void sdft(cplx<float> (&v)[R], float sg, const cplx<float>* tw, int stride) {
  Bfly<float, R>::run(v, sg, tw, stride);
}

// y inverse over the occupied rows (n2 = A B): natural -> transposed order
template <int A, int B>
__device__ __forceinline__ void ms_y_inv(const MsPlanes& p) {
  const int nl = p.nq * p.R;
  const float inv_nl = 1.f / (float)nl;
  for (int t = threadIdx.x; t < B * nl; t += blockDim.x) {
    const int g = qdiv(t, inv_nl), l = t - g * nl;
    cplx<float>* row = ms_row(p, l);
    cplx<float> v[A];
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) v[n1] = row[B * n1 + g];
    sdft<A>(v, 1.f, p.twy, B);
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) row[B * k1 + g] = k1 == 0 ? v[0] : v[k1] * conj(p.twy[g * k1]);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < A * nl; t += blockDim.x) {
    const int k1 = qdiv(t, inv_nl), l = t - k1 * nl;
    cplx<float>* row = ms_row(p, l) + B * k1;
    cplx<float> v[B];
#pragma unroll
    for (int g = 0; g < B; ++g) v[g] = row[g];
    sdft<B>(v, 1.f, p.twy, A);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) row[k2] = v[k2];
  }
  __syncthreads();
}

// y forward over the occupied rows: transposed -> natural order
template <int A, int B>
__device__ __forceinline__ void ms_y_fwd(const MsPlanes& p) {
  const int nl = p.nq * p.R;
  const float inv_nl = 1.f / (float)nl;
  for (int t = threadIdx.x; t < A * nl; t += blockDim.x) {
    const int k1 = qdiv(t, inv_nl), l = t - k1 * nl;
    cplx<float>* row = ms_row(p, l) + B * k1;
    cplx<float> v[B];
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) v[k2] = row[k2];
    sdft<B>(v, -1.f, p.twy, A);
#pragma unroll
    for (int m2 = 0; m2 < B; ++m2) row[m2] = m2 == 0 ? v[0] : v[m2] * p.twy[k1 * m2];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < B * nl; t += blockDim.x) {
    const int m2 = qdiv(t, inv_nl), l = t - m2 * nl;
    cplx<float>* row = ms_row(p, l);
    cplx<float> v[A];
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) v[k1] = row[B * k1 + m2];
    sdft<A>(v, -1.f, p.twy, B);
#pragma unroll
    for (int m1 = 0; m1 < A; ++m1) row[m2 + B * m1] = v[m1];
  }
  __syncthreads();
}

// x lines (n1 = A B), one per column of the CTA's planes: inverse (occupied rows in),
// times V_eff / N, forward (occupied rows out)
template <int A, int B>
__device__ __forceinline__ void ms_x(const MsPlanes& p) {
  const int nl = p.nq * p.n2, P2 = p.P2;
  const float inv_nl = 1.f / (float)nl;
  for (int t = threadIdx.x; t < B * nl; t += blockDim.x) {
    const int g = qdiv(t, inv_nl), l = t - g * nl;
    const int q = qdiv(l, p.inv_n2), c = l - q * p.n2;
    cplx<float>* col = p.S + q * p.pstride + c;
    cplx<float> v[A];
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) {
      const int e = B * n1 + g;
      v[n1] = ms_occ(p, e) ? col[e * P2] : mk(0.f, 0.f);
    }
    sdft<A>(v, 1.f, p.twx, B);
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) col[(B * k1 + g) * P2] = k1 == 0 ? v[0] : v[k1] * conj(p.twx[g * k1]);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < A * nl; t += blockDim.x) {
    const int k1 = qdiv(t, inv_nl), l = t - k1 * nl;
    const int q = qdiv(l, p.inv_n2), c = l - q * p.n2;
    cplx<float>* col = p.S + q * p.pstride + c + B * k1 * P2;
    const float* vq = p.V + q * p.n12 + c;
    cplx<float> v[B];
#pragma unroll
    for (int g = 0; g < B; ++g) v[g] = col[g * P2];
    sdft<B>(v, 1.f, p.twx, A);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) v[k2] = scale(v[k2], vq[(k1 + A * k2) * p.n2]);
    sdft<B>(v, -1.f, p.twx, A);
#pragma unroll
    for (int m2 = 0; m2 < B; ++m2) col[m2 * P2] = m2 == 0 ? v[0] : v[m2] * p.twx[k1 * m2];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < B * nl; t += blockDim.x) {
    const int m2 = qdiv(t, inv_nl), l = t - m2 * nl;
    const int q = qdiv(l, p.inv_n2), c = l - q * p.n2;
    cplx<float>* col = p.S + q * p.pstride + c;
    cplx<float> v[A];
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) v[k1] = col[(B * k1 + m2) * P2];
    sdft<A>(v, -1.f, p.twx, B);
#pragma unroll
    for (int m1 = 0; m1 < A; ++m1) {
      const int e = m2 + B * m1;
      if (ms_occ(p, e)) col[e * P2] = v[m1];
    }
  }
  __syncthreads();
}

#define SGO_MS_SIZES(X)                                                                                  \
  X(10, 2, 5) X(12, 3, 4) X(15, 3, 5) X(16, 4, 4) X(18, 3, 6) X(20, 4, 5) X(24, 4, 6) X(25, 5, 5) X(27, 3, 9) \
  X(30, 5, 6) X(32, 4, 8) X(36, 6, 6) X(40, 5, 8) X(45, 5, 9) X(48, 6, 8) X(50, 5, 10) X(54, 6, 9)         \
  X(60, 6, 10) X(64, 8, 8) X(72, 8, 9)

__device__ __forceinline__ void ms_y_inv_n(const MsPlanes& p) {
  switch (p.n2) {
#define SGO_CASE(N, A, B) \
  case N:                 \
    ms_y_inv<A, B>(p);    \
    break;
    SGO_MS_SIZES(SGO_CASE)
#undef SGO_CASE
    default: break;
  }
}
__device__ __forceinline__ void ms_y_fwd_n(const MsPlanes& p) {
  switch (p.n2) {
#define SGO_CASE(N, A, B) \
  case N:                 \
    ms_y_fwd<A, B>(p);    \
    break;
    SGO_MS_SIZES(SGO_CASE)
#undef SGO_CASE
    default: break;
  }
}
__device__ __forceinline__ void ms_x_n(const MsPlanes& p) {
  switch (p.n1) {
#define SGO_CASE(N, A, B) \
  case N:                 \
    ms_x<A, B>(p);        \
    break;
    SGO_MS_SIZES(SGO_CASE)
#undef SGO_CASE
    default: break;
  }
}

// offset of length n's table in c_tw (a register length), -1 otherwise
__device__ __forceinline__ int ms_tw_offset(int n) {
  switch (n) {
#define SGO_CASE(N, A, B) \
  case N:                 \
    return reg_table_offset(N);
    SGO_MS_SIZES(SGO_CASE)
#undef SGO_CASE
    default: return -1;
  }
}

}  // namespace

__global__ void __launch_bounds__(PLANE_MS_THREADS, PLANE_MS_MINB) k_plane_vpsi_ms(KArgs ka) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int n1 = P.n1, n2 = P.n2, n3 = P.n3, mx = P.m1max, ncol = P.ncol, n12 = n1 * n2;
  const int R = 2 * mx + 1, P2 = n2 | 1, pstride = n1 * P2;
  const int Q = ms_q(n1, n2, n3);
  const int nzb = (n3 + Q - 1) / Q;
  const int local = blockIdx.x - ka.start[p];
  const int grp = local / nzb, zb = local - grp * nzb;
  const int z0 = zb * Q, nq = min(Q, n3 - z0);
  const int pr0 = grp * PLANE_MS_PAIRS, pr1 = min(P.npair, pr0 + PLANE_MS_PAIRS);
  cplx<float>* const S = reinterpret_cast<cplx<float>*>(smem_raw);
  cplx<float>* const twx = S + Q * pstride;
  cplx<float>* const twy = twx + n1;
  float* const Vs = reinterpret_cast<float*>(twy + n2);
  const int ox = ms_tw_offset(n1), oy = ms_tw_offset(n2);
  const int ay = ms_a(n2), by = n2 / ay;
  for (int t = threadIdx.x; t < n1; t += blockDim.x) twx[t] = c_tw[ox + t];
  for (int t = threadIdx.x; t < n2; t += blockDim.x) twy[t] = c_tw[oy + t];
  // the occupied rows start zero (the compact columns fill part of them)
  for (int t = threadIdx.x; t < nq * R * P2; t += blockDim.x) {
    const int l = t / P2, j = t - l * P2;
    const int q = l / R, rho = l - q * R;
    const int e = rho <= mx ? rho : rho + n1 - R;
    S[q * pstride + e * P2 + j] = mk(0.f, 0.f);
  }
  // V_eff / N with its columns in the transposed y order (column position B k1 + k2 of the y
  // inverse holds y = k1 + A k2), so that the x pass reads it at consecutive addresses
  const float* veff = reinterpret_cast<const float*>(P.veff) + (size_t)z0 * n12;
  for (int t = threadIdx.x; t < nq * n12; t += blockDim.x) {
    const int row = t / n2, c = t - row * n2, k1 = c / by, k2 = c - k1 * by;
    cp_async4(Vs + t, veff + row * n2 + k1 + ay * k2);
  }
  cp_async_commit();
  MsPlanes mp{S, Vs, twx, twy, n1, n2, P2, pstride, n12, nq, mx, R, 1.f / (float)R, 1.f / (float)n2};
  const int* __restrict__ sidx = P.col_sidx;
  const float inv_P2 = 1.f / (float)P2;
  // compact slot rho P2 + i2 -> whole-row slot e P2 + i2
  auto slot = [&](int s) {
    const int rho = qdiv(s, inv_P2), i2 = s - rho * P2;
    return (rho <= mx ? rho : rho + n1 - R) * P2 + i2;
  };
  __syncthreads();
#pragma unroll 1
  for (int pair = pr0; pair < pr1; ++pair) {
    const cplx<float>* wc = reinterpret_cast<const cplx<float>*>(P.Wc) + ((size_t)pair * n3 + z0) * ncol;
    for (int q = 0; q < nq; ++q)
      for (int c = threadIdx.x; c < ncol; c += blockDim.x) cp_async8(S + q * pstride + slot(sidx[c]), wc + q * ncol + c);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    ms_y_inv_n(mp);
    ms_x_n(mp);
    ms_y_fwd_n(mp);
    cplx<float>* wo = reinterpret_cast<cplx<float>*>(P.Wc) + ((size_t)pair * n3 + z0) * ncol;
    for (int q = 0; q < nq; ++q)
      for (int c = threadIdx.x; c < ncol; c += blockDim.x) wo[q * ncol + c] = S[q * pstride + slot(sidx[c])];
    __syncthreads();
    for (int t = threadIdx.x; t < nq * R * P2; t += blockDim.x) {
      const int l = t / P2, j = t - l * P2;
      const int q = l / R, rho = l - q * R;
      const int e = rho <= mx ? rho : rho + n1 - R;
      S[q * pstride + e * P2 + j] = mk(0.f, 0.f);
    }
    __syncthreads();
  }
}

int plane_ms_ctas(int n1, int n2, int n3, int npair) {
  const int q = ms_q(n1, n2, n3);
  return ((npair + PLANE_MS_PAIRS - 1) / PLANE_MS_PAIRS) * ((n3 + q - 1) / q);
}
size_t plane_ms_smem(int n1, int n2, int n3) {
  return (size_t)ms_q(n1, n2, n3) * ms_plane_bytes(n1, n2) + ms_table_bytes(n1, n2);
}
void launch_plane_vpsi_ms(const Launch& L, size_t smem) {
  if (!L.map.total) return;
  k_plane_vpsi_ms<<<L.map.total, PLANE_MS_THREADS, smem, L.stream>>>(L.ka);
}
bool plane_ms_init() { return upload_twiddles(); }
void plane_ms_set_smem_limits(size_t bytes) {
  cudaFuncSetAttribute(k_plane_vpsi_ms, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace sgo
