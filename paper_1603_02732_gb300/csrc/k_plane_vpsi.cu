// Register-FFT plane pass of H.psi (mixed path, line lengths with a register transform;
// the line transforms are in fft_reg.cuh).
// CTA = (problem, group of PLANE_PAIR_GROUP band pairs, block of Q = blockDim / N2
// z-planes).  Shared memory holds only the occupied x rows of each plane (|m1| <= m1max,
// compact row index rho), twice (double buffer), rows padded to an odd length (N2 | 1) so
// that a thread per row and a thread per column both touch 16 distinct 8-byte bank pairs
// per half warp, and the planes' V_eff / N (loaded once for the group).  Per band pair:
// its compact columns have landed in one buffer by asynchronous copies to precomputed
// slots (issued while the previous pair computed), the next pair's start landing in the
// other; y inverse (thread per occupied row); per column: x inverse of the occupied rows,
// times V_eff/N, x forward, occupied rows back (thread per column, the full column in
// registers); y forward; gather the compact columns.
#include "fft_reg.cuh"
#include "kernels.h"

namespace sgo {

namespace {

// Column of N elements (x direction) at col[rho * stride]: occupied rows e <= mx and
// e >= N - mx sit at rho = e resp. e - N + 2 mx + 1, the others are zero.  Inverse
// transform, times v, forward transform, the forward one computed as
// conj(inverse(conj(.))): one transform body runs twice (a loop that is not unrolled),
// which halves the code the warps stream through.
template <int N>
__device__ __forceinline__ void col_vpsi(cplx<float>* col, int stride, const float* v, int vstride, int mx) {
  const int R = 2 * mx + 1;
  cplx<float> x[N];
#pragma unroll
  for (int e = 0; e < N; ++e) {
    const bool lo = e <= mx, hi = e >= N - mx;
    x[e] = (lo || hi) ? col[(lo ? e : e - N + R) * stride] : mk(0.f, 0.f);
  }
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    reg_fft<float, N, 1>(x, twf<N>());
    cplx<float> y[N];  // natural order, conjugated (pass 0: times v)
#pragma unroll
    for (int p = 0; p < N; ++p) {
      const int e = dif_freq<N>(p);
      const float f = pass == 0 ? v[e * vstride] : 1.f;
      y[e] = mk(f * x[p].x, -f * x[p].y);
    }
#pragma unroll
    for (int e = 0; e < N; ++e) x[e] = y[e];
  }
#pragma unroll
  for (int e = 0; e < N; ++e) {
    const bool lo = e <= mx, hi = e >= N - mx;
    if (lo || hi) col[(lo ? e : e - N + R) * stride] = x[e];
  }
}

template <int MAXN>
__device__ __forceinline__ void col_vpsi_n(int n, cplx<float>* col, int stride, const float* v, int vstride,
                                           int mx) {
  switch (n) {
#define SGO_COL(N)                                                     \
  case N:                                                              \
    if constexpr (N <= MAXN) col_vpsi<N>(col, stride, v, vstride, mx); \
    break;
    SGO_COL(10) SGO_COL(12) SGO_COL(15) SGO_COL(16) SGO_COL(18) SGO_COL(20) SGO_COL(24) SGO_COL(25) SGO_COL(27)
    SGO_COL(30) SGO_COL(32) SGO_COL(36) SGO_COL(40) SGO_COL(45) SGO_COL(48) SGO_COL(50) SGO_COL(54) SGO_COL(60)
    SGO_COL(64) SGO_COL(72)
#undef SGO_COL
    default: break;
  }
}

}  // namespace

template <int MAXN>
__global__ void __launch_bounds__(PLANE_REG_THREADS, MAXN <= 40 ? 2 : 1) k_plane_vpsi_reg(KArgs ka) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int n1 = P.n1, n2 = P.n2, n3 = P.n3, mx = P.m1max, ncol = P.ncol, n12 = n1 * n2;
  const int R = 2 * mx + 1, P2 = n2 | 1, plane = R * P2;
  const int Q = PLANE_REG_THREADS / n2;
  const int nzb = (n3 + Q - 1) / Q;
  const int local = blockIdx.x - ka.start[p];
  const int grp = local / nzb, zb = local - grp * nzb;
  const int z0 = zb * Q, nq = min(Q, n3 - z0);
  const int pr0 = grp * PLANE_PAIR_GROUP, pr1 = min(P.npair, pr0 + PLANE_PAIR_GROUP);
  cplx<float>* const S0 = reinterpret_cast<cplx<float>*>(smem_raw);
  cplx<float>* const S1 = S0 + Q * plane;
  float* Vs = reinterpret_cast<float*>(S1 + Q * plane);  // V_eff / N of the CTA's planes
  const int* __restrict__ sidx = P.col_sidx;
  auto wc_of = [&](int pair) {
    return reinterpret_cast<cplx<float>*>(P.Wc) + ((size_t)pair * n3 + z0) * ncol;
  };
  auto scatter = [&](cplx<float>* S, const cplx<float>* wc) {
    for (int q = 0; q < nq; ++q)
      for (int c = threadIdx.x; c < ncol; c += blockDim.x) cp_async8(S + q * plane + sidx[c], wc + q * ncol + c);
    cp_async_commit();
  };
  for (int t = threadIdx.x; t < 2 * Q * plane; t += blockDim.x) S0[t] = mk(0.f, 0.f);
  __syncthreads();
  // the potential (once for the CTA's band pairs) and the first pair's compact columns:
  // asynchronous copies; every later pair's columns land while the previous pair computes
  const float* veff = reinterpret_cast<const float*>(P.veff) + (size_t)z0 * n12;
  for (int t = threadIdx.x; t < nq * n12; t += blockDim.x) cp_async4(Vs + t, veff + t);
  cp_async_commit();
  scatter(S0, wc_of(pr0));
#pragma unroll 1
  for (int pair = pr0; pair < pr1; ++pair) {
    const bool odd = (pair - pr0) & 1;
    cplx<float>* S = odd ? S1 : S0;
    cplx<float>* Sn = odd ? S0 : S1;
    cp_async_wait<0>();
    __syncthreads();
    if (pair + 1 < pr1) scatter(Sn, wc_of(pair + 1));
    // y inverse, x pass, y forward; both y directions through one row-transform body
#pragma unroll 1
    for (int ph = 0; ph < 2; ++ph) {
      for (int l = threadIdx.x; l < nq * R; l += blockDim.x) row_fft_n<MAXN>(n2, S + l * P2, ph == 1);
      __syncthreads();
      if (ph == 1) break;
      for (int l = threadIdx.x; l < nq * n2; l += blockDim.x) {
        const int q = l / n2, i2 = l - q * n2;
        col_vpsi_n<MAXN>(n1, S + q * plane + i2, P2, Vs + q * n12 + i2, n2, mx);
      }
      __syncthreads();
    }
    cplx<float>* wc = wc_of(pair);
    for (int q = 0; q < nq; ++q)
      for (int c = threadIdx.x; c < ncol; c += blockDim.x) wc[q * ncol + c] = S[q * plane + sidx[c]];
    __syncthreads();
    for (int t = threadIdx.x; t < nq * plane; t += blockDim.x) S[t] = mk(0.f, 0.f);  // for pair + 2
  }
}

bool plane_reg_ok(int n1, int n2) {
  return reg_supported(n1) && reg_supported(n2) && n1 <= PLANE_REG_MAXN && n2 <= PLANE_REG_MAXN;
}
int plane_reg_class(int n1, int n2) { return (n1 <= 40 && n2 <= 40) ? 0 : 1; }
int plane_reg_ctas(int n2, int n3, int npair) {
  const int q = PLANE_REG_THREADS / n2;
  return ((npair + PLANE_PAIR_GROUP - 1) / PLANE_PAIR_GROUP) * ((n3 + q - 1) / q);
}
size_t plane_reg_smem(int n1, int n2, int m1max) {
  const size_t q = PLANE_REG_THREADS / n2;
  return 2 * q * (2 * m1max + 1) * (n2 | 1) * sizeof(cplx<float>) + q * n1 * n2 * sizeof(float);
}

void launch_plane_vpsi_reg(const Launch& L, int cls, size_t smem) {
  if (!L.map.total) return;
  if (cls == 0) k_plane_vpsi_reg<40><<<L.map.total, PLANE_REG_THREADS, smem, L.stream>>>(L.ka);
  else k_plane_vpsi_reg<PLANE_REG_MAXN><<<L.map.total, PLANE_REG_THREADS, smem, L.stream>>>(L.ka);
}

bool plane_vpsi_reg_init() { return upload_twiddles(); }

void plane_vpsi_reg_set_smem_limits(size_t bytes) {
  cudaFuncSetAttribute(k_plane_vpsi_reg<40>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_plane_vpsi_reg<PLANE_REG_MAXN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace sgo
