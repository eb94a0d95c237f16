// Register-FFT density pass (mixed path).  See fft_reg.cuh for the line transforms.
#include "fft_reg.cuh"
#include "kernels.h"

namespace sgo {

namespace {

// Column of the density pass: x inverse of the occupied rows, then acc[e] (FP64, stride
// astride) += fa Re^2 + fb Im^2 for every x row e.
template <int N>
__device__ __forceinline__ void col_density(const cplx<float>* col, int stride, double* acc, int astride, int mx,
                                            float fa, float fb) {
  const int R = 2 * mx + 1;
  cplx<float> x[N];
#pragma unroll
  for (int e = 0; e < N; ++e) {
    const bool lo = e <= mx, hi = e >= N - mx;
    x[e] = (lo || hi) ? col[(lo ? e : e - N + R) * stride] : mk(0.f, 0.f);
  }
  reg_fft<float, N, 1>(x, twf<N>());
#pragma unroll
  for (int p = 0; p < N; ++p) {
    const int e = dif_freq<N>(p);
    acc[e * astride] += (double)(fa * x[p].x * x[p].x + fb * x[p].y * x[p].y);
  }
}

template <int MAXN>
__device__ __forceinline__ void col_density_n(int n, const cplx<float>* col, int stride, double* acc, int astride,
                                              int mx, float fa, float fb) {
  switch (n) {
#define SGO_COL(N)                                                                \
  case N:                                                                         \
    if constexpr (N <= MAXN) col_density<N>(col, stride, acc, astride, mx, fa, fb); \
    break;
    SGO_COL(10) SGO_COL(12) SGO_COL(15) SGO_COL(16) SGO_COL(18) SGO_COL(20) SGO_COL(24) SGO_COL(25) SGO_COL(27)
    SGO_COL(30) SGO_COL(32) SGO_COL(36) SGO_COL(40) SGO_COL(45) SGO_COL(48) SGO_COL(50) SGO_COL(54) SGO_COL(60)
    SGO_COL(64) SGO_COL(72)
#undef SGO_COL
    default: break;
  }
}

}  // namespace
// Register-FFT density pass (mixed path): CTA = (problem, block of Q z-planes), looping
// over the band pairs with non-zero occupation; the same compact-row layout and passes
// as the H.psi plane kernel up to the x inverse, after which each column adds
// f_a Re^2 + f_b Im^2 (FP32 products) into FP64 accumulators of its planes.
template <int MAXN>
__global__ void __launch_bounds__(PLANE_REG_THREADS, 1) k_plane_density_reg(KArgs ka, const double* occ_override) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int n1 = P.n1, n2 = P.n2, n3 = P.n3, mx = P.m1max, ncol = P.ncol, n12 = n1 * n2;
  const int R = 2 * mx + 1, P2 = n2 | 1, plane = R * P2;
  const int Q = PLANE_REG_THREADS / n2;
  const int z0 = (blockIdx.x - ka.start[p]) * Q, nq = min(Q, n3 - z0);
  double* acc = reinterpret_cast<double*>(smem_raw);               // [Q][n1][n2]
  cplx<float>* S = reinterpret_cast<cplx<float>*>(acc + Q * n12);  // [Q][R][P2]
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
    for (int l = threadIdx.x; l < nq * R; l += blockDim.x) row_fft_n<MAXN>(n2, S + l * P2, false);
    __syncthreads();
    for (int l = threadIdx.x; l < nq * n2; l += blockDim.x) {
      const int q = l / n2, i2 = l - q * n2;
      col_density_n<MAXN>(n1, S + q * plane + i2, P2, acc + q * n12 + i2, n2, mx, (float)fa, (float)fb);
    }
    __syncthreads();
  }
  __syncthreads();
  const double io = 1.0 / P.omega;
  double* rho = P.rho_out + (size_t)z0 * n12;
  for (int t = threadIdx.x; t < nq * n12; t += blockDim.x) rho[t] = acc[t] * io;
}

size_t plane_density_reg_smem(int n1, int n2, int m1max) {
  const size_t q = PLANE_REG_THREADS / n2;
  return q * n1 * n2 * sizeof(double) + q * (2 * m1max + 1) * (n2 | 1) * sizeof(cplx<float>);
}
int plane_density_reg_ctas(int n2, int n3) {
  const int q = PLANE_REG_THREADS / n2;
  return (n3 + q - 1) / q;
}
void launch_plane_density_reg(const Launch& L, int cls, size_t smem, const double* occ_override) {
  if (!L.map.total) return;
  if (cls == 0) k_plane_density_reg<40><<<L.map.total, PLANE_REG_THREADS, smem, L.stream>>>(L.ka, occ_override);
  else k_plane_density_reg<PLANE_REG_MAXN><<<L.map.total, PLANE_REG_THREADS, smem, L.stream>>>(L.ka, occ_override);
}

bool plane_density_reg_init() { return upload_twiddles(); }

void plane_density_reg_set_smem_limits(size_t bytes) {
  cudaFuncSetAttribute(k_plane_density_reg<40>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_plane_density_reg<PLANE_REG_MAXN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace sgo
