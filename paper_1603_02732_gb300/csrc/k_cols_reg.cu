// Register-FFT z-column passes of H.psi and of the density (mixed path; the line
// transforms are in fft_reg.cuh).  CTA = (problem, band pair, chunk of ZREG_CP column
// pairs), one thread per compact column, the whole z line in registers.
//   sphere -> columns: the chunk's half-sphere entries are scattered into shared lines
//     (psi_a + i psi_b at G and its conjugate partner at -G, the band pair packing of
//     the plane kernels), then each thread takes the inverse z transform of its line
//     and writes it straight to Wc[pair][z][col] (consecutive threads, consecutive
//     columns).
//   columns -> sphere: each thread reads its column of Wc, takes the forward z
//     transform into a shared line, and the entries are gathered back with the band
//     separation (V psi_a)(G) = (F(G) + F(-G)^*)/2, (V psi_b)(G) = (F(G) - F(-G)^*)/(2i)
//     plus the kinetic term.
// Lines are padded to an odd length (n3 | 1): a thread per line touches distinct banks.
#include "fft_reg.cuh"
#include "kernels.h"

namespace sgo {

namespace {

// Column pair chunk [cp0, cp1) -> compact columns [col0, col1).
__device__ __forceinline__ void zreg_cols(int cp0, int cp1, int* col0, int* col1) {
  *col0 = cp0 == 0 ? 0 : 2 * cp0 - 1;
  *col1 = 2 * cp1 - 1;
}

template <int N>
__device__ __forceinline__ void zline_inv(const cplx<float>* line, cplx<float>* out, size_t zstride) {
  cplx<float> x[N];
#pragma unroll
  for (int e = 0; e < N; ++e) x[e] = line[e];
  reg_fft<float, N, 1>(x, twf<N>());
#pragma unroll
  for (int p = 0; p < N; ++p) out[(size_t)dif_freq<N>(p) * zstride] = x[p];
}

template <int N>
__device__ __forceinline__ void zline_fwd(const cplx<float>* in, size_t zstride, cplx<float>* line) {
  cplx<float> x[N];
#pragma unroll
  for (int e = 0; e < N; ++e) x[e] = in[(size_t)e * zstride];
  reg_fft<float, N, -1>(x, twf<N>());
#pragma unroll
  for (int p = 0; p < N; ++p) line[dif_freq<N>(p)] = x[p];
}

#define SGO_ZSIZES(X)                                                                                      \
  X(10) X(12) X(15) X(16) X(18) X(20) X(24) X(25) X(27) X(30) X(32) X(36) X(40) X(45) X(48) X(50) X(54) \
  X(60) X(64) X(72)

template <int MAXN>
__device__ __forceinline__ void zline_inv_n(int n, const cplx<float>* line, cplx<float>* out, size_t zstride) {
  switch (n) {
#define SGO_CASE(N)                                        \
  case N:                                                  \
    if constexpr (N <= MAXN) zline_inv<N>(line, out, zstride); \
    break;
    SGO_ZSIZES(SGO_CASE)
#undef SGO_CASE
    default: break;
  }
}

template <int MAXN>
__device__ __forceinline__ void zline_fwd_n(int n, const cplx<float>* in, size_t zstride, cplx<float>* line) {
  switch (n) {
#define SGO_CASE(N)                                        \
  case N:                                                  \
    if constexpr (N <= MAXN) zline_fwd<N>(in, zstride, line); \
    break;
    SGO_ZSIZES(SGO_CASE)
#undef SGO_CASE
    default: break;
  }
}

}  // namespace

template <int MAXN>
__global__ void __launch_bounds__(ZREG_THREADS) k_wave_to_cols_reg(KArgs ka, int src) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int nchunk = (P.ncp + ZREG_CP - 1) / ZREG_CP;
  const int local = blockIdx.x - ka.start[p];
  const int pair = local / nchunk, chunk = local - pair * nchunk;
  const int n3 = P.n3, L3 = n3 | 1;
  const int cp0 = chunk * ZREG_CP, cp1 = min(cp0 + ZREG_CP, P.ncp);
  int col0, col1;
  zreg_cols(cp0, cp1, &col0, &col1);
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
  if (threadIdx.x < ncl) {
    cplx<float>* wc = reinterpret_cast<cplx<float>*>(P.Wc) + (size_t)pair * n3 * P.ncol + col0 + threadIdx.x;
    zline_inv_n<MAXN>(n3, lines + threadIdx.x * L3, wc, (size_t)P.ncol);
  }
}

template <int MAXN>
__global__ void __launch_bounds__(ZREG_THREADS) k_cols_to_wave_reg(KArgs ka, int src, int dst) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int nchunk = (P.ncp + ZREG_CP - 1) / ZREG_CP;
  const int local = blockIdx.x - ka.start[p];
  const int pair = local / nchunk, chunk = local - pair * nchunk;
  const int n3 = P.n3, L3 = n3 | 1;
  const int cp0 = chunk * ZREG_CP, cp1 = min(cp0 + ZREG_CP, P.ncp);
  int col0, col1;
  zreg_cols(cp0, cp1, &col0, &col1);
  const int ncl = col1 - col0;
  cplx<float>* lines = reinterpret_cast<cplx<float>*>(smem_raw);
  if (threadIdx.x < ncl) {
    const cplx<float>* wc =
        reinterpret_cast<const cplx<float>*>(P.Wc) + (size_t)pair * n3 * P.ncol + col0 + threadIdx.x;
    zline_fwd_n<MAXN>(n3, wc, (size_t)P.ncol, lines + threadIdx.x * L3);
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
    // a: (fp + conj fm)/2 ; b: (fp - conj fm)/(2i)
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

int zreg_class(int n3) { return n3 <= 40 ? 0 : 1; }
bool zreg_ok(int n3) { return reg_supported(n3) && n3 <= PLANE_REG_MAXN; }
int zreg_ctas(int ncp, int npair) { return npair * ((ncp + ZREG_CP - 1) / ZREG_CP); }
size_t zreg_smem(int n3) { return (size_t)2 * ZREG_CP * (n3 | 1) * sizeof(cplx<float>); }

void launch_wave_to_cols_reg(const Launch& L, int cls, size_t smem, int src) {
  if (!L.map.total) return;
  if (cls == 0) k_wave_to_cols_reg<40><<<L.map.total, ZREG_THREADS, smem, L.stream>>>(L.ka, src);
  else k_wave_to_cols_reg<PLANE_REG_MAXN><<<L.map.total, ZREG_THREADS, smem, L.stream>>>(L.ka, src);
}

void launch_cols_to_wave_reg(const Launch& L, int cls, size_t smem, int src, int dst) {
  if (!L.map.total) return;
  if (cls == 0) k_cols_to_wave_reg<40><<<L.map.total, ZREG_THREADS, smem, L.stream>>>(L.ka, src, dst);
  else k_cols_to_wave_reg<PLANE_REG_MAXN><<<L.map.total, ZREG_THREADS, smem, L.stream>>>(L.ka, src, dst);
}

bool zreg_init() { return upload_twiddles(); }

void zreg_set_smem_limits(size_t bytes) {
  cudaFuncSetAttribute(k_wave_to_cols_reg<40>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_wave_to_cols_reg<PLANE_REG_MAXN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_cols_to_wave_reg<40>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_cols_to_wave_reg<PLANE_REG_MAXN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace sgo
