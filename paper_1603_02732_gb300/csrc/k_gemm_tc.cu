// Subspace and projector overlaps C = A^T B on the 5th-generation tensor cores (tcgen05),
// mixed path (FP32 operands).  The products are the bold steps of Algorithm 1 (lines 2, 12,
// 14, 15: H(i,j) = <Psi_i|H|Psi_j>, overlaps, projection coefficients) and <beta_I|psi_n>.
//
// Precision: 3xTF32.  Each FP32 operand x is split into hi = tf32(x) and lo = tf32(x - hi);
// the accumulator in TMEM (FP32) receives hi.hi + hi.lo + lo.hi, a relative error of about
// 2^-21 per product; each CTA's FP32 partial is written out as FP64 and the partials of all
// K chunks are added in fixed order by k_gemm_tn_reduce (FP64).
//
// CTA = (member, K chunk of TC_KC).  A tile: 128 rows (vectors of A, M dimension) x 32 K;
// B tile: N rows (vectors of B, N = count rounded up to 16) x 32 K; both K-major in the
// canonical no-swizzle layout (8-row x 16-byte core matrices, K-adjacent cores 128 B apart,
// 8-row groups 1024 B apart).  Two stages: threads stage chunk s+1 (global -> split ->
// shared) while the tensor core runs chunk s.  One thread issues the MMAs and commits them
// to a per-stage mbarrier; every wait is bounded (clock) and reports a timeout in status[2].
#include <stdint.h>

#include "kernels.h"

namespace sgo {

namespace {

constexpr int TC_M = 128;
constexpr int TC_K = 32;                       // K per stage
constexpr int TC_STAGE_A = TC_M * TC_K * 4;    // bytes of one A split (16 KB)
constexpr int TC_STAGE_B = 128 * TC_K * 4;     // bytes of one B split (N <= 128)
constexpr int TC_STAGE = 2 * TC_STAGE_A + 2 * TC_STAGE_B;  // hi, lo of A and B
constexpr long long TC_WAIT_CYCLES = 4000000000LL;          // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// byte offset of element (row, k) in a canonical no-swizzle K-major tile (32-bit elements)
__device__ __forceinline__ uint32_t kmajor_off(int row, int k) {
  return (uint32_t)((k >> 2) * 128 + (row >> 3) * 1024 + (row & 7) * 16 + (k & 3) * 4);
}

// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte offsets,
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::tf32: FP32 accumulate, TF32 A and B, both K-major
__host__ __device__ __forceinline__ uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_test(bar, parity)) {
    if (clock64() - t0 > TC_WAIT_CYCLES) return false;
  }
  return true;
}

template <typename T>
__device__ __forceinline__ const T* opnd_tc(const Prob& P, int kind, int role) {
  if (kind == OPK_WB) return wbuf<T>(P, role);
  if (kind == OPK_B) return reinterpret_cast<const T*>(P.B);
  return reinterpret_cast<const T*>(P.dB);
}
__device__ __forceinline__ int count_tc(const Prob& P, int kind) {
  return kind == OPK_WB ? P.nb : (kind == OPK_B ? P.natom : 3 * P.natom);
}

// Stage one 32-wide K chunk of `rows` vectors (row r = vector v0 + r) as hi/lo splits.
// Lane layout: a warp covers 8 rows x 16 k (float4 per thread), quarter-warps write
// contiguous 128-byte core-matrix rows.
__device__ __forceinline__ void stage_tile(const float* __restrict__ src, int ld, int nvec, int v0, int kb, int k1,
                                           unsigned char* hi, unsigned char* lo, int rows) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r8 = lane & 7, k4 = lane >> 3;  // k4 in 0..3
  const int nunits = (rows >> 3) * 2;       // (8-row group, 16-k half) units; rows % 8 == 0
  for (int u = warp; u < nunits; u += blockDim.x >> 5) {
    const int row = (u >> 1) * 8 + r8;
    const int k = (u & 1) * 16 + k4 * 4;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    const int vi = v0 + row, kg = kb + k;
    if (vi < nvec) {
      const float* p = src + (size_t)vi * ld + kg;
      if (kg + 3 < k1 && ((reinterpret_cast<uintptr_t>(p) & 15) == 0)) {
        float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = (kg + j < k1) ? p[j] : 0.f;
      }
    }
    float4 h, l;
    h.x = tf32_round(v[0]); l.x = tf32_round(v[0] - h.x);
    h.y = tf32_round(v[1]); l.y = tf32_round(v[1] - h.y);
    h.z = tf32_round(v[2]); l.z = tf32_round(v[2] - h.z);
    h.w = tf32_round(v[3]); l.w = tf32_round(v[3] - h.w);
    const uint32_t off = kmajor_off(row, k);
    *reinterpret_cast<float4*>(hi + off) = h;
    *reinterpret_cast<float4*>(lo + off) = l;
  }
}

}  // namespace

__global__ void __launch_bounds__(256, 1) k_gemm_tn_tc(KArgs ka, int akind, int arole, int bkind, int brole,
                                                      double* part_base, size_t part_stride) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[3];
  __shared__ uint32_t tmem_base;
  __shared__ int fail;
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int na = count_tc(P, akind), nbv = count_tc(P, bkind);
  const int npad = (nbv + 15) & ~15;
  const int split = blockIdx.x - ka.start[p];
  const int k0 = split * TC_KC, k1 = min(P.npw, k0 + TC_KC);
  const float* A = opnd_tc<float>(P, akind, arole);
  const float* Bm = opnd_tc<float>(P, bkind, brole);
  const int warp = threadIdx.x >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)), "r"(128));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    fail = 0;
    for (int i = 0; i < 3; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&bar[i])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t dtm = tmem_base;
  const uint32_t idesc = idesc_tf32(TC_M, npad);
  const int nsteps = (k1 - k0 + TC_K - 1) / TC_K;
  for (int it = 0; it < nsteps; ++it) {
    const int s = it & 1;
    unsigned char* st = smem_raw + s * TC_STAGE;
    unsigned char* ahi = st;
    unsigned char* alo = st + TC_STAGE_A;
    unsigned char* bhi = st + 2 * TC_STAGE_A;
    unsigned char* blo = bhi + TC_STAGE_B;
    if (it >= 2) {
      // the MMAs that read this stage two chunks ago must have completed
      if (!mbar_wait(&bar[s], (uint32_t)(((it >> 1) - 1) & 1))) fail = 1;
      __syncthreads();
      if (fail) break;
    }
    const int kb = k0 + it * TC_K;
    // Only the rows that exist are staged: output (i, j) reads row i of A and row j of B
    // alone, so whatever the rows beyond the counts hold reaches only discarded outputs.
    stage_tile(A, P.ld, na, 0, kb, k1, ahi, alo, (na + 7) & ~7);
    stage_tile(Bm, P.ld, nbv, 0, kb, k1, bhi, blo, (nbv + 7) & ~7);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < TC_K / 8; ++kk) {
        const uint32_t o = kk * 256;  // two K-adjacent core matrices per MMA (K = 8)
        const uint64_t dah = smem_desc(su32(ahi) + o, 128, 1024), dal = smem_desc(su32(alo) + o, 128, 1024);
        const uint64_t dbh = smem_desc(su32(bhi) + o, 128, 1024), dbl = smem_desc(su32(blo) + o, 128, 1024);
        mma_tf32(dtm, dah, dbh, idesc, (it > 0 || kk > 0) ? 1u : 0u);
        mma_tf32(dtm, dah, dbl, idesc, 1u);
        mma_tf32(dtm, dal, dbh, idesc, 1u);
      }
      mma_commit(&bar[s]);
    }
  }
  // wait for every MMA of this CTA (a final commit tracks all earlier ones)
  if (threadIdx.x == 0) mma_commit(&bar[2]);
  if (!mbar_wait(&bar[2], 0)) fail = 1;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (!fail) {
    // TMEM -> registers -> FP64 partials.  Warp w reads lanes 32 (w%4) .. +31 (rows of C)
    // and column half w/4.
    const int quad = warp & 3, half = warp >> 2;
    const int row = quad * 32 + (threadIdx.x & 31);
    double* part = part_base + (size_t)p * part_stride + (size_t)split * na * nbv;
    const int c_begin = half * 64, c_end = min(npad, c_begin + 64);
    for (int c0 = c_begin; c0 < c_end; c0 += 16) {
      uint32_t r[16];
      const uint32_t taddr = dtm + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < na) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int col = c0 + j;
          if (col < nbv) part[(size_t)row * nbv + col] = (double)__uint_as_float(r[j]);
        }
      }
    }
  } else if (threadIdx.x == 0) {
    atomicExch(&P.status[2], 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(dtm), "r"(128));
}

void launch_gemm_tn_tc(const Launch& L, int akind, int arole, int bkind, int brole, double* part, size_t stride) {
  if (!L.map.total) return;
  k_gemm_tn_tc<<<L.map.total, 256, 2 * TC_STAGE, L.stream>>>(L.ka, akind, arole, bkind, brole, part, stride);
}

void gemm_tc_set_smem_limits() {
  cudaFuncSetAttribute(k_gemm_tn_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * TC_STAGE);
}

}  // namespace sgo
