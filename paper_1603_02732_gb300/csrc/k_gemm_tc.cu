// Subspace and projector GEMMs on the 5th-generation tensor cores (tcgen05), fed by TMA,
// mixed path (FP32 operands).  They are the bold products of Algorithm 1 (the subspace
// matrix H(i,j) = <Psi_i|H|Psi_j>, the projection of the search directions against Psi,
// the rotations by the Rayleigh-Ritz eigenvectors) and the Kleinman-Bylander
// contractions <beta_I|psi_n> and sum_I beta_I D_I <beta_I|psi_n> of H.psi.
//
// Precision: 3xTF32.  Each FP32 operand x is split into hi = tf32(x) and lo = tf32(x - hi);
// the TMEM accumulator (FP32) receives hi.hi + hi.lo + lo.hi, a relative error of about
// 2^-21 per product.
//
// Both kernels are warp-specialised pipelines over shared-memory stages:
//   warp 0    one lane issues TMA tile loads (cp.async.bulk.tensor, 128-byte swizzle);
//   warp 1    allocates TMEM; one lane issues tcgen05.mma and commits each stage back;
//   warps 2-5 split each landed FP32 tile in place into hi and a lo copy (at the same
//             swizzled offsets: the split is elementwise), then release it to the MMA lane;
//   epilogue  TMEM -> registers (tcgen05.ld) -> global memory.
// Every wait is bounded (clock64); a timeout sets status[2] of the problem, and the CTA
// still waits (bounded) for its own loads and MMAs in flight, frees TMEM and returns.
//
// TN (C = A^T B, split-K): CTA = (problem, K chunk of kc, TC_KC by default).  A rows (M = 128 TMEM
// lanes) and B rows (N = count rounded up to 16) are K-major tiles of 32 K (128 bytes),
// packed to the operand counts rounded up to 8 rows (one TMA box each), so that short
// operands buy deeper pipelines.  Each CTA writes its FP32 partial as FP64;
// k_gemm_tn_reduce adds the chunks in order.
//
// NN (Y = alpha X M + beta Y): CTA = (problem, tpc tiles of 128 plane waves, NN_TPC by default).  The
// MMA's M is the plane-wave index, K the input row and N the output band.  TMA lands X
// as 32-row x 32-wave boxes (rows of X along K); the converter warps transpose each
// 4 x 4 block while splitting, into a K-major A tile [128 waves][32 rows], the same
// layout as the TN operands.  B = M^T is a K-major image of the small matrix, split into
// hi/lo once per launch by k_nn_image and copied whole into shared memory by one bulk
// copy.  The accumulator is double-buffered in TMEM, so the epilogue of one tile
// overlaps the MMAs of the next.
#include <cuda.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "kernels.h"

namespace sgo {

namespace {

constexpr int TC_K = 32;                      // floats per 128-byte swizzle row
constexpr int TN_MAX_STAGES = 8;
constexpr int TN_SMEM = 225 * 1024;           // dynamic shared memory of the TN kernel
constexpr int TN_PAD = 16 * 1024;             // slack after the last stage (see the TN kernel)
constexpr int TN_THREADS = 192;
constexpr int NN_BOX = 32 * 128;              // one 32-row x 32-wave box (4 KB)
constexpr int NN_STAGE = 3 * 4 * NN_BOX;      // landed boxes (128 waves), hi, lo
constexpr int NN_MAX_STAGES = 4;
constexpr int NN_THREADS = 320;
constexpr int TC_SMEM_BUDGET = 225 * 1024;    // dynamic shared memory per CTA
constexpr long long TC_DRAIN_NS = 2000000000LL;     // bound of the waits for a CTA's own copies and MMAs

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle (descriptor
// version 1): rows of 128 B (32 TF32 along K), 8-row groups 1024 B apart (SBO); the
// leading offset is unused by this layout.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major,
// M x N.
__device__ __forceinline__ uint32_t idesc_tf32(int m, int n) {
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

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
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

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for the phase of the given parity.  Gives up (false) when another role
// has failed (*fail) or after limit_ns nanoseconds of wall time, which marks the CTA
// failed.  fail = null: a drain wait for the CTA's own copies and MMAs, which ignores
// other roles' failures and is bounded by TC_DRAIN_NS whatever the caller's watchdog.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* fail,
                                          long long limit_ns = TC_DRAIN_NS) {
  const unsigned long long t0 = global_ns();
  while (!mbar_test(bar, parity)) {
    if (fail && *fail) return false;
    if ((long long)(global_ns() - t0) > limit_ns) {
      if (fail) *fail = 1;
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(su32(bar))
      : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   su32(dst)),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(su32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Split nunits float4 units in place: hi over the FP32 value, lo into the twin buffer.
__device__ __forceinline__ void split_units(unsigned char* hi, unsigned char* lo, int nunits, int t, int nt) {
  for (int u = t; u < nunits; u += nt) {
    float4 v = reinterpret_cast<float4*>(hi)[u];
    float4 h, l;
    h.x = tf32_round(v.x); l.x = tf32_round(v.x - h.x);
    h.y = tf32_round(v.y); l.y = tf32_round(v.y - h.y);
    h.z = tf32_round(v.z); l.z = tf32_round(v.z - h.z);
    h.w = tf32_round(v.w); l.w = tf32_round(v.w - h.w);
    reinterpret_cast<float4*>(hi)[u] = h;
    reinterpret_cast<float4*>(lo)[u] = l;
  }
}

// Transpose-and-split of one NN stage.  raw: 4 TMA boxes g (waves 32 g .. 32 g + 31), in
// each 32 rows r of 128 B with 16-byte chunk c (waves 4c .. 4c+3) at position c ^ (r % 8).
// Output: K-major tile, wave w at (w/8) 1024 + (w%8) 128, chunk d (rows 4d .. 4d+3) at
// position d ^ (w % 8).  Thread t moves 4 x 4 blocks (box g, wave chunk c = l ^ s, row
// chunk d = l), l = t % 8: the eight lanes of a 16-byte access phase then touch eight
// distinct chunk positions on both the read and the write side.
__device__ __forceinline__ void split_transpose(const unsigned char* raw, unsigned char* hi, unsigned char* lo, int t) {
  const int l = t & 7;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int combo = (t >> 3) + 16 * h;  // 0..31
    const int g = combo & 3, c = l ^ (combo >> 2), d = l;
    float v[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = 4 * d + q;
      const float4 x = *reinterpret_cast<const float4*>(raw + g * NN_BOX + r * 128 + ((c ^ (r & 7)) << 4));
      v[q][0] = x.x; v[q][1] = x.y; v[q][2] = x.z; v[q][3] = x.w;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int w = 32 * g + 4 * c + e;
      const int off = (w >> 3) * 1024 + (w & 7) * 128 + ((d ^ (w & 7)) << 4);
      float4 hv, lv;
      hv.x = tf32_round(v[0][e]); lv.x = tf32_round(v[0][e] - hv.x);
      hv.y = tf32_round(v[1][e]); lv.y = tf32_round(v[1][e] - hv.y);
      hv.z = tf32_round(v[2][e]); lv.z = tf32_round(v[2][e] - hv.z);
      hv.w = tf32_round(v[3][e]); lv.w = tf32_round(v[3][e] - hv.w);
      *reinterpret_cast<float4*>(hi + off) = hv;
      *reinterpret_cast<float4*>(lo + off) = lv;
    }
  }
}

__device__ __forceinline__ int count_tc(const Prob& P, int kind) {
  return kind == OPK_WB ? P.nb : (kind == OPK_B ? P.nproj : 3 * P.nproj);
}

// map slot of an operand: wave buffers by physical index, then B, dB
__device__ __forceinline__ int slot_of(const Prob& P, int kind, int role) {
  return kind == OPK_WB ? P.role[role] : (kind == OPK_B ? NWB : NWB + 1);
}

__device__ __forceinline__ const CUtensorMap* map_of(const CUtensorMap* maps, int p, int slot, int kind) {
  return maps + ((size_t)p * TC_NSLOT + slot) * TC_NMAPKIND + kind;
}

__device__ __forceinline__ unsigned char* align1024(unsigned char* p) {
  return reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~(uintptr_t)1023);
}

__device__ __forceinline__ const double* dense_tc(const Prob& P, int sel) {
  switch (sel) {
    case DD_S: return P.S;
    case DD_HS: return P.Hs;
    case DD_CM: return P.Cm;
    case DD_TM: return P.Tm;
    case DD_PROJ: case DD_PROJ_D: return P.proj;
    default: return P.dproj;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// TN: part[split][i][j] = sum_{k in chunk} A[i][k] B[j][k]
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TN_THREADS, 1)
    k_gemm_tn_tma(KArgs ka, const CUtensorMap* __restrict__ maps, int akind, int arole, int bkind, int brole,
                  double* part_base, size_t part_stride, int kc, long long wait_ns) {
  extern __shared__ unsigned char smem_dyn[];
  __shared__ __align__(8) uint64_t full[TN_MAX_STAGES], conv[TN_MAX_STAGES], empty[TN_MAX_STAGES], done;
  __shared__ uint32_t tmem_base;
  __shared__ int fail_s;
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  unsigned char* smem = align1024(smem_dyn);
  volatile int* fail = &fail_s;
  const int na = count_tc(P, akind), nbv = count_tc(P, bkind);
  const int npad = (nbv + 15) & ~15;
  // stage = [A hi | A lo | B hi | B lo], ra resp. rb rows of 128 B each (multiples of 8
  // rows keep every part on a 1024-byte swizzle-atom boundary).  The MMA reads 128 A rows
  // and npad B rows from the start of a part: rows past ra / rb belong to the next part
  // (or to the TN_PAD slack after the last stage) and reach only output rows >= na or
  // columns >= nbv, which are never stored.
  const int ra = (na + 7) & ~7, rb = (nbv + 7) & ~7;
  const int stage_bytes = 2 * (ra + rb) * 128;
  const int nst = min(TN_MAX_STAGES, (TN_SMEM - 1024 - TN_PAD) / stage_bytes);
  const int split = blockIdx.x - ka.start[p];
  const int k0 = split * kc, k1 = min(P.npw, k0 + kc);
  const int nsteps = (k1 - k0 + TC_K - 1) / TC_K;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)), "r"(128));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    fail_s = 0;
    for (int s = 0; s < nst; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 128);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const int a_lo = ra * 128, b_hi = 2 * ra * 128, b_lo = b_hi + rb * 128;

  if (warp == 0) {
    if (lane == 0) {
      const CUtensorMap* ma = map_of(maps, p, slot_of(P, akind, arole), 0);
      const CUtensorMap* mb = map_of(maps, p, slot_of(P, bkind, brole), 0);
      int issued[TN_MAX_STAGES];
      for (int s = 0; s < TN_MAX_STAGES; ++s) issued[s] = 0;
      for (int it = 0; it < nsteps; ++it) {
        const int s = it % nst, r = it / nst;
        if (r > 0 && !mbar_wait(&empty[s], (uint32_t)((r - 1) & 1), fail, wait_ns)) break;
        unsigned char* st = smem + s * stage_bytes;
        mbar_expect_tx(&full[s], (uint32_t)((ra + rb) * 128));
        tma_load_2d(st, ma, k0 + it * TC_K, 0, &full[s]);
        tma_load_2d(st + b_hi, mb, k0 + it * TC_K, 0, &full[s]);
        issued[s] = r + 1;
      }
      // every load issued has landed before the CTA may exit
      for (int s = 0; s < nst; ++s)
        if (issued[s] > 0) mbar_wait(&full[s], (uint32_t)((issued[s] - 1) & 1), nullptr);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(128, npad);
      for (int it = 0; it < nsteps; ++it) {
        const int s = it % nst, r = it / nst;
        if (!mbar_wait(&conv[s], (uint32_t)(r & 1), fail, wait_ns)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st = su32(smem + s * stage_bytes);
#pragma unroll
        for (int kk = 0; kk < TC_K / 8; ++kk) {
          const uint32_t o = kk * 32;  // K = 8 TF32 = 32 bytes along the swizzled row
          const uint64_t ah = desc_sw128(st + o, 16, 1024), al = desc_sw128(st + a_lo + o, 16, 1024);
          const uint64_t bh = desc_sw128(st + b_hi + o, 16, 1024), bl = desc_sw128(st + b_lo + o, 16, 1024);
          mma_tf32(tmem, ah, bh, idesc, (it > 0 || kk > 0) ? 1u : 0u);
          mma_tf32(tmem, ah, bl, idesc, 1u);
          mma_tf32(tmem, al, bh, idesc, 1u);
        }
        mma_commit(&empty[s]);
      }
      mma_commit(&done);
      mbar_wait(&done, 0, nullptr);
    }
    __syncwarp();
  } else {
    const int t = threadIdx.x - 64;
    for (int it = 0; it < nsteps; ++it) {
      const int s = it % nst, r = it / nst;
      if (!mbar_wait(&full[s], (uint32_t)(r & 1), fail, wait_ns)) break;
      unsigned char* st = smem + s * stage_bytes;
      split_units(st, st + a_lo, ra * 8, t, 128);
      split_units(st + b_hi, st + b_lo, rb * 8, t, 128);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&conv[s]);
    }
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows of C)
    const bool ok = mbar_wait(&done, 0, fail, wait_ns);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (__all_sync(0xffffffffu, ok && !*fail)) {  // tcgen05.ld is warp-collective
      const int quad = warp & 3;
      const int row = quad * 32 + lane;
      double* part = part_base + (size_t)p * part_stride + (size_t)split * na * nbv;
      for (int c0 = 0; c0 < npad; c0 += 16) {
        uint32_t v[16];
        tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, v);
        if (row < na) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (c0 + j < nbv) part[(size_t)row * nbv + c0 + j] = (double)__uint_as_float(v[j]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && fail_s) atomicExch(&P.status[2], 1);
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
}

// ---------------------------------------------------------------------------
// NN image: the B operand of the NN GEMM, M^T as K-major 128-byte-swizzled tiles, hi
// then lo.  Element (j, i) (output band j < npad, input row i < kpad) holds M[i][j]
// (times D_I for DD_PROJ_D), zero in the padding.  Atom column q = i / 32 starts at
// q npad 128 bytes; in it row j sits at (j/8) 1024 + (j%8) 128 and the 16-byte chunk
// c = (i%32)/4 at position c ^ (j%8).  CTA per problem.
// ---------------------------------------------------------------------------
__global__ void k_nn_image(KArgs ka, int akind, int msel, float* img_base, size_t img_stride) {
  const int p = blockIdx.x;
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int nin = count_tc(P, akind), nb = P.nb;
  const int npad = (nb + 15) & ~15, kpad = (nin + 31) & ~31;
  const double* M = dense_tc(P, msel);
  unsigned char* hi = reinterpret_cast<unsigned char*>(img_base + (size_t)p * img_stride);
  unsigned char* lo = hi + (size_t)npad * kpad * 4;
  for (int e = threadIdx.x; e < npad * kpad; e += blockDim.x) {
    const int j = e / kpad, i = e - j * kpad;
    float v = 0.f;
    if (i < nin && j < nb) {
      double m = M[(size_t)i * nb + j];
      if (msel == DD_PROJ_D) m *= P.pj_d[i];
      v = (float)m;
    }
    const float h = tf32_round(v), l = tf32_round(v - h);
    const int q = i >> 5, c = (i & 31) >> 2;
    const size_t off = (size_t)q * npad * 128 + (size_t)(j >> 3) * 1024 + (j & 7) * 128 + ((c ^ (j & 7)) << 4) +
                       (i & 3) * 4;
    *reinterpret_cast<float*>(hi + off) = h;
    *reinterpret_cast<float*>(lo + off) = l;
  }
}

// ---------------------------------------------------------------------------
// NN: Y[j][k] = alpha sum_i X[i][k] M[i][j] + beta Y[j][k], k over this CTA's tiles.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NN_THREADS, 1)
    k_gemm_nn_tma(KArgs ka, const CUtensorMap* __restrict__ maps, const float* __restrict__ img_base,
                  size_t img_stride, int img_max, int nstages, int akind, RolePairs rp, float alpha,
                  float beta, int tpc, long long wait_ns) {
  const int arole = rp.a[blockIdx.y], yrole = rp.y[blockIdx.y];
  extern __shared__ unsigned char smem_dyn[];
  __shared__ __align__(8) uint64_t full[NN_MAX_STAGES], conv[NN_MAX_STAGES], empty[NN_MAX_STAGES], tfull[2],
      tempty[2], imgbar, done;
  __shared__ uint32_t tmem_base;
  __shared__ int fail_s;
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  unsigned char* smem = align1024(smem_dyn);
  unsigned char* stages = smem + img_max;
  volatile int* fail = &fail_s;
  const int nin = count_tc(P, akind), nb = P.nb, npw = P.npw;
  const int npad = (nb + 15) & ~15, kpad = (nin + 31) & ~31, nkc = kpad / 32;
  const int img_half = npad * kpad * 4;
  const int ntile = (npw + 127) / 128;
  const int t0 = (blockIdx.x - ka.start[p]) * tpc, t1 = min(ntile, t0 + tpc);
  const int ntl = t1 - t0, niter = ntl * nkc;
  const uint32_t tcols = npad <= 64 ? 128u : 256u;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    fail_s = 0;
    for (int s = 0; s < nstages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 128);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 128);
    }
    mbar_init(&imgbar, 1);
    mbar_init(&done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      mbar_expect_tx(&imgbar, (uint32_t)(2 * img_half));
      bulk_load(smem, img_base + (size_t)p * img_stride, (uint32_t)(2 * img_half), &imgbar);
      const CUtensorMap* mx = map_of(maps, p, slot_of(P, akind, arole), 1);
      int issued[NN_MAX_STAGES];
      for (int s = 0; s < NN_MAX_STAGES; ++s) issued[s] = 0;
      for (int it = 0; it < niter; ++it) {
        const int s = it % nstages, r = it / nstages;
        const int tl = it / nkc, kc = it - tl * nkc;
        if (r > 0 && !mbar_wait(&empty[s], (uint32_t)((r - 1) & 1), fail, wait_ns)) break;
        unsigned char* st = stages + s * NN_STAGE;
        mbar_expect_tx(&full[s], 4 * NN_BOX);
        const int x0 = (t0 + tl) * 128;
#pragma unroll
        for (int g = 0; g < 4; ++g) tma_load_2d(st + g * NN_BOX, mx, x0 + 32 * g, 32 * kc, &full[s]);
        issued[s] = r + 1;
      }
      // every load issued has landed before the CTA may exit
      mbar_wait(&imgbar, 0, nullptr);
      for (int s = 0; s < nstages; ++s)
        if (issued[s] > 0) mbar_wait(&full[s], (uint32_t)((issued[s] - 1) & 1), nullptr);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(128, npad);
      const uint32_t ih = su32(smem), il = ih + img_half;
      bool ok = mbar_wait(&imgbar, 0, fail, wait_ns);
      for (int tl = 0; ok && tl < ntl; ++tl) {
        const int b = tl & 1, use = tl >> 1;
        if (use > 0 && !mbar_wait(&tempty[b], (uint32_t)((use - 1) & 1), fail, wait_ns)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(b * npad);
        for (int kc = 0; kc < nkc; ++kc) {
          const int it = tl * nkc + kc;
          const int s = it % nstages, r = it / nstages;
          if (!mbar_wait(&conv[s], (uint32_t)(r & 1), fail, wait_ns)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sh = su32(stages + s * NN_STAGE) + 4 * NN_BOX, sl = sh + 4 * NN_BOX;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            if (kc * 32 + kk * 8 >= nin) break;  // K steps wholly in the zero padding
            // A: K-major tile [128 waves][32 rows], K offset kk * 8 TF32 = 32 B
            const uint64_t ah = desc_sw128(sh + kk * 32, 16, 1024);
            const uint64_t al = desc_sw128(sl + kk * 32, 16, 1024);
            // B: K-major image, atom column kc, K offset kk * 8 TF32 = 32 B
            const uint32_t bo = (uint32_t)(kc * npad * 128 + kk * 32);
            const uint64_t bh = desc_sw128(ih + bo, 16, 1024), bl = desc_sw128(il + bo, 16, 1024);
            mma_tf32(d, ah, bh, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
            mma_tf32(d, ah, bl, idesc, 1u);
            mma_tf32(d, al, bh, idesc, 1u);
          }
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        mma_commit(&tfull[b]);
      }
      mma_commit(&done);
      mbar_wait(&done, 0, nullptr);
    }
    __syncwarp();
  } else if (warp < 6) {
    const int t = threadIdx.x - 64;
    for (int it = 0; it < niter; ++it) {
      const int s = it % nstages, r = it / nstages;
      if (!mbar_wait(&full[s], (uint32_t)(r & 1), fail, wait_ns)) break;
      unsigned char* st = stages + s * NN_STAGE;
      split_transpose(st, st + 4 * NN_BOX, st + 8 * NN_BOX, t);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&conv[s]);
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 = plane waves of the tile
    const int quad = warp & 3;
    float* Y = reinterpret_cast<float*>(P.wb[P.role[yrole]]);
    const int ld = P.ld;
    for (int tl = 0; tl < ntl; ++tl) {
      const int b = tl & 1, use = tl >> 1;
      const bool ok = mbar_wait(&tfull[b], (uint32_t)(use & 1), fail, wait_ns);
      if (!__all_sync(0xffffffffu, ok)) break;  // tcgen05.ld is warp-collective
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int k = (t0 + tl) * 128 + quad * 32 + lane;
      for (int c0 = 0; c0 < npad; c0 += 16) {
        // the 16 reads of Y go out together, before any store of this chunk
        float yv[16];
#pragma unroll
        for (int j = 0; j < 16; ++j)
          yv[j] = (beta != 0.f && k < npw && c0 + j < nb) ? Y[(size_t)(c0 + j) * ld + k] : 0.f;
        uint32_t v[16];
        tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(b * npad + c0), v);
        if (k < npw) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (c0 + j < nb) Y[(size_t)(c0 + j) * ld + k] = alpha * __uint_as_float(v[j]) + beta * yv[j];
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&tempty[b]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && fail_s) atomicExch(&P.status[2], 1);
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(f);
  });
  return fn;
}

// 2D FP32 map over rows x cols (row stride ld floats), box 32 x box_rows, 128-byte
// swizzle, zero fill outside the tensor.
bool encode_2d(CUtensorMap* m, const void* base, int cols, int rows, int ld, int box_rows) {
  EncodeTiled fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled unavailable from the driver");
    return false;
  }
  if (!base || cols < 1 || rows < 1 || (reinterpret_cast<uintptr_t>(base) & 15) || ((size_t)ld * 4) % 16 ||
      ld < cols) {
    set_error("tensor map: base, extent or stride not 16-byte compatible");
    return false;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  const cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return false;
  }
  return true;
}

}  // namespace

size_t tc_map_bytes() { return sizeof(CUtensorMap); }

bool tc_encode_maps(const Prob& d, void* host_maps) {
  CUtensorMap* m = reinterpret_cast<CUtensorMap*>(host_maps);
  for (int s = 0; s < TC_NSLOT; ++s) {
    const void* base = s < NWB ? d.wb[s] : (s == NWB ? d.B : d.dB);
    const int rows = s < NWB ? d.nb : (s == NWB ? d.nproj : 3 * d.nproj);
    if (!encode_2d(m + s * TC_NMAPKIND + 0, base, d.npw, rows, d.ld, std::min(128, (rows + 7) & ~7))) return false;
    if (!encode_2d(m + s * TC_NMAPKIND + 1, base, d.npw, rows, d.ld, 32)) return false;
  }
  return true;
}

int nn_tc_image_bytes(int nin, int nb) { return 2 * ((nb + 15) & ~15) * ((nin + 31) & ~31) * 4; }

int nn_tc_stages(int img_bytes) {
  const int img = (img_bytes + 1023) & ~1023;
  const int s = (TC_SMEM_BUDGET - 1024 - img) / NN_STAGE;
  return s < NN_MAX_STAGES ? s : NN_MAX_STAGES;
}

void launch_gemm_tn_tc(const Launch& L, const void* maps, int akind, int arole, int bkind, int brole, double* part,
                       size_t stride, int kc) {
  if (!L.map.total) return;
  k_gemm_tn_tma<<<L.map.total, TN_THREADS, TN_SMEM, L.stream>>>(
      L.ka, reinterpret_cast<const CUtensorMap*>(maps), akind, arole, bkind, brole, part, stride, kc, L.wait_ns);
}

void launch_nn_image(const Launch& Lprob, int akind, int msel, float* img, size_t img_stride) {
  k_nn_image<<<Lprob.ka.nprob, 256, 0, Lprob.stream>>>(Lprob.ka, akind, msel, img, img_stride);
}

void launch_gemm_nn_tc(const Launch& L, const void* maps, const float* img, size_t img_stride, int img_max,
                       int akind, const RolePairs& rp, double alpha, double beta, int tpc) {
  if (!L.map.total || rp.n < 1) return;
  const int img_al = (img_max + 1023) & ~1023;
  const int ns = nn_tc_stages(img_max);
  k_gemm_nn_tma<<<dim3(L.map.total, rp.n), NN_THREADS, 1024 + img_al + ns * NN_STAGE, L.stream>>>(
      L.ka, reinterpret_cast<const CUtensorMap*>(maps), img, img_stride, img_al, ns, akind, rp, (float)alpha,
      (float)beta, tpc, L.wait_ns);
}

void gemm_tc_set_smem_limits() {
  cudaFuncSetAttribute(k_gemm_tn_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, TN_SMEM);
  cudaFuncSetAttribute(k_gemm_nn_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_BUDGET);
}

}  // namespace sgo
