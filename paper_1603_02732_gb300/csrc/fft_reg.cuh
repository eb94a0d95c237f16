// Register-resident FFTs of compile-time length for the plane passes (device side).
//
// One thread transforms one whole line held in registers: an in-place mixed-radix
// decimation-in-frequency transform (Gentleman & Sande, 1966) with radices 2, 3, 4, 5.
// For a block of length L = R M at offset off, every n1 < M takes the radix-R DFT of
// x[off + n1 + M r] (r < R), multiplies output k2 by W_L^(n1 k2) (W_L = exp(sign 2 pi i / L))
// and writes it back to x[off + n1 + M k2]; each block x[off + M k2 ...] of length M then
// recurses with the next radix.  The result is in digit-reversed order: position p holds
// frequency dif_freq<N>(p), a compile-time map, so reordering costs no instruction.  All
// indices and twiddle offsets are compile-time constants after unrolling: the line never
// leaves registers and every twiddle is a constant-bank operand.  No scaling.
#pragma once

#include <cmath>
#include <mutex>
#include <vector>

#include "fft.cuh"

namespace sgo {

// Line lengths with a register transform (all other lengths use the shared-memory engine).
constexpr int kRegSizes[] = {10, 12, 15, 16, 18, 20, 24, 25, 27, 30, 32, 36, 40, 45, 48, 50, 54, 60, 64, 72};
constexpr int kRegCount = sizeof(kRegSizes) / sizeof(int);
// Lengths N = 2M transformed by a pair of lanes (M of the single-thread lengths each).
constexpr int kPairSizes[] = {96, 100, 108, 120, 128};
constexpr int kPairCount = sizeof(kPairSizes) / sizeof(int);

// twiddle tables: every single-thread length, then every pair length
constexpr int tw_size(int i) { return i < kRegCount ? kRegSizes[i] : kPairSizes[i - kRegCount]; }
constexpr int reg_table_offset(int n) {
  int o = 0;
  for (int i = 0; i < kRegCount + kPairCount; ++i) {
    if (tw_size(i) == n) return o;
    o += tw_size(i);
  }
  return -1;
}
constexpr int reg_table_total() {
  int o = 0;
  for (int i = 0; i < kRegCount + kPairCount; ++i) o += tw_size(i);
  return o;
}
constexpr bool reg_supported(int n) {
  for (int i = 0; i < kRegCount; ++i)
    if (kRegSizes[i] == n) return true;
  return false;
}
constexpr bool pair_supported(int n) {
  for (int i = 0; i < kPairCount; ++i)
    if (kPairSizes[i] == n) return true;
  return false;
}

// radices, outermost stage first (packed one per 4 bits, stage 0 lowest)
constexpr unsigned reg_plan(int n) {
  switch (n) {
    case 10: return 0x52u;  // 2 x 5
    case 12: return 0x34u;  // 4 x 3
    case 15: return 0x53u;  // 3 x 5
    case 16: return 0x44u;  // 4 x 4
    case 18: return 0x332u;  // 2 x 3 x 3
    case 20: return 0x54u;  // 4 x 5
    case 24: return 0x324u;  // 4 x 2 x 3
    case 25: return 0x55u;  // 5 x 5
    case 27: return 0x333u;  // 3 x 3 x 3
    case 30: return 0x532u;  // 2 x 3 x 5
    case 32: return 0x244u;  // 4 x 4 x 2
    case 36: return 0x334u;  // 4 x 3 x 3
    case 40: return 0x524u;  // 4 x 2 x 5
    case 45: return 0x533u;  // 3 x 3 x 5
    case 48: return 0x344u;  // 4 x 4 x 3
    case 50: return 0x552u;  // 2 x 5 x 5
    case 54: return 0x3332u;  // 2 x 3 x 3 x 3
    case 60: return 0x534u;  // 4 x 3 x 5
    case 64: return 0x444u;  // 4 x 4 x 4
    case 72: return 0x3324u;  // 4 x 2 x 3 x 3
    default: return 0u;
  }
}
constexpr int reg_radix(int n, int s) { return (int)((reg_plan(n) >> (4 * s)) & 15u); }
constexpr int reg_nstages(int n) {
  int s = 0;
  while (reg_radix(n, s) != 0) ++s;
  return s;
}

// frequency index held at position p after the transform
template <int N>
__host__ __device__ constexpr int dif_freq(int p) {
  int k = 0, w = 1, L = N;
  for (int s = 0; s < reg_nstages(N); ++s) {
    const int R = reg_radix(N, s), M = L / R;
    const int d = p / M;
    p -= d * M;
    k += d * w;
    w *= R;
    L = M;
  }
  return k;
}

// Stage S on the block x[off .. off + L); tab[t] = exp(-2 pi i t / NT).
template <typename T, int NT, int L, int S, int SIGN>
__device__ __forceinline__ void reg_dif(cplx<T> (&x)[NT], const cplx<T>* __restrict__ tab, int off) {
  constexpr int R = reg_radix(NT, S);
  constexpr int M = L / R;
#pragma unroll
  for (int n1 = 0; n1 < M; ++n1) {
    cplx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = x[off + n1 + M * r];
    Bfly<T, R>::run(v, T(SIGN), tab, NT / R);
#pragma unroll
    for (int k2 = 0; k2 < R; ++k2) {
      cplx<T> a = v[k2];
      if (n1 > 0 && k2 > 0) {
        cplx<T> w = tab[n1 * k2 * (NT / L)];
        if (SIGN > 0) w.y = -w.y;
        a = a * w;
      }
      x[off + n1 + M * k2] = a;
    }
  }
  if constexpr (S + 1 < reg_nstages(NT)) {
#pragma unroll
    for (int k2 = 0; k2 < R; ++k2) reg_dif<T, NT, M, S + 1, SIGN>(x, tab, off + M * k2);
  }
}

// In-register DFT of length N (sign -1 forward r -> G, +1 inverse G -> r); the result
// for frequency dif_freq<N>(p) is left in x[p].
template <typename T, int N, int SIGN>
__device__ __forceinline__ void reg_fft(cplx<T> (&x)[N], const cplx<T>* tab) {
  reg_dif<T, N, N, 0, SIGN>(x, tab, 0);
}

// ---------------------------------------------------------------------------
// Line passes shared by the register plane kernels (one copy per translation unit).
// ---------------------------------------------------------------------------
namespace {


// per length N: exp(-2 pi i t / N); one copy per translation unit, filled by upload_twiddles()
__constant__ cplx<float> c_tw[reg_table_total()];

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <int N>
__device__ __forceinline__ const cplx<float>* twf() {
  return c_tw + reg_table_offset(N);
}

// One row of length N in place: the inverse transform, or (fwd) the forward one computed
// as conj(inverse(conj(.))), so that both directions run the same code body.
template <int N>
__device__ __forceinline__ void row_fft(cplx<float>* row, bool fwd) {
  const float s = fwd ? -1.f : 1.f;
  cplx<float> x[N];
#pragma unroll
  for (int e = 0; e < N; ++e) x[e] = mk(row[e].x, s * row[e].y);
  reg_fft<float, N, 1>(x, twf<N>());
#pragma unroll
  for (int p = 0; p < N; ++p) row[dif_freq<N>(p)] = mk(x[p].x, s * x[p].y);
}

template <int MAXN>
__device__ __forceinline__ void row_fft_n(int n, cplx<float>* row, bool fwd) {
  switch (n) {
#define SGO_ROW(N)                                  \
  case N:                                           \
    if constexpr (N <= MAXN) row_fft<N>(row, fwd);  \
    break;
    SGO_ROW(10) SGO_ROW(12) SGO_ROW(15) SGO_ROW(16) SGO_ROW(18) SGO_ROW(20) SGO_ROW(24) SGO_ROW(25) SGO_ROW(27)
    SGO_ROW(30) SGO_ROW(32) SGO_ROW(36) SGO_ROW(40) SGO_ROW(45) SGO_ROW(48) SGO_ROW(50) SGO_ROW(54) SGO_ROW(60)
    SGO_ROW(64) SGO_ROW(72)
#undef SGO_ROW
    default: break;
  }
}

// ---- lengths N = 2M over a lane pair (lanes 2k and 2k+1 of a warp, h = lane & 1) ----
// All 32 lanes of the warp must take part (the pair exchanges data by shuffles).

__device__ __forceinline__ cplx<float> shfl_pair(cplx<float> v) {
  return mk(__shfl_xor_sync(0xffffffffu, v.x, 1), __shfl_xor_sync(0xffffffffu, v.y, 1));
}

// Inverse DFT of length 2M.  On entry lane h holds X[h M + j] in x[j]; a radix-2
// decimation-in-frequency step across the pair, y_0[j] = X[j] + X[j + M] and
// y_1[j] = (X[j] - X[j + M]) W_2M^-j, then the lane's M-point inverse: on exit lane h holds
// the sample of time index h + 2 dif_freq<M>(p) in x[p].
template <int M>
__device__ __forceinline__ void pair_inv(cplx<float> (&x)[M], int h) {
  const cplx<float>* tn = twf<2 * M>();
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const cplx<float> o = shfl_pair(x[j]);
    if (h == 0) {
      x[j] = x[j] + o;
    } else {
      cplx<float> w = tn[j];
      w.y = -w.y;
      x[j] = (o - x[j]) * w;
    }
  }
  reg_fft<float, M, 1>(x, twf<M>());
}

// Row of length 2M in place (both directions through pair_inv; forward as conj o inv o conj).
template <int M>
__device__ __forceinline__ void row_pair(cplx<float>* row, bool fwd, int h, bool act) {
  const float s = fwd ? -1.f : 1.f;
  cplx<float> x[M];
#pragma unroll
  for (int j = 0; j < M; ++j) {
    const cplx<float> v = act ? row[h * M + j] : mk(0.f, 0.f);
    x[j] = mk(v.x, s * v.y);
  }
  pair_inv<M>(x, h);
  if (act) {
#pragma unroll
    for (int p = 0; p < M; ++p) row[h + 2 * dif_freq<M>(p)] = mk(x[p].x, s * x[p].y);
  }
}

template <int MAXN>
__device__ __forceinline__ void row_pair_n(int n, cplx<float>* row, bool fwd, int h, bool act) {
  switch (n) {
#define SGO_ROW(N)                                                  \
  case N:                                                           \
    if constexpr (N <= MAXN) row_pair<N / 2>(row, fwd, h, act);     \
    break;
    SGO_ROW(96) SGO_ROW(100) SGO_ROW(108) SGO_ROW(120) SGO_ROW(128)
#undef SGO_ROW
    default: break;
  }
}

// Fill this translation unit's twiddle table on the current device (once per device).
inline bool upload_twiddles() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return true;
  std::vector<cplx<float>> h(reg_table_total());
  for (int i = 0, o = 0; i < kRegCount + kPairCount; o += tw_size(i), ++i)
    for (int t = 0; t < tw_size(i); ++t) {
      const double a = 2.0 * PI * t / tw_size(i);
      h[o + t] = mk((float)std::cos(a), (float)(-std::sin(a)));
    }
  if (cudaMemcpyToSymbol(c_tw, h.data(), sizeof(cplx<float>) * h.size()) != cudaSuccess) return false;
  done[dev] = true;
  return true;
}

}  // namespace

}  // namespace sgo
