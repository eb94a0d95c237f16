// Subspace linear algebra of the all-band CG eigensolver (Algorithm 1).
//
//  * gemm_tn: C = A^T B over the packed plane-wave index (K = npw) -- the subspace
//    matrices H(i,j) = <Psi_i|H|Psi_j> and overlaps, the projection coefficients
//    <Psi_j|P_i> of the search directions and the projector overlaps <beta_I|Psi_n>.
//    Split-K: every CTA sums one K chunk in the working precision and writes an FP64
//    partial; a second kernel adds the partials in a fixed order (deterministic).
//  * gemm_nn: Y = beta Y + alpha A M with a small FP64 matrix M -- subspace rotations
//    by the Rayleigh-Ritz eigenvectors, the projection P -= Psi C, the nonlocal apply.
//  * per-band kernels: residual + preconditioner + conjugate direction, normalisation,
//    line minimisation.
//  * rr: FP64 Cholesky of the overlap, L^-1 H L^-T and a parallel cyclic Jacobi
//    eigensolve (the subspace diagonalisation of Algorithm 1).
//  * occupations: Fermi-Dirac with the chemical potential by safeguarded Newton.
#include <cooperative_groups.h>

#include "ff.cuh"
#include "kernels.h"

namespace sgo {

namespace {

template <typename T>
__device__ __forceinline__ const T* opnd(const Prob& P, int kind, int role) {
  if (kind == OPK_WB) return wbuf<T>(P, role);
  if (kind == OPK_B) return reinterpret_cast<const T*>(P.B);
  return reinterpret_cast<const T*>(P.dB);
}
__device__ __forceinline__ int opnd_count(const Prob& P, int kind) {
  return kind == OPK_WB ? P.nb : (kind == OPK_B ? P.nproj : 3 * P.nproj);
}
__device__ __forceinline__ double* dense_ptr(const Prob& P, int sel) {
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

// Subspace of one Rayleigh-Ritz call: blk = 1, the n_b x n_b matrices S, Hs of the bands;
// blk = 2, the 2 n_b x 2 n_b matrices S2, H2 of the block [X, W] (block Davidson).
__device__ __forceinline__ const double* rr_in_s(const Prob& P, int blk) { return blk == 2 ? P.S2 : P.S; }
__device__ __forceinline__ const double* rr_in_h(const Prob& P, int blk) { return blk == 2 ? P.H2 : P.Hs; }
// Eigenvector j of rank rk (ascending eigenvalue), component i: column rk of the rotation.
// Only the lowest n_b Ritz pairs are kept: rows i < n_b go to Tm (the coefficients on X),
// rows n_b .. 2 n_b - 1 to Cm (those on W).
__device__ __forceinline__ void rr_out_vec(const Prob& P, int i, int rk, double v) {
  const int nb = P.nb;
  if (rk >= nb) return;
  if (i < nb) P.Tm[(size_t)i * nb + rk] = v;
  else P.Cm[(size_t)(i - nb) * nb + rk] = v;
}
__device__ __forceinline__ void rr_out_eps(const Prob& P, int rk, double e) {
  if (rk < P.nb) P.eps[rk] = e;
}
// Near-dependent directions of the block [X, W] (blk = 2): a W vector whose component
// orthogonal to the basis vectors before it has squared norm at most RR_DROP (its own norm
// is 1) is left out of the subspace instead of failing the Cholesky (the preconditioned
// residuals of a random start are nearly collinear): its column of the factor is zero, its
// row of the inverse factor is zero (so the projected matrix has a zero row and column,
// which no rotation touches), and its eigenvalue is taken as RR_DROP_DIAG, so that it ranks
// above every kept Ritz value.  (In the FP32 and cluster kernels the same bound fails the
// Cholesky of an X direction.)
constexpr double RR_DROP = 1e-3;
constexpr double RR_DROP_DIAG = 1e12;
constexpr float RR_DROPPED = -2.f;  // pivot deviation recorded for a left-out direction
// Jacobi sweeps of the FP32 eigensolve with at most this many entries above the threshold run
// as sparse passes (k_rr_f32)
constexpr int RR_SPARSE = 256;

// ---------------------------------------------------------------------------
// C = A^T B, split-K partials.  CTA = (problem, tile_i, tile_j, split).  Thread (ti, tj)
// owns rows 4 ti .. 4 ti + 3 and columns 4 tj .. 4 tj + 3 of the 64 x 64 tile, so every
// K step reads its A and B values as one 16-byte shared load each (two for FP64).  A K
// chunk of 32 is staged from 16-byte global loads along K (zero beyond the split's end:
// splits end on multiples of 32 or at npw, whose tail up to ld is zero).  A^T A (same
// operand twice) computes the tiles with tile_i <= tile_j only; the reduction mirrors them.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void lds4(const T* p, T (&o)[4]) {
  if constexpr (sizeof(T) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  } else {
    const double2 v0 = *reinterpret_cast<const double2*>(p), v1 = *reinterpret_cast<const double2*>(p + 2);
    o[0] = v0.x; o[1] = v0.y; o[2] = v1.x; o[3] = v1.y;
  }
}

template <typename T>
struct alignas(16) KPack {
  static constexpr int W = 16 / sizeof(T);
  T e[W];
};

template <typename T>
__global__ void __launch_bounds__(256) k_gemm_tn(KArgs ka, int akind, int arole, int bkind, int brole, double* part_base,
                                                size_t part_stride, int kc) {
  constexpr int W = KPack<T>::W;                 // K values per 16-byte load
  constexpr int NLD = 32 * TN_TILE / W / 256;    // loads per thread per operand per chunk
  constexpr int LS = TN_TILE + 4;                // row stride (16-byte aligned rows)
  __shared__ __align__(16) T As[32][LS];
  __shared__ __align__(16) T Bs[32][LS];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  int local = blockIdx.x - ka.start[p];
  const int na = opnd_count(P, akind), nbv = opnd_count(P, bkind);
  const int ta = (na + TN_TILE - 1) / TN_TILE, tb = (nbv + TN_TILE - 1) / TN_TILE;
  const int split = local / (ta * tb);
  local -= split * ta * tb;
  const int ti0 = (local / tb) * TN_TILE, tj0 = (local % tb) * TN_TILE;
  if (akind == bkind && arole == brole && ti0 > tj0) return;  // mirrored by the reduction
  const T* A = opnd<T>(P, akind, arole);
  const T* Bm = opnd<T>(P, bkind, brole);
  const int ld = P.ld;
  const int k0 = split * kc, k1 = min(P.npw, k0 + kc);
  const int t = threadIdx.x;
  const int ti = t & 15, tj = t >> 4;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  // load f = t + 256 q: vector f % 64, K offset (f / 64) W within the chunk
  KPack<T> ra[NLD], rb[NLD];
  auto fetch = [&](int kb) {
#pragma unroll
    for (int q = 0; q < NLD; ++q) {
      const int f = t + 256 * q;
      const int v = f & (TN_TILE - 1), k = kb + (f / TN_TILE) * W;
      KPack<T> za, zb;
#pragma unroll
      for (int c = 0; c < W; ++c) za.e[c] = zb.e[c] = T(0);
      if (k < k1) {
        if (ti0 + v < na) za = *reinterpret_cast<const KPack<T>*>(A + (size_t)(ti0 + v) * ld + k);
        if (tj0 + v < nbv) zb = *reinterpret_cast<const KPack<T>*>(Bm + (size_t)(tj0 + v) * ld + k);
      }
      ra[q] = za;
      rb[q] = zb;
    }
  };
  fetch(k0);
  for (int kb = k0; kb < k1; kb += 32) {
#pragma unroll
    for (int q = 0; q < NLD; ++q) {
      const int f = t + 256 * q;
      const int v = f & (TN_TILE - 1), kq = (f / TN_TILE) * W;
#pragma unroll
      for (int c = 0; c < W; ++c) {
        As[kq + c][v] = ra[q].e[c];
        Bs[kq + c][v] = rb[q].e[c];
      }
    }
    __syncthreads();
    if (kb + 32 < k1) fetch(kb + 32);
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      T a[4], b[4];
      lds4(&As[kk][4 * ti], a);
      lds4(&Bs[kk][4 * tj], b);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j2 = 0; j2 < 4; ++j2) acc[i][j2] += a[i] * b[j2];
    }
    __syncthreads();
  }
  double* part = part_base + (size_t)p * part_stride + (size_t)split * na * nbv;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int i = ti0 + 4 * ti + a, j = tj0 + 4 * tj + b;
      if (i < na && j < nbv) part[(size_t)i * nbv + j] = (double)acc[a][b];
    }
}

// Sum the partials in split order.  CTA = (problem, chunk of 256 outputs).  sym: A^T A
// from k_gemm_tn, whose tiles below the diagonal were not computed (read mirrored).
__global__ void k_gemm_tn_reduce(KArgs ka, int akind, int bkind, int dst, const double* part_base, size_t part_stride,
                                 int kc, int sym) {
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int na = opnd_count(P, akind), nbv = opnd_count(P, bkind);
  const int o = (blockIdx.x - ka.start[p]) * 256 + threadIdx.x;
  if (o >= na * nbv) return;
  const int nsplit = (P.npw + kc - 1) / kc;
  const double* part = part_base + (size_t)p * part_stride;
  int src = o;
  if (sym) {
    const int i = o / nbv, j = o - i * nbv;
    if (i / TN_TILE > j / TN_TILE) src = j * nbv + i;
  }
  double s = 0.0;
  for (int k = 0; k < nsplit; ++k) s += part[(size_t)k * na * nbv + src];
  dense_ptr(P, dst)[o] = s;
}

// ---------------------------------------------------------------------------
// Y = beta Y + alpha A M: rows npw, inner = count(A), columns nb.
// M is row-major [inner][nb] FP64 (DD_PROJ_D: rows scaled by the atoms' D).
// CTA = (problem, row tile, column tile), 64 x 64 outputs, 4 x 4 per thread.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_gemm_nn(KArgs ka, int akind, RolePairs rp, int msel, double alpha,
                                                double beta) {
  const int arole = rp.a[blockIdx.y], yrole = rp.y[blockIdx.y];
  // CTA = (problem, group of NN_RT row tiles of 64, column tile of 64).  The small matrix
  // M[0:inner][c0:c0+64] is staged once per CTA (in passes of NN_KP rows of M) and reused
  // by every row tile; thread (tr, tc) owns rows tr + 16 i and columns tc + 16 j (i, j < 4).
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ms = reinterpret_cast<T*>(smem_raw);        // [NN_KP][64]
  __shared__ T As[32][64];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int local = blockIdx.x - ka.start[p];
  const int nct = (P.nb + 63) / 64;
  const int rg = local / nct, c0 = (local % nct) * 64;
  const int inner = opnd_count(P, akind);
  const int nb = P.nb, ld = P.ld, npw = P.npw;
  const T* A = opnd<T>(P, akind, arole);
  const double* M = dense_ptr(P, msel);
  T* Y = wbuf<T>(P, yrole);
  const int t = threadIdx.x, tr = t & 15, tc = t >> 4;
  const int npass = (inner + NN_KP - 1) / NN_KP;
  for (int rt = 0; rt < NN_RT; ++rt) {
    const int r0 = (rg * NN_RT + rt) * 64;
    if (r0 >= npw) break;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    for (int ps = 0; ps < npass; ++ps) {
      const int kp0 = ps * NN_KP, kpn = min(NN_KP, inner - kp0);
      if (rt == 0 || npass > 1) {
        __syncthreads();
        for (int e = t; e < kpn * 64; e += 256) {
          const int kk = e >> 6, cc = e & 63;
          const int k = kp0 + kk;
          double mv = 0.0;
          if (c0 + cc < nb) {
            mv = M[(size_t)k * nb + c0 + cc];
            if (msel == DD_PROJ_D) mv *= P.pj_d[k];
          }
          Ms[e] = (T)mv;
        }
      }
      T ra[8];
      auto fetch = [&](int kb) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int e = t + 256 * q;  // 2048 = 32 x 64
          const int kk = e >> 6, rr = e & 63;
          ra[q] = (kb + kk < kpn && r0 + rr < npw) ? A[(size_t)(kp0 + kb + kk) * ld + r0 + rr] : T(0);
        }
      };
      fetch(0);
      for (int kb = 0; kb < kpn; kb += 32) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int e = t + 256 * q;
          As[e >> 6][e & 63] = ra[q];
        }
        __syncthreads();
        if (kb + 32 < kpn) fetch(kb + 32);
        const int kn = min(32, kpn - kb);
        for (int kk = 0; kk < kn; ++kk) {
          T a[4], m[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) a[i] = As[kk][tr + 16 * i];
#pragma unroll
          for (int j = 0; j < 4; ++j) m[j] = Ms[(kb + kk) * 64 + tc + 16 * j];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * m[j];
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tc + 16 * j;
      if (c >= nb) continue;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = r0 + tr + 16 * i;
        if (r >= npw) continue;
        T* y = Y + (size_t)c * ld + r;
        T v = T(alpha) * acc[i][j];
        if (beta != 0.0) v += T(beta) * (*y);
        *y = v;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// per-band kernels: CTA = (problem, band)
// ---------------------------------------------------------------------------
// Per-band kernels stream a band's ld components as 16-byte packs (4 FP32 or 2 FP64).
// Components npw .. ld-1 of every band buffer and of the kinetic tables are zero (the
// arena is cleared at set-up and every writer stores zeros or only k < npw there), so
// they add nothing to the sums and stay zero.
template <typename T>
struct alignas(16) Pack16 {
  static constexpr int W = 16 / sizeof(T);
  T e[W];
};

template <typename T>
__device__ __forceinline__ const Pack16<T>* pk(const T* p) {
  return reinterpret_cast<const Pack16<T>*>(p);
}
template <typename T>
__device__ __forceinline__ Pack16<T>* pk(T* p) {
  return reinterpret_cast<Pack16<T>*>(p);
}
template <typename T>
__device__ __forceinline__ const Pack16<T>* ekin_pk(const Prob& P) {
  return reinterpret_cast<const Pack16<T>*>(sizeof(T) == 4 ? (const void*)P.ekin32 : (const void*)P.ekin);
}

template <typename T>
__global__ void __launch_bounds__(BAND_THREADS) k_band_kinetic(KArgs ka, int xr) {
  __shared__ double red[33];
  constexpr int W = Pack16<T>::W;
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int i = blockIdx.x - ka.start[p];
  const Pack16<T>* x = pk(wbuf<T>(P, xr) + (size_t)i * P.ld);
  const Pack16<T>* ek = ekin_pk<T>(P);
  T st = T(0);
  for (int v = threadIdx.x; v < P.ld / W; v += blockDim.x) {
    const Pack16<T> a = x[v], g = ek[v];
#pragma unroll
    for (int j = 0; j < W; ++j) st += g.e[j] * a.e[j] * a.e[j];
  }
  const double s = block_sum((double)st, red);
  if (threadIdx.x == 0) P.bv[BV_EKIN * P.nb + i] = s;
}

// |H x_i - eps_i x_i| of every band (the convergence test of Algorithm 1's CG loop).
template <typename T>
__global__ void __launch_bounds__(BAND_THREADS) k_band_residual(KArgs ka, int xr, int hxr) {
  __shared__ double red[33];
  constexpr int W = Pack16<T>::W;
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int i = blockIdx.x - ka.start[p];
  const size_t off = (size_t)i * P.ld;
  const Pack16<T>* x = pk(wbuf<T>(P, xr) + off);
  const Pack16<T>* hx = pk(wbuf<T>(P, hxr) + off);
  const T eps = T(P.eps[i]);
  T st = T(0);
  for (int v = threadIdx.x; v < P.ld / W; v += blockDim.x) {
    const Pack16<T> a = x[v], h = hx[v];
#pragma unroll
    for (int j = 0; j < W; ++j) {
      const T r = h.e[j] - eps * a.e[j];
      st += r * r;
    }
  }
  const double s = block_sum((double)st, red);
  if (threadIdx.x == 0) P.bv[BV_RES * P.nb + i] = sqrt(s);
}

// Teter-Payne-Allan preconditioner factor, y = T(G) / E_kin(band).
template <typename T>
__device__ __forceinline__ T tpa(T y) {
  T y2 = y * y, y3 = y2 * y;
  T num = T(27) + T(18) * y + T(12) * y2 + T(8) * y3;
  return num / (num + T(16) * y2 * y2);
}

// Residual R = HX - eps X, G = A R (TPA preconditioner), conjugate direction
// P = G + gamma P_prev with Polak-Ribiere gamma = <G, R - R_prev>/<G_prev, R_prev>, >= 0
// (Algorithm 1).  Writes P and R (for the next step).
template <typename T>
__global__ void __launch_bounds__(BAND_THREADS) k_cg_precond(KArgs ka, int xr, int hxr, int pr, int rr_out, int ppr, int rpr) {
  __shared__ double red[33];
  constexpr int W = Pack16<T>::W;
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int i = blockIdx.x - ka.start[p];
  const size_t off = (size_t)i * P.ld;
  const int nv = P.ld / W;
  const Pack16<T>* x = pk(wbuf<T>(P, xr) + off);
  const Pack16<T>* hx = pk(wbuf<T>(P, hxr) + off);
  Pack16<T>* pv = pk(wbuf<T>(P, pr) + off);
  Pack16<T>* rv = pk(wbuf<T>(P, rr_out) + off);
  // rpr < 0: no conjugation history (the preconditioned residual alone, block Davidson)
  const bool first = rpr < 0 || P.scal[SC_FIRSTCG] != 0.0;
  const Pack16<T>* pp = first ? nullptr : pk(wbuf<T>(P, ppr) + off);
  const Pack16<T>* rp = first ? nullptr : pk(wbuf<T>(P, rpr) + off);
  const Pack16<T>* ek = ekin_pk<T>(P);
  T ekp = T(0);
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    const Pack16<T> a = x[v], g = ek[v];
#pragma unroll
    for (int j = 0; j < W; ++j) ekp += g.e[j] * a.e[j] * a.e[j];
  }
  double ekd = block_sum((double)ekp, red);
  ekd = fmax(ekd, 1e-3);
  const T eps = T(P.eps[i]);
  const T iek = T(1.0 / ekd);
  T grt = T(0), grpt = T(0), r2t = T(0);
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    const Pack16<T> a = x[v], h = hx[v], g = ek[v];
    Pack16<T> rprev;
    if (!first) rprev = rp[v];
    Pack16<T> ro, go;
#pragma unroll
    for (int j = 0; j < W; ++j) {
      const T r = h.e[j] - eps * a.e[j];
      const T gg = tpa<T>(g.e[j] * iek) * r;
      grt += gg * r;
      r2t += r * r;
      if (!first) grpt += gg * rprev.e[j];
      ro.e[j] = r;
      go.e[j] = gg;
    }
    rv[v] = ro;
    pv[v] = go;
  }
  double gr = block_sum((double)grt, red);
  double grp = block_sum((double)grpt, red);
  double r2 = block_sum((double)r2t, red);
  double gamma = 0.0;
  if (!first) {
    double den = P.bv[BV_GRP * P.nb + i];
    gamma = den > 0.0 ? fmax(0.0, (gr - grp) / den) : 0.0;
  }
  if (gamma != 0.0) {
    const T gm = T(gamma);
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
      Pack16<T> a = pv[v];
      const Pack16<T> b = pp[v];
#pragma unroll
      for (int j = 0; j < W; ++j) a.e[j] = a.e[j] + gm * b.e[j];
      pv[v] = a;
    }
  }
  if (threadIdx.x == 0) {
    P.bv[BV_GR * P.nb + i] = gr;
    P.bv[BV_RES * P.nb + i] = sqrt(r2);
    P.bv[BV_GAMMA * P.nb + i] = gamma;
    P.bv[BV_EKIN * P.nb + i] = ekd;
  }
}

// PP = P (history direction, unnormalised); P = P / |P|.
template <typename T>
__global__ void __launch_bounds__(BAND_THREADS) k_normalize(KArgs ka, int pr, int ppr) {
  __shared__ double red[33];
  constexpr int W = Pack16<T>::W;
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int i = blockIdx.x - ka.start[p];
  const size_t off = (size_t)i * P.ld;
  const int nv = P.ld / W;
  Pack16<T>* pv = pk(wbuf<T>(P, pr) + off);
  Pack16<T>* pp = ppr < 0 ? nullptr : pk(wbuf<T>(P, ppr) + off);  // ppr < 0: no history copy
  T st = T(0);
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    const Pack16<T> a = pv[v];
#pragma unroll
    for (int j = 0; j < W; ++j) st += a.e[j] * a.e[j];
  }
  const double s = sqrt(block_sum((double)st, red));
  const T inv = s > 1e-150 ? T(1.0 / s) : T(0);
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    Pack16<T> a = pv[v];
    if (pp) pp[v] = a;
#pragma unroll
    for (int j = 0; j < W; ++j) a.e[j] *= inv;
    pv[v] = a;
  }
  if (threadIdx.x == 0) {
    P.bv[BV_PNORM * P.nb + i] = s;
    // end of this CG step's use of the Polak-Ribiere history: the current <g, r> becomes
    // the previous one, and the history is valid from the next step on
    P.bv[BV_GRP * P.nb + i] = P.bv[BV_GR * P.nb + i];
    if (i == 0) P.scal[SC_FIRSTCG] = 0.0;
  }
}

// Line minimisation (Algorithm 1): in span{x, p} (p unit, p orthogonal to x) the Rayleigh
// quotient is a cos^2 + 2 b sin cos + c sin^2; theta = atan2(-2b, c - a)/2 minimises it.
template <typename T>
__global__ void __launch_bounds__(BAND_THREADS) k_line_min(KArgs ka, int xr, int hxr, int pr, int hpr) {
  __shared__ double red[33];
  constexpr int W = Pack16<T>::W;
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int i = blockIdx.x - ka.start[p];
  const size_t off = (size_t)i * P.ld;
  const int nv = P.ld / W;
  Pack16<T>* x = pk(wbuf<T>(P, xr) + off);
  Pack16<T>* hx = pk(wbuf<T>(P, hxr) + off);
  const Pack16<T>* pv = pk(wbuf<T>(P, pr) + off);
  const Pack16<T>* hp = pk(wbuf<T>(P, hpr) + off);
  T at = T(0), bt = T(0), ct = T(0);
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    const Pack16<T> xv = x[v], pq = pv[v], h = hx[v], q = hp[v];
#pragma unroll
    for (int j = 0; j < W; ++j) {
      at += xv.e[j] * h.e[j];
      bt += pq.e[j] * h.e[j];
      ct += pq.e[j] * q.e[j];
    }
  }
  double a = block_sum((double)at, red);
  double b = block_sum((double)bt, red);
  double c = block_sum((double)ct, red);
  double th = 0.0;
  if (P.bv[BV_PNORM * P.nb + i] > 1e-150) th = 0.5 * atan2(-2.0 * b, c - a);
  const double lim = 0.25 * PI;
  th = fmin(fmax(th, -lim), lim);
  const T cs = (T)cos(th), sn = (T)sin(th);
  if (th != 0.0) {
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
      Pack16<T> xv = x[v], h = hx[v];
      const Pack16<T> pq = pv[v], q = hp[v];
#pragma unroll
      for (int j = 0; j < W; ++j) {
        xv.e[j] = cs * xv.e[j] + sn * pq.e[j];
        h.e[j] = cs * h.e[j] + sn * q.e[j];
      }
      x[v] = xv;
      hx[v] = h;
    }
  }
  if (threadIdx.x == 0) {
    P.bv[BV_THETA * P.nb + i] = th;
    P.bv[BV_A * P.nb + i] = a;
    P.bv[BV_B * P.nb + i] = b;
    P.bv[BV_C * P.nb + i] = c;
  }
}

// Random start (Sec. II D: the CG "begins with an initial set of wavefunctions"):
// splitmix64 (Steele, Lea & Flood, OOPSLA 2014) of (seed, band, component), uniform in
// [-1/2, 1/2), damped by 1/(1 + |G|^2/2).
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename T>
__global__ void k_random_init(KArgs ka, int xr, unsigned long long seed) {
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int i = blockIdx.x - ka.start[p];
  T* x = wbuf<T>(P, xr) + (size_t)i * P.ld;
  for (int k = threadIdx.x; k < P.ld; k += blockDim.x) {
    double v = 0.0;
    if (k < P.npw) {
      unsigned long long h = splitmix64(seed ^ splitmix64(((unsigned long long)i << 32) | (unsigned)k));
      v = ((double)(h >> 11) * (1.0 / 9007199254740992.0) - 0.5) / (1.0 + P.ekin[k]);
    }
    x[k] = (T)v;
  }
}

// Host <-> packed buffers (rows of npw doubles) for the component entry points.
template <typename T>
__global__ void k_copy_in(KArgs ka, int role, const double* src, int nvec, int keep_tail) {
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  const Prob& P = ka.probs[p];
  const int i = blockIdx.x - ka.start[p];
  if (keep_tail && i >= nvec) return;  // rows beyond nvec keep their contents
  T* x = wbuf<T>(P, role) + (size_t)i * P.ld;
  for (int k = threadIdx.x; k < P.ld; k += blockDim.x)
    x[k] = (i < nvec && k < P.npw) ? (T)src[(size_t)i * P.npw + k] : T(0);
}
template <typename T>
__global__ void k_copy_out(KArgs ka, int role, double* dst, int nvec) {
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  const Prob& P = ka.probs[p];
  const int i = blockIdx.x - ka.start[p];
  if (i >= nvec) return;
  const T* x = wbuf<T>(P, role) + (size_t)i * P.ld;
  for (int k = threadIdx.x; k < P.npw; k += blockDim.x) dst[(size_t)i * P.npw + k] = (double)x[k];
}

// ---------------------------------------------------------------------------
// Rayleigh-Ritz in FP64, one CTA per problem (orthonormalisation + subspace
// diagonalisation of Algorithm 1).
//   S = L L^T (Cholesky), C = L^-1 Hs L^-T, C = V diag(eps) V^T (cyclic Jacobi,
//   round-robin parallel ordering; Golub & Van Loan, Alg. 8.4.3), Tm = L^-T V,
//   so that X Tm is orthonormal and diagonalises H in the subspace.
// Matrices: A, L, V in shared memory when 3 nb^2 doubles fit, else in global scratch.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(RR_THREADS) k_rr(KArgs ka, int use_smem, double* gscratch, size_t gstride,
                                                   int max_sweeps, int blk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[33];
  __shared__ double cs_c[256], cs_s[256];
  __shared__ int pr_p[256], pr_q[256];
  __shared__ int flag;
  __shared__ unsigned char drp[512];  // left-out directions (blk = 2)
  const int p = blockIdx.x;
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int n = blk * P.nb;
  const double* Sin = rr_in_s(P, blk);
  const double* Hin = rr_in_h(P, blk);
  double *A, *L, *V;
  if (use_smem) {
    A = reinterpret_cast<double*>(smem_raw);
  } else {
    A = gscratch + (size_t)p * gstride;
  }
  L = A + n * n;
  V = L + n * n;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) flag = 0;
  // symmetrised inputs
  for (int e = tid; e < n * n; e += nt) {
    int i = e / n, j = e % n;
    L[e] = 0.5 * (Sin[i * n + j] + Sin[j * n + i]);
    A[e] = 0.5 * (Hin[i * n + j] + Hin[j * n + i]);
  }
  __syncthreads();
  // Cholesky of L in place (lower triangle); a left-out direction (blk = 2) gets a unit
  // pivot and a zero column (its row of L^-1 is cleared below)
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      double d = L[k * n + k];
      const bool dr = blk == 2 && k >= P.nb && d <= RR_DROP;
      if (dr) d = 1.0;
      if (!(d > 0.0)) { flag = 1; d = 1.0; }
      L[k * n + k] = sqrt(d);
      drp[k] = dr ? 1 : 0;
    }
    __syncthreads();
    const bool drop = drp[k] != 0;
    const double dk = L[k * n + k];
    for (int i = k + 1 + tid; i < n; i += nt) L[i * n + k] = drop ? 0.0 : L[i * n + k] / dk;
    __syncthreads();
    const int m = n - k - 1;
    for (int e = tid; e < m * m; e += nt) {
      int i = k + 1 + e / m, j = k + 1 + e % m;
      if (j <= i) L[i * n + j] -= L[i * n + k] * L[j * n + k];
    }
    __syncthreads();
  }
  // L := L^-1 (lower), row by row: X[i][j] = -(sum_{k=j}^{i-1} L[i][k] X[k][j]) / L[i][i]
  // done out of place into V, then copied back.
  for (int e = tid; e < n * n; e += nt) V[e] = 0.0;
  __syncthreads();
  for (int i = 0; i < n; ++i) {
    const double lii = L[i * n + i];
    for (int j = tid; j <= i; j += nt) {
      if (j == i) {
        V[i * n + i] = 1.0 / lii;
      } else {
        double s = 0.0;
        for (int k = j; k < i; ++k) s += L[i * n + k] * V[k * n + j];
        V[i * n + j] = -s / lii;
      }
    }
    __syncthreads();
  }
  // (rows of L^-1 of left-out directions cleared)
  for (int e = tid; e < n * n; e += nt) L[e] = drp[e / n] ? 0.0 : V[e];
  __syncthreads();
  // V := A L^T ; A := L V   (C = L^-1 Hs L^-T, symmetric)
  for (int e = tid; e < n * n; e += nt) {
    int i = e / n, j = e % n;
    double s = 0.0;
    for (int k = 0; k <= j; ++k) s += A[i * n + k] * L[j * n + k];
    V[e] = s;
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += nt) {
    int i = e / n, j = e % n;
    double s = 0.0;
    for (int k = 0; k <= i; ++k) s += L[i * n + k] * V[k * n + j];
    A[e] = s;
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += nt) {
    int i = e / n, j = e % n;
    if (j > i) {
      double s = 0.5 * (A[i * n + j] + A[j * n + i]);
      A[i * n + j] = s;
      A[j * n + i] = s;
    }
  }
  // accumulate the rotations onto L^-T, so that V ends as Tm = L^-T U directly
  for (int e = tid; e < n * n; e += nt) {
    int i = e / n, j = e % n;
    V[e] = L[j * n + i];
  }
  __syncthreads();
  // cyclic Jacobi, round-robin pairing over m = n rounded up to even.  A rotation whose
  // |a_pq| is below 1e-14 sqrt(|a_pp a_qq|) is skipped; sweeps stop once the
  // off-diagonal norm is below 1e-11 of the diagonal norm (FP64 rounding floor ~1e-15).
  const int m = n + (n & 1);
  const int half = m / 2;
  int sweeps = 0, capped = 0;
  for (int sweep = 0;; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int e = tid; e < n * n; e += nt) {
      int i = e / n, j = e % n;
      double v = A[e] * A[e];
      if (i == j) dia += v; else off += v;
    }
    off = block_sum(off, red);
    dia = block_sum(dia, red);
    if (off <= 1e-22 * dia || off == 0.0) break;
    if (sweep == max_sweeps) {
      capped = 1;
      break;
    }
    ++sweeps;
    for (int r = 0; r < m - 1; ++r) {
      if (tid < half) {
        // tournament: position 0 fixed, positions 1..m-1 rotate by r
        int a = tid, b = m - 1 - tid;
        int pa = a == 0 ? 0 : 1 + (a - 1 + r) % (m - 1);
        int pb = b == 0 ? 0 : 1 + (b - 1 + r) % (m - 1);
        int pp = min(pa, pb), qq = max(pa, pb);
        double c = 1.0, s = 0.0;
        if (qq < n) {
          double apq = A[pp * n + qq];
          double app = A[pp * n + pp], aqq = A[qq * n + qq];
          if (fabs(apq) > 1e-14 * sqrt(fabs(app * aqq)) && fabs(apq) > 1e-300) {
            double tau = (aqq - app) / (2.0 * apq);
            double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        cs_c[tid] = c;
        cs_s[tid] = s;
        pr_p[tid] = pp;
        pr_q[tid] = qq;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int e = tid; e < half * n; e += nt) {
        int k = e / n, j = e % n;
        double s = cs_s[k];
        if (s == 0.0) continue;
        int pp = pr_p[k], qq = pr_q[k];
        double c = cs_c[k];
        double ap = A[pp * n + j], aq = A[qq * n + j];
        A[pp * n + j] = c * ap - s * aq;
        A[qq * n + j] = s * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int e = tid; e < half * n; e += nt) {
        int k = e / n, i = e % n;
        double s = cs_s[k];
        if (s == 0.0) continue;
        int pp = pr_p[k], qq = pr_q[k];
        double c = cs_c[k];
        double ap = A[i * n + pp], aq = A[i * n + qq];
        A[i * n + pp] = c * ap - s * aq;
        A[i * n + qq] = s * ap + c * aq;
        double vp = V[i * n + pp], vq = V[i * n + qq];
        V[i * n + pp] = c * vp - s * vq;
        V[i * n + qq] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  // ascending order: rank of each eigenvalue (a left-out direction ranks last)
  for (int j = tid; j < n; j += nt) {
    double ej = drp[j] ? RR_DROP_DIAG : A[j * n + j];
    int rank = 0;
    for (int k2 = 0; k2 < n; ++k2) {
      double ek = drp[k2] ? RR_DROP_DIAG : A[k2 * n + k2];
      rank += (ek < ej) || (ek == ej && k2 < j);
    }
    rr_out_eps(P, rank, ej);
    P.bv[BV_TMP0 * P.nb + j] = (double)rank;  // (blk = 2: rows BV_TMP0 and BV_TMP1)
  }
  __syncthreads();
  // Tm[:, rank(j)] = V[:, j]  (= L^-T U)
  for (int e = tid; e < n * n; e += nt) {
    int i = e / n, j = e % n;
    rr_out_vec(P, i, (int)P.bv[BV_TMP0 * P.nb + j], V[e]);
  }
  if (tid == 0) {
    P.scal[SC_RRSWEEPS] += sweeps;
    P.scal[SC_RRCAP] += capped;
  }
  if (tid == 0 && flag) P.status[0] = 1;
}

// ---------------------------------------------------------------------------
// Rayleigh-Ritz for the mixed path, one CTA per problem, in FP32 shared memory.
// The overlap is factored in deviation form: S = I + E, L = I + D (Cholesky), L^-1 =
// I + G.  Every stored quantity is then of the size of E and keeps FP32 relative
// accuracy, so the factors are as accurate as an FP64 factorisation of the same S (whose
// entries carry the GEMM's FP32 rounding anyway): for column k, with x = E_kk - sum D_kj^2
// (the running trailing entry), d_k = sqrt(1 + x) - 1 = x / (1 + sqrt(1 + x)), and
// D_ik = (E_ik - sum_j D_ij D_kj) / (1 + d_k).  G follows from (I + D)(I + G) = I row by
// row.  Then C = (I + G) H (I + G)^T, its cyclic Jacobi eigensolve accumulated onto
// V = (I + G)^T, and Tm = V in ascending eigenvalue order.  The eigen-rotation feeds the
// FP32 block rotation, so accuracy beyond FP32 would be discarded there.
// Shared memory: D, G, Hf (then V^T), W, A, each n x ns floats with an odd row stride
// ns = n | 1, so that walks down a column hit distinct banks.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(RR_THREADS) k_rr_f32(KArgs ka, float* gscratch, size_t gstride, int max_sweeps,
                                                       int blk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float red[32];
  __shared__ float dkv[512];  // Cholesky pivots d_k (n <= 512: the pair tables below hold 256 pairs)
  // (the rotations of a round, or, while a sparse pass is being scheduled, the round
  // masks of every index)
  __shared__ union {
    struct {
      float c[256], s[256];
    } cs;
    unsigned used[512];
  } ru;
  float* cs_c = ru.cs.c;
  float* cs_s = ru.cs.s;
  __shared__ int pr_p[256], pr_q[256];
  __shared__ int sp_list[RR_SPARSE], sp_sorted[RR_SPARSE], sp_rstart[33];
  __shared__ unsigned char sp_stamp[512];
  __shared__ int flag, nbig, sp_rounds, wcnt[32];
  const int p = blockIdx.x;
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int n = blk * P.nb, ns = n | 1, nn = n * ns;
  const double* Sin = rr_in_s(P, blk);
  const double* Hin = rr_in_h(P, blk);
  // the five matrices live in shared memory, or (large n) in this problem's global scratch
  float* D = gscratch ? gscratch + (size_t)p * gstride : reinterpret_cast<float*>(smem_raw);
  float* G = D + nn;
  float* Hf = G + nn;
  float* W = Hf + nn;
  float* A = W + nn;
  float* Vt = Hf;  // V^T, once Hf is consumed
  const int tid = threadIdx.x, nt = blockDim.x, tx = tid & 31, ty = tid >> 5, nty = nt >> 5;
  if (tid == 0) flag = 0;
  for (int i = ty; i < n; i += nty)
    for (int j = tx; j < n; j += 32) {
      D[i * ns + j] = (float)(0.5 * (Sin[i * n + j] + Sin[j * n + i]) - (i == j ? 1.0 : 0.0));
      Hf[i * ns + j] = (float)(0.5 * (Hin[i * n + j] + Hin[j * n + i]));
      G[i * ns + j] = 0.f;
    }
  __syncthreads();
  // Cholesky in deviation form, right-looking, one barrier per column: step k reads the
  // lower column k (final after step k - 1), writes the scaled column L_ik = D_ik / (1 + d_k)
  // into the upper row k (D_ki, never read in step k) and updates the lower trailing block
  // with the scaled values formed on the fly; d_k goes to dkv
  // (a left-out direction of the block [X, W]: zero scaled column, no update, pivot mark
  // RR_DROPPED in dkv)
  for (int k = 0; k < n; ++k) {
    const float x = D[k * ns + k];
    const bool drop = blk == 2 && k >= P.nb && x <= (float)RR_DROP - 1.f;
    const float xs = drop ? 0.f : fmaxf(x, -0.999f);
    const float dk = xs / (1.f + sqrtf(1.f + xs));
    const float inv = drop ? 0.f : 1.f / (1.f + dk);
    if (tid == 0) {
      if (!drop && !(x > -0.999f)) flag = 1;  // S not positive definite (to FP32 resolution)
      dkv[k] = drop ? RR_DROPPED : dk;
    }
    for (int i = k + 1 + tid; i < n; i += nt) D[k * ns + i] = D[i * ns + k] * inv;
    if (!drop)
      for (int i = k + 1 + ty; i < n; i += nty) {
        const float lik = D[i * ns + k] * inv;
        for (int j = k + 1 + tx; j <= i; j += 32) D[i * ns + j] -= lik * (D[j * ns + k] * inv);
      }
    __syncthreads();
  }
  // G: G_ii = -d_i / (1 + d_i), G_ij = -(L_ij + sum_{j<=k<i} L_ik G_kj) / (1 + d_i) with
  // L_ik = D_ki; every column j of G is an independent forward substitution: one warp per
  // column, lanes splitting the sum, no block barrier until all columns are done
  // (a left-out direction's row of I + G is zero: G_jj = -1, G_ij = 0)
  for (int j = ty; j < n; j += nty) {
    if (tx == 0) G[j * ns + j] = dkv[j] == RR_DROPPED ? -1.f : -dkv[j] / (1.f + dkv[j]);
    __syncwarp();
    for (int i = j + 1; i < n; ++i) {
      float sacc = 0.f;
      for (int k = j + tx; k < i; k += 32) sacc += D[k * ns + i] * G[k * ns + j];
      sacc = warp_sum_f(sacc);
      if (tx == 0) G[i * ns + j] = dkv[i] == RR_DROPPED ? 0.f : -(D[j * ns + i] + sacc) / (1.f + dkv[i]);
      __syncwarp();
    }
  }
  __syncthreads();
  // W = (I + G) Hf, A = W (I + G)^T
  for (int i = ty; i < n; i += nty)
    for (int j = tx; j < n; j += 32) {
      float s = 0.f;
      for (int k = 0; k <= i; ++k) s += G[i * ns + k] * Hf[k * ns + j];
      W[i * ns + j] = Hf[i * ns + j] + s;
    }
  __syncthreads();
  for (int i = ty; i < n; i += nty)
    for (int j = tx; j < n; j += 32) {
      float s = 0.f;
      for (int k = 0; k <= j; ++k) s += W[i * ns + k] * G[j * ns + k];
      A[i * ns + j] = W[i * ns + j] + s;
    }
  __syncthreads();
  float amax = 0.f;
  for (int i = ty; i < n; i += nty)
    for (int j = tx; j < n; j += 32) {
      if (j > i) {
        const float sy = 0.5f * (A[i * ns + j] + A[j * ns + i]);
        A[i * ns + j] = sy;
        A[j * ns + i] = sy;
      }
      if (i == j) amax = fmaxf(amax, fabsf(A[i * ns + i]));
      Vt[i * ns + j] = (i == j ? 1.f : 0.f) + G[i * ns + j];  // V = (I + G)^T = L^-T
    }
  for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  if (tx == 0) red[ty] = amax;
  __syncthreads();
  float mm = 0.f;
  for (int w = 0; w < nty; ++w) mm = fmaxf(mm, red[w]);
  // rotations below 2e-7 max|a_ii| (about the FP32 resolution of the matrix) are skipped
  const float thr = 2e-7f * mm;
  // Threshold Jacobi.  Each sweep starts by listing the off-diagonal entries above thr.
  // Many of them (more than RR_SPARSE, or more than two per index, where the colouring
  // below would need about as many rounds as a sweep): a cyclic sweep in round-robin
  // order, where a round
  // maps every 2x2 block of pair rows P and pair columns Q as A_PQ <- J_P^T A_PQ J_Q (one
  // pass) and V_{:,Q} <- V_{:,Q} J_Q.  Few (the sweeps after the first, once the
  // convergence is quadratic): a sparse pass that rotates only the listed pairs, packed
  // into rounds of disjoint pairs by a greedy edge colouring (a pair takes the first round
  // in which neither of its indices is used yet; pairs that find none of the 32 rounds
  // free wait for the next pass).  Any order that keeps visiting every entry above the
  // threshold converges (the threshold cyclic Jacobi with a skipped-rotation rule).
  const int m = n + (n & 1);
  const int half = m / 2;
  int sweeps = 0, capped = 0;
  for (int sweep = 0;; ++sweep) {
    // the entries above the threshold: counted per warp, then (a sparse pass) listed in a
    // fixed order, warp after warp, each warp's rows in order, so that the rotation order
    // and hence the rounding never depend on the scheduling
    {
      int cnt = 0;
      for (int i = ty; i < n; i += nty)
        for (int j0 = i + 1; j0 < n; j0 += 32) {
          const int j = j0 + tx;
          cnt += __popc(__ballot_sync(0xffffffffu, j < n && fabsf(A[i * ns + j]) > thr));
        }
      if (tx == 0) wcnt[ty] = cnt;
    }
    __syncthreads();
    if (tid == 0) {
      int s = 0;
      for (int w = 0; w < nty; ++w) {
        const int c = wcnt[w];
        wcnt[w] = s;
        s += c;
      }
      nbig = s;
    }
    __syncthreads();
    const int nlist = nbig;
    if (nlist == 0) break;
    const bool sparse = nlist <= min(RR_SPARSE, 2 * m);
    if (sparse) {
      int k = wcnt[ty];
      for (int i = ty; i < n; i += nty)
        for (int j0 = i + 1; j0 < n; j0 += 32) {
          const int j = j0 + tx;
          const bool big = j < n && fabsf(A[i * ns + j]) > thr;
          const unsigned bal = __ballot_sync(0xffffffffu, big);
          if (big) sp_list[k + __popc(bal & ((1u << tx) - 1u))] = i | (j << 10);
          k += __popc(bal);
        }
      __syncthreads();
    }
    if (sweep == max_sweeps) {  // still off-diagonal entries above the threshold
      capped = 1;
      break;
    }
    ++sweeps;
    if (sparse) {
      // schedule: round masks and stamps cleared, greedy colouring by one thread, then the
      // pairs bucketed by round (counts, scan, placement)
      for (int i = tid; i < n; i += nt) {
        ru.used[i] = 0u;
        sp_stamp[i] = 0;
      }
      if (tid < 33) sp_rstart[tid] = 0;
      __syncthreads();
      if (tid == 0) {
        int nr = 0;
        for (int k = 0; k < nlist; ++k) {
          const int e = sp_list[k];
          const int a = e & 1023, b = e >> 10;
          const unsigned fr = ~(ru.used[a] | ru.used[b]);
          if (fr == 0u) {
            sp_list[k] = -1;
            continue;
          }
          const int r = __ffs(fr) - 1;
          ru.used[a] |= 1u << r;
          ru.used[b] |= 1u << r;
          sp_list[k] = e | (r << 20);
          sp_rstart[r + 1] += 1;
          nr = max(nr, r + 1);
        }
        for (int r = 0; r < nr; ++r) sp_rstart[r + 1] += sp_rstart[r];
        sp_rounds = nr;
      }
      __syncthreads();
      if (tid < 32) {  // placement: one warp, pairs in list order within each round
        for (int k0 = 0; k0 < nlist; k0 += 32) {
          const int k = k0 + tid;
          const int e = k < nlist ? sp_list[k] : -1;
          const int r = e < 0 ? -1 : e >> 20;
          for (int rr = 0; rr < sp_rounds; ++rr) {
            const unsigned bal = __ballot_sync(0xffffffffu, r == rr);
            if (r == rr) sp_sorted[sp_rstart[rr] + __popc(bal & ((1u << tid) - 1u))] = e & 0xfffff;
            __syncwarp();
            if (tid == 0) sp_rstart[rr] += __popc(bal);
            __syncwarp();
          }
        }
        // (sp_rstart[r] now holds the end of round r; the start is the end of r - 1)
      }
      __syncthreads();
      const int nr = sp_rounds;
      for (int r = 0; r < nr; ++r) {
        const int b0 = r == 0 ? 0 : sp_rstart[r - 1], kr = sp_rstart[r] - b0;
        if (tid < kr) {
          const int e = sp_sorted[b0 + tid];
          const int pp = e & 1023, qq = e >> 10;
          float c = 1.f, s = 0.f;
          const float apq = A[pp * ns + qq];
          if (fabsf(apq) > thr) {
            const float tau = __fdividef(A[qq * ns + qq] - A[pp * ns + pp], 2.f * apq);
            const float t = copysignf(__fdividef(1.f, fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f))), tau);
            c = rsqrtf(fmaf(t, t, 1.f));
            s = t * c;
          }
          cs_c[tid] = c;
          cs_s[tid] = s;
          pr_p[tid] = pp;
          pr_q[tid] = qq;
          sp_stamp[pp] = (unsigned char)(r + 1);
          sp_stamp[qq] = (unsigned char)(r + 1);
        }
        __syncthreads();
        // 2x2 blocks between the round's pairs; pair rows against the other columns (row
        // rotation, mirrored into the symmetric column entries); V
        for (int P2 = ty; P2 < kr; P2 += nty) {
          const float sp = cs_s[P2], cp = cs_c[P2];
          const int p0 = pr_p[P2], p1 = pr_q[P2];
          for (int Q2 = tx; Q2 < kr; Q2 += 32) {
            const float sq = cs_s[Q2];
            if (sp == 0.f && sq == 0.f) continue;
            const float cq = cs_c[Q2];
            const int q0 = pr_p[Q2], q1 = pr_q[Q2];
            const float a00 = A[p0 * ns + q0], a01 = A[p0 * ns + q1];
            const float a10 = A[p1 * ns + q0], a11 = A[p1 * ns + q1];
            const float b00 = cp * a00 - sp * a10, b01 = cp * a01 - sp * a11;
            const float b10 = sp * a00 + cp * a10, b11 = sp * a01 + cp * a11;
            A[p0 * ns + q0] = cq * b00 - sq * b01;
            A[p0 * ns + q1] = sq * b00 + cq * b01;
            A[p1 * ns + q0] = cq * b10 - sq * b11;
            A[p1 * ns + q1] = sq * b10 + cq * b11;
          }
          if (sp == 0.f) continue;
          for (int j = tx; j < n; j += 32) {
            if (sp_stamp[j] == (unsigned char)(r + 1)) continue;
            const float a0 = A[p0 * ns + j], a1 = A[p1 * ns + j];
            const float b0 = cp * a0 - sp * a1, b1 = sp * a0 + cp * a1;
            A[p0 * ns + j] = b0;
            A[p1 * ns + j] = b1;
            A[j * ns + p0] = b0;
            A[j * ns + p1] = b1;
          }
          for (int i = tx; i < n; i += 32) {
            const float v0 = Vt[p0 * ns + i], v1 = Vt[p1 * ns + i];
            Vt[p0 * ns + i] = cp * v0 - sp * v1;
            Vt[p1 * ns + i] = sp * v0 + cp * v1;
          }
        }
        __syncthreads();
      }
      continue;
    }
    for (int r = 0; r < m - 1; ++r) {
      if (tid < half) {
        const int a = tid, b = m - 1 - tid;
        int ta = a - 1 + r, tb = b - 1 + r;  // (both < 2 (m - 1): one conditional subtraction)
        if (ta >= m - 1) ta -= m - 1;
        if (tb >= m - 1) tb -= m - 1;
        const int pa = a == 0 ? 0 : 1 + ta;
        const int pb = b == 0 ? 0 : 1 + tb;
        const int pp = min(pa, pb), qq = max(pa, pb);
        float c = 1.f, s = 0.f;
        if (qq < n) {
          const float apq = A[pp * ns + qq];
          if (fabsf(apq) > thr) {
            // (fast reciprocals: any orthogonal rotation near the exact one converges the sweep)
            const float tau = __fdividef(A[qq * ns + qq] - A[pp * ns + pp], 2.f * apq);
            const float t = copysignf(__fdividef(1.f, fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f))), tau);
            c = rsqrtf(fmaf(t, t, 1.f));
            s = t * c;
          }
        }
        cs_c[tid] = c;
        cs_s[tid] = s;
        pr_p[tid] = pp;
        pr_q[tid] = qq;
      }
      __syncthreads();
      // blocks (P, Q) with P <= Q, each written with its mirror (Q, P): the upper triangle
      // of the half x half block grid, folded so that block rows P and half - 1 - P share
      // one row of half + 1 items, dealt to all threads; rows / columns equal to n (the
      // odd dummy) are absent
      {
        const int wrow = half + 1, nitem = ((half + 1) / 2) * wrow;
        const float inv_wrow = 1.f / (float)wrow;
        for (int e = tid; e < nitem; e += nt) {
          int P2 = __float2int_rz(((float)e + 0.5f) * inv_wrow);
          int Q2 = e - P2 * wrow;  // (offset d in the folded row)
          if (Q2 < half - P2) {
            Q2 += P2;
          } else {
            const int P3 = half - 1 - P2;
            if (P3 == P2) continue;  // (odd half: the middle row holds only its own part)
            Q2 = P3 + Q2 - (half - P2);
            P2 = P3;
          }
          const float sp = cs_s[P2], sq = cs_s[Q2];
          if (sp == 0.f && sq == 0.f) continue;
          const float cp = cs_c[P2], cq = cs_c[Q2];
          const int p0 = pr_p[P2], p1 = pr_q[P2], q0 = pr_p[Q2], q1 = pr_q[Q2];
          const bool h1 = p1 < n, g1 = q1 < n;
          const float a00 = A[p0 * ns + q0];
          const float a01 = g1 ? A[p0 * ns + q1] : 0.f;
          const float a10 = h1 ? A[p1 * ns + q0] : 0.f;
          const float a11 = (h1 && g1) ? A[p1 * ns + q1] : 0.f;
          const float b00 = cp * a00 - sp * a10, b01 = cp * a01 - sp * a11;  // rows: J_P^T
          const float b10 = sp * a00 + cp * a10, b11 = sp * a01 + cp * a11;
          const float c00 = cq * b00 - sq * b01, c01 = sq * b00 + cq * b01;  // columns: J_Q
          const float c10 = cq * b10 - sq * b11, c11 = sq * b10 + cq * b11;
          A[p0 * ns + q0] = c00;
          if (g1) A[p0 * ns + q1] = c01;
          if (h1) A[p1 * ns + q0] = c10;
          if (h1 && g1) A[p1 * ns + q1] = c11;
          if (P2 != Q2) {
            A[q0 * ns + p0] = c00;
            if (g1) A[q1 * ns + p0] = c01;
            if (h1) A[q0 * ns + p1] = c10;
            if (h1 && g1) A[q1 * ns + p1] = c11;
          }
        }
      }
      // V_{:,Q} <- V_{:,Q} J_Q, (pair, row) items dealt to all threads
      {
        const int nitem = half * n;
        const float inv_n = 1.f / (float)n;
        for (int e = tid; e < nitem; e += nt) {
          const int Q2 = __float2int_rz(((float)e + 0.5f) * inv_n);
          const float sq = cs_s[Q2];
          if (sq == 0.f) continue;
          const float cq = cs_c[Q2];
          const int q0 = pr_p[Q2], q1 = pr_q[Q2], i = e - Q2 * n;
          const float v0 = Vt[q0 * ns + i], v1 = Vt[q1 * ns + i];
          Vt[q0 * ns + i] = cq * v0 - sq * v1;
          Vt[q1 * ns + i] = sq * v0 + cq * v1;
        }
      }
      __syncthreads();
    }
  }
  for (int j = tid; j < n; j += nt) {  // (a left-out direction ranks last)
    const float ej = dkv[j] == RR_DROPPED ? (float)RR_DROP_DIAG : A[j * ns + j];
    int rank = 0;
    for (int k2 = 0; k2 < n; ++k2) {
      const float ek = dkv[k2] == RR_DROPPED ? (float)RR_DROP_DIAG : A[k2 * ns + k2];
      rank += (ek < ej) || (ek == ej && k2 < j);
    }
    rr_out_eps(P, rank, (double)ej);
    P.bv[BV_TMP0 * P.nb + j] = (double)rank;  // (blk = 2: rows BV_TMP0 and BV_TMP1)
  }
  __syncthreads();
  for (int j = ty; j < n; j += nty) {
    const int rj = (int)P.bv[BV_TMP0 * P.nb + j];
    if (rj >= P.nb) continue;
    for (int i = tx; i < n; i += 32) rr_out_vec(P, i, rj, (double)Vt[j * ns + i]);
  }
  if (tid == 0) {
    P.scal[SC_RRSWEEPS] += sweeps;
    P.scal[SC_RRCAP] += capped;
    if (flag) P.status[0] = 1;
  }
}

// ---------------------------------------------------------------------------
// Rayleigh-Ritz for subspaces too large for one CTA's shared memory (the 330-band cluster):
// one thread-block cluster of RR_CLUSTER CTAs per problem, its matrices in the problem's
// global scratch (L2-resident), row i dealt to the CTA of rank i % RR_CLUSTER, hardware
// cluster barriers between the steps.  Same mathematics as k_rr_f32 (deviation form):
//  1. D = S - I and Hf, symmetrised.
//  2. Cholesky S = (I + L)(I + L)^T in deviation form: column k's pivot d_k and scaled
//     entries are formed by every CTA from the column (final after step k - 1), and each
//     CTA updates its own trailing rows: one barrier per column.
//  3. (I + L)^-1 = I + G by forward substitution down each column of G, a warp per column
//     (the columns are independent), stored transposed (GT row j = column j of G).
//  4. C = (I + G) Hf (I + G)^T, symmetrised; V = (I + G)^T.
//  5. Eigenvectors by one-sided Jacobi (Hestenes, J. SIAM 6, 51 (1958)) on
//     X = C - sigma I, sigma below the Gershgorin bound of C's spectrum, so that X is
//     positive definite and its right singular vectors are C's eigenvectors: in each
//     round-robin round every CTA sums the three dot products of every column pair over
//     its rows (FP64 partials), one barrier, and every CTA forms the same rotations from
//     the partials added in rank order and rotates its rows of X and V.  A sweep without a
//     rotation above the rounding threshold ends the loop; max_sweeps caps it (counted in
//     SC_RRCAP).
//  6. eps_j = |x_j| + sigma (|x_j| = eps_j - sigma for the unit eigenvector), ascending
//     ranks, Tm[:, rank(j)] = V[:, j].
// ---------------------------------------------------------------------------
// Sums of the Jacobi's column dot products: float-float on the FP32 path (FP64 runs at
// about 1/64 of the FP32 rate on this GPU), FP64 on the FP64 path; the rotation angles in
// the working precision.
template <typename T>
struct JacSum;
template <>
struct JacSum<float> {
  using A = ff;
  static constexpr float cosine = 3e-6f;  // column-pair cosine below which no rotation is made
  static __device__ __forceinline__ A zero() { return ff(0.f, 0.f); }
  static __device__ __forceinline__ A prod(float a, float b) {
    const float p = mul_rn(a, b);
    return ff(p, fmaf(a, b, -p));
  }
  static __device__ __forceinline__ A shfl(A v, int o) {
    return ff(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
  }
  static __device__ __forceinline__ float val(A v) { return v.hi + v.lo; }
};
template <>
struct JacSum<double> {
  using A = double;
  static constexpr double cosine = 1e-13;
  static __device__ __forceinline__ A zero() { return 0.0; }
  static __device__ __forceinline__ A prod(double a, double b) { return a * b; }
  static __device__ __forceinline__ A shfl(A v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
  static __device__ __forceinline__ double val(A v) { return v; }
};

size_t rr_cluster_scratch_bytes(int n, size_t tsize) {
  const size_t nn = (size_t)n * n, npairs = (size_t)(n + (n & 1)) / 2;
  return 5 * nn * tsize + 256 + (2 * RR_CLUSTER * npairs * 3 + RR_CLUSTER * (size_t)n + 2 * RR_CLUSTER + n) * 8 + 256;
}

template <typename T>
__global__ void __launch_bounds__(RR_THREADS) k_rr_cluster(KArgs ka, unsigned char* scratch_base, size_t stride,
                                                           int max_sweeps, int rows_smem, int blk) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  constexpr int C = RR_CLUSTER;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[33];
  __shared__ int flag_s, rot_s;
  const int p = blockIdx.x / C;
  const int rank = (int)cluster.block_rank();
  if (!ka.active[p]) return;  // the whole cluster shares p
  const Prob& P = ka.probs[p];
  const int n = blk * P.nb, m = n + (n & 1), npairs = m / 2;
  const double* Sin = rr_in_s(P, blk);
  const double* Hin = rr_in_h(P, blk);
  const size_t nn = (size_t)n * n;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  // global scratch of this problem
  unsigned char* base = scratch_base + (size_t)p * stride;
  T* Dm = reinterpret_cast<T*>(base);  // Cholesky working matrix, then X
  T* Hm = Dm + nn;                     // Hf, then C
  T* Lm = Hm + nn;                     // scaled Cholesky columns, then V
  T* GT = Lm + nn;                     // G transposed
  T* Wm = GT + nn;                     // (I + G) Hf
  double* part = reinterpret_cast<double*>(base + ((5 * nn * sizeof(T) + 255) / 256) * 256);  // [2][C][npairs][3]
  double* colp = part + 2 * (size_t)C * npairs * 3;  // [C][n] column partial sums
  double* gpart = colp + (size_t)C * n;              // [C] Gershgorin minima, [C] flags
  double* dkv = gpart + 2 * C;                       // [n] pivots d_k
  // shared memory: column k of the Cholesky, the rotations and pairs, and (rows_smem) the
  // Jacobi's rows of X and V, else those rows stay in the global X (Dm) and V (Lm);
  // eigenvalues and ranks at the end
  const int myrows = (n - rank + C - 1) / C;  // rows rank, rank + C, ...
  const int myrows_max = (n + C - 1) / C;
  T* colk = reinterpret_cast<T*>(smem_raw);   // [n]
  T* csc = colk + n;                          // [npairs]
  T* css = csc + npairs;                      // [npairs]
  int* pp = reinterpret_cast<int*>(css + npairs);  // [npairs]
  int* pq = pp + npairs;                           // [npairs]
  T* const xbase = reinterpret_cast<T*>(smem_raw + (((size_t)(n + 2 * npairs) * sizeof(T) + 2 * npairs * sizeof(int) +
                                                      15) / 16) * 16);
  // row r of mine: i = rank + C r; rows in shared memory have the odd stride n | 1, so that
  // a warp walking down a column meets distinct banks
  const int ls = n | 1;
  auto xrow = [&](int r) -> T* { return rows_smem ? xbase + (size_t)r * ls : Dm + (size_t)(rank + C * r) * n; };
  auto vrow = [&](int r) -> T* {
    return rows_smem ? xbase + (size_t)(myrows_max + r) * ls : Lm + (size_t)(rank + C * r) * n;
  };
  double* lam = reinterpret_cast<double*>(xbase);  // [n] (reuses the rows after the Jacobi)
  int* rnk = reinterpret_cast<int*>(lam + n);      // [n]
  if (tid == 0) flag_s = 0;

  // 1. D = S - I, Hf (symmetrised), my rows
  for (int e = tid; e < myrows * n; e += nt) {
    const int i = rank + C * (e / n), j = e % n;
    Dm[(size_t)i * n + j] = (T)(0.5 * (Sin[i * n + j] + Sin[j * n + i]) - (i == j ? 1.0 : 0.0));
    Hm[(size_t)i * n + j] = (T)(0.5 * (Hin[i * n + j] + Hin[j * n + i]));
  }
  cluster.sync();

  // 2. Cholesky in deviation form
  // (a left-out direction of the block [X, W]: zero scaled column, no update, pivot mark
  // RR_DROPPED in dkv)
  for (int k = 0; k < n; ++k) {
    const T x = Dm[(size_t)k * n + k];
    const bool drop = blk == 2 && k >= P.nb && x <= T(RR_DROP) - T(1);
    const T xs = drop ? T(0) : (x > T(-0.999) ? x : T(-0.999));
    const T dk = xs / (T(1) + sqrt(T(1) + xs));
    const T inv = drop ? T(0) : T(1) / (T(1) + dk);
    if (tid == 0) {
      if (!drop && !(x > T(-0.999))) flag_s = 1;
      if (rank == 0) dkv[k] = drop ? (double)RR_DROPPED : (double)dk;
    }
    for (int j = k + 1 + tid; j < n; j += nt) colk[j] = Dm[(size_t)j * n + k] * inv;
    __syncthreads();
    const int r0 = (k + 1 - rank + C - 1) / C > 0 ? (k + 1 - rank + C - 1) / C : 0;  // first my row > k
    const T* __restrict__ ck = colk;
    for (int r = r0 + warp; r < myrows; r += nwarps) {
      const int i = rank + C * r;
      const T li = ck[i];
      if (lane == 0) Lm[(size_t)i * n + k] = li;
      T* __restrict__ Di = Dm + (size_t)i * n;
#pragma unroll 4
      for (int j = k + 1 + lane; j <= i; j += 32) Di[j] -= li * ck[j];
    }
    cluster.sync();
  }

  // 3. G by columns: GT[j][i] = G_ij, G_jj = -d_j / (1 + d_j),
  //    G_ij = -(L_ij + sum_{j <= k < i} L_ik G_kj) / (1 + d_i)
  //    (a left-out direction's row of I + G is zero: G_jj = -1, G_ij = 0)
  for (int j = rank * nwarps + warp; j < n; j += C * nwarps) {
    T* gj = GT + (size_t)j * n;
    const T dj = (T)dkv[j];
    if (lane == 0) gj[j] = dkv[j] == (double)RR_DROPPED ? T(-1) : -dj / (T(1) + dj);
    __syncwarp();
    for (int i = j + 1; i < n; ++i) {
      const T* Li = Lm + (size_t)i * n;
      T sacc = T(0);
      for (int k = j + lane; k < i; k += 32) sacc += Li[k] * gj[k];
      for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
      if (lane == 0) gj[i] = dkv[i] == (double)RR_DROPPED ? T(0) : -(Li[j] + sacc) / (T(1) + (T)dkv[i]);
      __syncwarp();
    }
  }
  cluster.sync();

  // 4. W = (I + G) Hf: W_ij = Hf_ij + sum_{k <= i} G_ik Hf_kj
  for (int e = tid; e < myrows * n; e += nt) {
    const int i = rank + C * (e / n), j = e % n;
    const T* __restrict__ gi = GT + i;   // G_ik = GT[k][i]
    const T* __restrict__ hj = Hm + j;   // Hf_kj
    T acc = hj[(size_t)i * n], acc2 = T(0);
#pragma unroll 4
    for (int k = 0; k <= i; k += 2) {
      acc += gi[(size_t)k * n] * hj[(size_t)k * n];
      if (k + 1 <= i) acc2 += gi[(size_t)(k + 1) * n] * hj[(size_t)(k + 1) * n];
    }
    Wm[(size_t)i * n + j] = acc + acc2;
  }
  cluster.sync();
  //    C = W (I + G)^T: C_ij = W_ij + sum_{k <= j} W_ik G_jk  (into Hm)
  for (int e = tid; e < myrows * n; e += nt) {
    const int i = rank + C * (e / n), j = e % n;
    const T* __restrict__ Wi = Wm + (size_t)i * n;
    const T* __restrict__ gj = GT + j;   // G_jk = GT[k][j]
    T acc = Wi[j], acc2 = T(0);
#pragma unroll 4
    for (int k = 0; k <= j; k += 2) {
      acc += Wi[k] * gj[(size_t)k * n];
      if (k + 1 <= j) acc2 += Wi[k + 1] * gj[(size_t)(k + 1) * n];
    }
    Hm[(size_t)i * n + j] = acc + acc2;
  }
  cluster.sync();
  //    X = sym(C) (into Dm), V = (I + G)^T (into Lm), Gershgorin minimum of my rows
  double gmin = 1e300;
  for (int r = warp; r < myrows; r += nwarps) {
    const int i = rank + C * r;
    double off = 0.0, dia = 0.0;
    for (int j = lane; j < n; j += 32) {
      const T v = T(0.5) * (Hm[(size_t)i * n + j] + Hm[(size_t)j * n + i]);
      Dm[(size_t)i * n + j] = v;
      Lm[(size_t)i * n + j] = (i == j ? T(1) : T(0)) + GT[(size_t)i * n + j];
      if (j == i) dia = (double)v; else off += fabs((double)v);
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      dia += __shfl_xor_sync(0xffffffffu, dia, o);
    }
    gmin = fmin(gmin, dia - off);
  }
  if (lane == 0) red[warp] = gmin;
  __syncthreads();
  if (tid == 0) {
    double g = 1e300;
    for (int w = 0; w < nwarps; ++w) g = fmin(g, red[w]);
    gpart[rank] = g;
    gpart[C + rank] = flag_s;
  }
  cluster.sync();
  double sigma = 1e300;
  int flag = 0;
  for (int r = 0; r < C; ++r) {
    sigma = fmin(sigma, gpart[r]);
    flag |= gpart[C + r] != 0.0;
  }
  sigma -= 1e-3 * (1.0 + fabs(sigma));
  // my rows of X - sigma I and V (into shared memory when they fit)
  for (int e = tid; e < myrows * n; e += nt) {
    const int r = e / n, j = e % n, i = rank + C * r;
    const T v = Dm[(size_t)i * n + j];
    xrow(r)[j] = i == j ? (T)((double)v - sigma) : v;
    if (rows_smem) vrow(r)[j] = Lm[(size_t)i * n + j];
  }
  __syncthreads();

  // 5. one-sided Jacobi, round-robin column pairs (position 0 fixed, 1..m-1 rotating)
  int sweeps = 0, capped = 0, round = 0;
  for (int sweep = 0;; ++sweep) {
    if (tid == 0) rot_s = 0;
    __syncthreads();
    for (int rr = 0; rr < m - 1; ++rr, ++round) {
      for (int t = tid; t < npairs; t += nt) {
        const int a = t, b = m - 1 - t;
        const int pa = a == 0 ? 0 : 1 + (a - 1 + rr) % (m - 1);
        const int pb = b == 0 ? 0 : 1 + (b - 1 + rr) % (m - 1);
        pp[t] = min(pa, pb);
        pq[t] = max(pa, pb);
      }
      __syncthreads();
      using JS = JacSum<T>;
      using A = typename JS::A;
      A* pr = reinterpret_cast<A*>(part) + ((size_t)(round & 1) * C + rank) * npairs * 3;
      // a quad of lanes per pair, each summing a quarter of my rows
      const int npq = (npairs + 7) / 8 * 8;  // pairs padded so that every warp holds whole quads
      for (int t4 = tid; t4 < 4 * npq; t4 += nt) {
        const int t = t4 >> 2, qd = t4 & 3;
        const bool live = t < npairs && pq[t] < n;
        const int a = live ? pp[t] : 0, b = live ? pq[t] : 0;
        A al = JS::zero(), be = JS::zero(), ga = JS::zero();
        if (live)
          for (int r = qd; r < myrows; r += 4) {
            const T* xr = xrow(r);
            const T xa = xr[a], xb = xr[b];
            al = al + JS::prod(xa, xa);
            be = be + JS::prod(xb, xb);
            ga = ga + JS::prod(xa, xb);
          }
        for (int o = 1; o < 4; o <<= 1) {
          al = al + JS::shfl(al, o);
          be = be + JS::shfl(be, o);
          ga = ga + JS::shfl(ga, o);
        }
        if (qd == 0 && t < npairs) {
          pr[3 * t] = al;
          pr[3 * t + 1] = be;
          pr[3 * t + 2] = ga;
        }
      }
      cluster.sync();
      const A* pb0 = reinterpret_cast<const A*>(part) + (size_t)(round & 1) * C * npairs * 3;
      for (int t = tid; t < npairs; t += nt) {
        A al = JS::zero(), be = JS::zero(), ga = JS::zero();
        for (int r = 0; r < C; ++r) {
          const A* q = pb0 + ((size_t)r * npairs + t) * 3;
          al = al + q[0];
          be = be + q[1];
          ga = ga + q[2];
        }
        const T alv = (T)JS::val(al), bev = (T)JS::val(be), gav = (T)JS::val(ga);
        T c = T(1), sn = T(0);
        if (pq[t] < n && fabs(gav) > (T)JS::cosine * sqrt(alv * bev) && gav != T(0)) {
          const T zeta = (bev - alv) / (T(2) * gav);
          const T tt = (zeta >= T(0) ? T(1) : T(-1)) / (fabs(zeta) + sqrt(T(1) + zeta * zeta));
          c = T(1) / sqrt(T(1) + tt * tt);
          sn = c * tt;
          rot_s = 1;
        }
        csc[t] = c;
        css[t] = sn;
      }
      __syncthreads();
      for (int e = tid; e < npairs * myrows; e += nt) {
        const int t = e / myrows, r = e - t * myrows;
        const T sn = css[t];
        if (sn == T(0)) continue;
        const T c = csc[t];
        const int a = pp[t], b = pq[t];
        T* xr = xrow(r);
        T* vr = vrow(r);
        const T xa = xr[a], xb = xr[b], va = vr[a], vb = vr[b];
        xr[a] = c * xa - sn * xb;
        xr[b] = sn * xa + c * xb;
        vr[a] = c * va - sn * vb;
        vr[b] = sn * va + c * vb;
      }
      __syncthreads();
    }
    ++sweeps;
    if (rot_s == 0) break;
    if (sweep + 1 == max_sweeps) {
      capped = 1;
      break;
    }
  }

  // 6. eigenvalues from the column norms, ranks, Tm and eps
  for (int j = tid; j < n; j += nt) {
    double sq = 0.0;
    for (int r = 0; r < myrows; ++r) {
      const double v = (double)xrow(r)[j];
      sq += v * v;
    }
    colp[(size_t)rank * n + j] = sq;
  }
  // V rows to global before the shared memory is reused
  if (rows_smem)
    for (int e = tid; e < myrows * n; e += nt) Lm[(size_t)(rank + C * (e / n)) * n + e % n] = vrow(e / n)[e % n];
  cluster.sync();
  for (int j = tid; j < n; j += nt) {  // (a left-out direction ranks last)
    double sq = 0.0;
    for (int r = 0; r < C; ++r) sq += colp[(size_t)r * n + j];
    lam[j] = dkv[j] == (double)RR_DROPPED ? RR_DROP_DIAG : sqrt(sq) + sigma;
  }
  __syncthreads();
  for (int j = tid; j < n; j += nt) {
    const double ej = lam[j];
    int rk = 0;
    for (int k2 = 0; k2 < n; ++k2) {
      const double ek = lam[k2];
      rk += (ek < ej) || (ek == ej && k2 < j);
    }
    rnk[j] = rk;
    if (rank == 0) rr_out_eps(P, rk, ej);
  }
  __syncthreads();
  for (int e = tid; e < myrows * n; e += nt) {
    const int i = rank + C * (e / n), j = e % n;
    if (i < n) rr_out_vec(P, i, rnk[j], (double)Lm[(size_t)i * n + j]);
  }
  if (rank == 0 && tid == 0) {
    P.scal[SC_RRSWEEPS] += sweeps;
    P.scal[SC_RRCAP] += capped;
    if (flag) P.status[0] = 1;
  }
  cluster.sync();  // no CTA leaves while another may still read its shared memory (none does) or scratch
}

// Shared memory of the cluster Rayleigh-Ritz for subspace size n: the head (column k,
// rotations, pairs), then either the rows of X and V (rows_smem) or the final eigenvalues
// and ranks, whichever is larger.
static size_t rr_cluster_smem_t(int n, size_t tsize, bool rows_smem) {
  const size_t myrows = (n + RR_CLUSTER - 1) / RR_CLUSTER, npairs = (n + (n & 1)) / 2;
  const size_t head = ((n + 2 * npairs) * tsize + 2 * npairs * sizeof(int) + 15) / 16 * 16;
  const size_t rows = rows_smem ? 2 * myrows * (size_t)(n | 1) * tsize : 0;
  const size_t fin = (size_t)n * (sizeof(double) + sizeof(int));
  return head + std::max(rows, fin) + 16;
}
static bool rr_cluster_rows_fit(int n, size_t tsize) { return rr_cluster_smem_t(n, tsize, true) <= 200 * 1024; }
size_t rr_cluster_smem(int n) { return rr_cluster_smem_t(n, 4, rr_cluster_rows_fit(n, 4)); }
size_t rr_cluster_smem64(int n) { return rr_cluster_smem_t(n, 8, rr_cluster_rows_fit(n, 8)); }

template <typename T>
bool launch_rr_cluster(const Launch& L, int n_max, unsigned char* scratch, size_t stride, int max_sweeps, int blk) {
  const bool rows_smem = rr_cluster_rows_fit(n_max, sizeof(T));
  const size_t smem = rr_cluster_smem_t(n_max, sizeof(T), rows_smem);
  if (smem > 227 * 1024) return false;
  cudaFuncSetAttribute(k_rr_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(L.ka.nprob * RR_CLUSTER);
  cfg.blockDim = dim3(RR_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = L.stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = RR_CLUSTER;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_rr_cluster<T>, L.ka, scratch, stride, max_sweeps, rows_smem ? 1 : 0, blk) ==
         cudaSuccess;
}
template bool launch_rr_cluster<float>(const Launch&, int, unsigned char*, size_t, int, int);
template bool launch_rr_cluster<double>(const Launch&, int, unsigned char*, size_t, int, int);

// ---------------------------------------------------------------------------
// Occupations: integer (kT = 0) or Fermi-Dirac with mu from sum f = N_el; entropy
// S = -2 sum [x ln x + (1-x) ln(1-x)], x = f/2.  One warp per problem.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double fd_x(double e, double mu, double kT) {
  double a = (e - mu) / kT;
  if (a > 700.0) return 0.0;
  if (a < -700.0) return 1.0;
  return 1.0 / (1.0 + exp(a));
}

__global__ void k_occupations(KArgs ka) {
  const int p = blockIdx.x;
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  // occupations over the nbo requested bands; the eigensolver's extra bands above them
  // stay empty
  const int n = P.nbo, lane = threadIdx.x;
  const double kT = P.kT, nel = P.nel;
  const double* eps = P.eps;
  for (int i = n + lane; i < P.nb; i += 32) P.occ[i] = 0.0;
  if (kT <= 0.0) {
    const int nocc = (int)llround(nel * 0.5);
    for (int i = lane; i < n; i += 32) P.occ[i] = i < nocc ? 2.0 : 0.0;
    if (lane == 0) {
      P.scal[SC_MU] = nocc < n ? 0.5 * (eps[nocc - 1] + eps[nocc]) : eps[n - 1];
      P.scal[SC_ENTROPY] = 0.0;
    }
    return;
  }
  double lo = eps[0] - 40.0 * kT - 1.0, hi = eps[n - 1] + 40.0 * kT + 1.0;
  double mu = 0.5 * (lo + hi);
  for (int it = 0; it < 200; ++it) {
    double cnt = 0.0, der = 0.0;
    for (int i = lane; i < n; i += 32) {
      double x = fd_x(eps[i], mu, kT);
      cnt += 2.0 * x;
      der += 2.0 * x * (1.0 - x) / kT;
    }
    cnt = warp_sum(cnt);
    der = warp_sum(der);
    double diff = cnt - nel;
    if (fabs(diff) < 1e-13 * fmax(1.0, nel)) break;
    if (diff < 0.0) lo = mu; else hi = mu;
    double nmu = der > 0.0 ? mu - diff / der : 0.5 * (lo + hi);
    if (!(nmu > lo && nmu < hi)) nmu = 0.5 * (lo + hi);
    if (hi - lo < 1e-15 * fmax(1.0, fabs(mu))) break;
    mu = nmu;
  }
  double ent = 0.0;
  for (int i = lane; i < n; i += 32) {
    double x = fd_x(eps[i], mu, kT);
    P.occ[i] = 2.0 * x;
    if (x > 0.0) ent += x * log(x);
    if (x < 1.0) ent += (1.0 - x) * log1p(-x);
  }
  ent = warp_sum(ent);
  if (lane == 0) {
    P.scal[SC_MU] = mu;
    P.scal[SC_ENTROPY] = -2.0 * ent;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename T>
void launch_gemm_tn(const Launch& L, int akind, int arole, int bkind, int brole, double* part, size_t stride,
                    int kc) {
  if (!L.map.total) return;
  k_gemm_tn<T><<<L.map.total, 256, 0, L.stream>>>(L.ka, akind, arole, bkind, brole, part, stride, kc);
}
void launch_gemm_tn_reduce(const Launch& L, int akind, int bkind, int dst, const double* part, size_t stride, int kc,
                           bool sym) {
  if (!L.map.total) return;
  k_gemm_tn_reduce<<<L.map.total, 256, 0, L.stream>>>(L.ka, akind, bkind, dst, part, stride, kc, sym ? 1 : 0);
}
template <typename T>
void launch_gemm_nn(const Launch& L, int akind, const RolePairs& rp, int msel, double alpha, double beta) {
  if (!L.map.total || rp.n < 1) return;
  k_gemm_nn<T><<<dim3(L.map.total, rp.n), 256, (size_t)NN_KP * 64 * sizeof(T), L.stream>>>(L.ka, akind, rp, msel, alpha,
                                                                               beta);
}
template <typename T>
void launch_band_kinetic(const Launch& L, int xrole) {
  if (!L.map.total) return;
  k_band_kinetic<T><<<L.map.total, BAND_THREADS, 0, L.stream>>>(L.ka, xrole);
}
template <typename T>
void launch_band_residual(const Launch& L, int xrole, int hxrole) {
  if (!L.map.total) return;
  k_band_residual<T><<<L.map.total, BAND_THREADS, 0, L.stream>>>(L.ka, xrole, hxrole);
}
template <typename T>
void launch_cg_precond(const Launch& L, int x, int hx, int p, int r, int pp, int rp) {
  if (!L.map.total) return;
  k_cg_precond<T><<<L.map.total, BAND_THREADS, 0, L.stream>>>(L.ka, x, hx, p, r, pp, rp);
}
template <typename T>
void launch_normalize(const Launch& L, int p, int pp) {
  if (!L.map.total) return;
  k_normalize<T><<<L.map.total, BAND_THREADS, 0, L.stream>>>(L.ka, p, pp);
}
template <typename T>
void launch_line_min(const Launch& L, int x, int hx, int p, int hp) {
  if (!L.map.total) return;
  k_line_min<T><<<L.map.total, BAND_THREADS, 0, L.stream>>>(L.ka, x, hx, p, hp);
}
template <typename T>
void launch_random_init(const Launch& L, int xrole, unsigned long long seed) {
  if (!L.map.total) return;
  k_random_init<T><<<L.map.total, 256, 0, L.stream>>>(L.ka, xrole, seed);
}
template <typename T>
void launch_copy_in(const Launch& L, int role, const double* src, int nvec, bool keep_tail) {
  if (!L.map.total) return;
  k_copy_in<T><<<L.map.total, 256, 0, L.stream>>>(L.ka, role, src, nvec, keep_tail ? 1 : 0);
}
template <typename T>
void launch_copy_out(const Launch& L, int role, double* dst, int nvec) {
  if (!L.map.total) return;
  k_copy_out<T><<<L.map.total, 256, 0, L.stream>>>(L.ka, role, dst, nvec);
}
void launch_rr_f32(const Launch& L, size_t smem, float* gscratch, size_t gstride, int max_sweeps, int blk) {
  k_rr_f32<<<L.ka.nprob, RR_THREADS, gscratch ? 0 : smem, L.stream>>>(L.ka, gscratch, gstride, max_sweeps, blk);
}
void launch_rr(const Launch& L, int use_smem, size_t smem, double* gscratch, size_t gstride, int max_sweeps,
               int blk) {
  k_rr<<<L.ka.nprob, RR_THREADS, use_smem ? smem : 0, L.stream>>>(L.ka, use_smem, gscratch, gstride, max_sweeps,
                                                                     blk);
}
// S2 and H2 of the block [X, W] from n_b x n_b products (block Davidson): part 0 takes
// S = X^T X, Hs = X^T HX, Tm = X^T W, Cm = X^T HW (the X rows and, by symmetry, the X
// columns); part 1 takes S = W^T W, Hs = W^T HW (the W W block).  CTA = (problem, 256
// entries of the n_b x n_b block).
__global__ void k_rr2_assemble(KArgs ka, int part) {
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int nb = P.nb, n2 = 2 * nb;
  const int e = (blockIdx.x - ka.start[p]) * 256 + threadIdx.x;
  if (e >= nb * nb) return;
  const int i = e / nb, j = e % nb;
  if (part == 0) {
    P.S2[(size_t)i * n2 + j] = P.S[e];
    P.H2[(size_t)i * n2 + j] = P.Hs[e];
    P.S2[(size_t)i * n2 + nb + j] = P.Tm[e];
    P.S2[(size_t)(nb + j) * n2 + i] = P.Tm[e];
    P.H2[(size_t)i * n2 + nb + j] = P.Cm[e];
    P.H2[(size_t)(nb + j) * n2 + i] = P.Cm[e];
  } else {
    P.S2[(size_t)(nb + i) * n2 + nb + j] = P.S[e];
    P.H2[(size_t)(nb + i) * n2 + nb + j] = P.Hs[e];
  }
}
void launch_rr2_assemble(const Launch& L, int part) {
  if (!L.map.total) return;
  k_rr2_assemble<<<L.map.total, 256, 0, L.stream>>>(L.ka, part);
}
void launch_occupations(const Launch& L) { k_occupations<<<L.ka.nprob, 32, 0, L.stream>>>(L.ka); }
void linalg_set_smem_limits(size_t bytes) {
  cudaFuncSetAttribute(k_rr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  // (k_rr_f32 keeps its matrices in shared memory up to 216 KB; its static arrays take the
  // rest of the 227 KB)
  cudaFuncSetAttribute(k_rr_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::min(bytes, (size_t)216 * 1024));
  // the NN kernel also has 8-16 KB of static shared memory: request only what it uses
  cudaFuncSetAttribute(k_gemm_nn<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, NN_KP * 64 * (int)sizeof(float));
  cudaFuncSetAttribute(k_gemm_nn<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, NN_KP * 64 * (int)sizeof(double));
}

#define INST(T)                                                                                  \
  template void launch_gemm_tn<T>(const Launch&, int, int, int, int, double*, size_t, int);     \
  template void launch_gemm_nn<T>(const Launch&, int, const RolePairs&, int, double, double);     \
  template void launch_band_kinetic<T>(const Launch&, int);                                     \
  template void launch_band_residual<T>(const Launch&, int, int);                               \
  template void launch_cg_precond<T>(const Launch&, int, int, int, int, int, int);              \
  template void launch_normalize<T>(const Launch&, int, int);                                   \
  template void launch_line_min<T>(const Launch&, int, int, int, int);                          \
  template void launch_random_init<T>(const Launch&, int, unsigned long long);                  \
  template void launch_copy_in<T>(const Launch&, int, const double*, int, bool);                \
  template void launch_copy_out<T>(const Launch&, int, double*, int);
INST(float)
INST(double)
#undef INST

}  // namespace sgo
