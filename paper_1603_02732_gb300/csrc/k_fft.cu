// FFT kernels of the all-band H.psi apply (every H|Psi_i> product of Algorithm 1) and
// of the density (Sec. II D: rho_out from the occupied states).
//
// A band pair (a, b) shares one complex transform: psi_a + i psi_b is real-space
// complex, both bands being real at the Gamma point.  The inverse transform runs
//   sphere -> compact z-columns (z FFT) -> per z-plane: y FFT on the occupied x rows,
//   x FFT on all columns, times V_eff(r)/N, x FFT back, y FFT back -> z-columns ->
//   z FFT back -> sphere, where (V psi_a)(G) = (F(G) + F(-G)^*)/2 and
//   (V psi_b)(G) = (F(G) - F(-G)^*)/(2i).
// The grid kernels at the end transform full FP64 complex grids (densities,
// potentials) with the same line engine.
#include "fft.cuh"
#include "kernels.h"

namespace sgo {

namespace {

// Working type T and the type S its grids and root tables are stored in: the same for
// float and double; float-float works on FP64 data (converted on load and store).
template <typename T>
struct Work {
  using S = T;
  static __device__ __forceinline__ cplx<T> in(cplx<S> v) { return v; }
  static __device__ __forceinline__ cplx<S> out(cplx<T> v) { return v; }
};
template <>
struct Work<ff> {
  using S = double;
  static __device__ __forceinline__ cplx<ff> in(cplx<double> v) { return mk(ff_from(v.x), ff_from(v.y)); }
  static __device__ __forceinline__ cplx<double> out(cplx<ff> v) { return mk(ff_to(v.x), ff_to(v.y)); }
};

template <typename S>
struct RootsOf;
template <>
struct RootsOf<float> {
  static __device__ __forceinline__ const cplx<float>* get(const Prob& P) {
    return reinterpret_cast<const cplx<float>*>(P.roots32);
  }
};
template <>
struct RootsOf<double> {
  static __device__ __forceinline__ const cplx<double>* get(const Prob& P) {
    return reinterpret_cast<const cplx<double>*>(P.roots64);
  }
};

template <typename T>
__device__ __forceinline__ void load_roots(cplx<T>* dst, const Prob& P, int off, int n) {
  const auto* src = RootsOf<typename Work<T>::S>::get(P) + off;
  for (int t = threadIdx.x; t < n; t += blockDim.x) dst[t] = Work<T>::in(src[t]);
}

__device__ __forceinline__ int wrapi(int m, int n) {
  int r = m % n;
  return r < 0 ? r + n : r;
}

// Column-pair chunk [cp0, cp1) -> compact columns [col0, col1).
__device__ __forceinline__ void chunk_cols(int cp0, int cp1, int* col0, int* col1) {
  *col0 = cp0 == 0 ? 0 : 2 * cp0 - 1;
  *col1 = 2 * cp1 - 1;
}

}  // namespace

// ---------------------------------------------------------------------------
// sphere -> compact z-columns (inverse z FFT).  CTA = (problem, band pair, chunk).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(ZCOL_THREADS) k_wave_to_cols(KArgs ka, int src) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int local = blockIdx.x - ka.start[p];
  const int nchunk = (P.ncp + QCP - 1) / QCP;
  const int pair = local / nchunk;
  const int chunk = local - pair * nchunk;
  const int n3 = P.n3;
  const int cp0 = chunk * QCP, cp1 = min(cp0 + QCP, P.ncp);
  int col0, col1;
  chunk_cols(cp0, cp1, &col0, &col1);
  const int ncl = col1 - col0;
  cplx<T>* lines = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* alt = lines + 2 * QCP * n3;
  cplx<T>* roots = alt + 2 * QCP * n3;
  load_roots<T>(roots, P, P.n1 + P.n2, n3);
  for (int t = threadIdx.x; t < ncl * n3; t += blockDim.x) lines[t] = mk(T(0), T(0));
  __syncthreads();

  const int ia = 2 * pair, ib = 2 * pair + 1;
  const bool hasb = ib < P.nb;
  const T* xa = wbuf<T>(P, src) + (size_t)ia * P.ld;
  const T* xb = wbuf<T>(P, src) + (size_t)(hasb ? ib : ia) * P.ld;
  const T rs2 = T(1.0 / SQRT2);
  const int e0 = P.cp_off[cp0], e1 = P.cp_off[cp1];
  for (int k = e0 + threadIdx.x; k < e1; k += blockDim.x) {
    int cp = cp0;
    while (P.cp_off[cp + 1] <= k) ++cp;
    const int m3 = P.ent_m3[k];
    cplx<T> ca = mk(xa[1 + 2 * k] * rs2, xa[2 + 2 * k] * rs2);
    cplx<T> cb = hasb ? mk(xb[1 + 2 * k] * rs2, xb[2 + 2 * k] * rs2) : mk(T(0), T(0));
    cplx<T> vp = mk(ca.x - cb.y, ca.y + cb.x);   // c_a(G) + i c_b(G)
    cplx<T> vm = mk(ca.x + cb.y, -ca.y + cb.x);  // c_a(G)^* + i c_b(G)^*  (value at -G)
    int lp, lm;
    if (cp == 0) { lp = 0; lm = 0; }
    else { lp = 2 * cp - 1 - col0; lm = 2 * cp - col0; }
    lines[lp * n3 + wrapi(m3, n3)] = vp;
    lines[lm * n3 + wrapi(-m3, n3)] = vm;
  }
  if (cp0 == 0 && threadIdx.x == 0) {
    lines[0] = mk(xa[0], hasb ? xb[0] : T(0));
  }
  __syncthreads();
  const cplx<T>* res = fft_lines<T>(lines, alt, ncl, n3, 1, contiguous(ncl), P.fd[2], roots, T(1));
  cplx<T>* wc = reinterpret_cast<cplx<T>*>(P.Wc) + (size_t)pair * n3 * P.ncol;
  for (int t = threadIdx.x; t < ncl * n3; t += blockDim.x) {
    int z = t / ncl, c = t - z * ncl;
    wc[(size_t)z * P.ncol + col0 + c] = res[c * n3 + z];
  }
}

// ---------------------------------------------------------------------------
// compact z-columns -> sphere (forward z FFT), band separation, + kinetic term.
// dst = V psi + T psi (the nonlocal part is added by the projector GEMMs).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(ZCOL_THREADS) k_cols_to_wave(KArgs ka, int src, int dst) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int local = blockIdx.x - ka.start[p];
  const int nchunk = (P.ncp + QCP - 1) / QCP;
  const int pair = local / nchunk;
  const int chunk = local - pair * nchunk;
  const int n3 = P.n3;
  const int cp0 = chunk * QCP, cp1 = min(cp0 + QCP, P.ncp);
  int col0, col1;
  chunk_cols(cp0, cp1, &col0, &col1);
  const int ncl = col1 - col0;
  cplx<T>* lines = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* alt = lines + 2 * QCP * n3;
  cplx<T>* roots = alt + 2 * QCP * n3;
  load_roots<T>(roots, P, P.n1 + P.n2, n3);
  const cplx<T>* wc = reinterpret_cast<const cplx<T>*>(P.Wc) + (size_t)pair * n3 * P.ncol;
  for (int t = threadIdx.x; t < ncl * n3; t += blockDim.x) {
    int z = t / ncl, c = t - z * ncl;
    lines[c * n3 + z] = wc[(size_t)z * P.ncol + col0 + c];
  }
  __syncthreads();
  lines = fft_lines<T>(lines, alt, ncl, n3, 1, contiguous(ncl), P.fd[2], roots, T(-1));

  const int ia = 2 * pair, ib = 2 * pair + 1;
  const bool hasb = ib < P.nb;
  const T* xa = wbuf<T>(P, src) + (size_t)ia * P.ld;
  const T* xb = wbuf<T>(P, src) + (size_t)(hasb ? ib : ia) * P.ld;
  T* ya = wbuf<T>(P, dst) + (size_t)ia * P.ld;
  T* yb = wbuf<T>(P, dst) + (size_t)(hasb ? ib : ia) * P.ld;
  const T hs2 = T(0.5 * SQRT2);
  const int e0 = P.cp_off[cp0], e1 = P.cp_off[cp1];
  for (int k = e0 + threadIdx.x; k < e1; k += blockDim.x) {
    int cp = cp0;
    while (P.cp_off[cp + 1] <= k) ++cp;
    const int m3 = P.ent_m3[k];
    int lp, lm;
    if (cp == 0) { lp = 0; lm = 0; }
    else { lp = 2 * cp - 1 - col0; lm = 2 * cp - col0; }
    cplx<T> fp = lines[lp * n3 + wrapi(m3, n3)];
    cplx<T> fm = lines[lm * n3 + wrapi(-m3, n3)];
    // a: (fp + conj fm)/2 ; b: (fp - conj fm)/(2i)
    const T ek = ekin_at<T>(P, 1 + 2 * k);
    T ar = (fp.x + fm.x) * hs2, ai = (fp.y - fm.y) * hs2;
    T br = (fp.y + fm.y) * hs2, bi = (fm.x - fp.x) * hs2;
    ya[1 + 2 * k] = ar + ek * xa[1 + 2 * k];
    ya[2 + 2 * k] = ai + ek * xa[2 + 2 * k];
    if (hasb) {
      yb[1 + 2 * k] = br + ek * xb[1 + 2 * k];
      yb[2 + 2 * k] = bi + ek * xb[2 + 2 * k];
    }
  }
  if (cp0 == 0 && threadIdx.x == 0) {
    cplx<T> f0 = lines[0];
    ya[0] = f0.x;
    if (hasb) yb[0] = f0.y;
  }
}

// ---------------------------------------------------------------------------
// Per (problem, band pair, z): y and x FFTs to real space, times V_eff/N, and back.
// In place on the compact columns of plane z.
// ---------------------------------------------------------------------------
// Zero both ping-pong planes (rows outside the y-FFT range must read as zero in
// whichever buffer the data ends up in), then scatter the compact columns.
template <typename T>
__device__ __forceinline__ void plane_scatter(const Prob& P, cplx<T>* plane, cplx<T>* alt, const cplx<T>* wcz) {
  const int n12 = P.n1 * P.n2;
  for (int t = threadIdx.x; t < n12; t += blockDim.x) {
    plane[t] = mk(T(0), T(0));
    alt[t] = mk(T(0), T(0));
  }
  __syncthreads();
  for (int c = threadIdx.x; c < P.ncol; c += blockDim.x) plane[P.col_xy[c]] = wcz[c];
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(PLANE_THREADS, sizeof(T) == 4 ? PLANE_MIN_BLOCKS : 2) k_plane_vpsi(KArgs ka) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int local = blockIdx.x - ka.start[p];
  const int pair = local / P.n3;
  const int z = local - pair * P.n3;
  const int n1 = P.n1, n2 = P.n2;
  cplx<T>* b0 = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* b1 = b0 + n1 * n2;
  cplx<T>* r1 = b1 + n1 * n2;
  cplx<T>* r2 = r1 + n1;
  load_roots<T>(r1, P, 0, n1);
  load_roots<T>(r2, P, n1, n2);
  cplx<T>* wcz = reinterpret_cast<cplx<T>*>(P.Wc) + ((size_t)pair * P.n3 + z) * P.ncol;
  plane_scatter<T>(P, b0, b1, wcz);
  // rows i1 with |m1| <= m1max: [0, m1max] and [n1 - m1max, n1)
  const int mx = P.m1max;
  const LineMap rows{mx + 1, n1 - 2 * mx - 1};
  cplx<T>* cur = b0;
  cur = fft_lines<T>(cur, cur == b0 ? b1 : b0, 2 * mx + 1, n2, 1, rows, P.fd[1], r2, T(1));   // y, inverse
  cur = fft_lines<T>(cur, cur == b0 ? b1 : b0, n2, 1, n2, contiguous(n2), P.fd[0], r1, T(1));  // x, inverse
  const T* v = reinterpret_cast<const T*>(P.veff) + (size_t)z * n1 * n2;
  for (int t = threadIdx.x; t < n1 * n2; t += blockDim.x) cur[t] = scale(cur[t], v[t]);
  __syncthreads();
  cur = fft_lines<T>(cur, cur == b0 ? b1 : b0, n2, 1, n2, contiguous(n2), P.fd[0], r1, T(-1));  // x, forward
  cur = fft_lines<T>(cur, cur == b0 ? b1 : b0, 2 * mx + 1, n2, 1, rows, P.fd[1], r2, T(-1));   // y, forward
  for (int c = threadIdx.x; c < P.ncol; c += blockDim.x) wcz[c] = cur[P.col_xy[c]];
}

// ---------------------------------------------------------------------------
// Per (problem, z): rho(r) = (1/Omega) sum_pairs f_a Re^2 + f_b Im^2 over all band pairs,
// accumulated in registers (point t + i*blockDim per thread) in FP64.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(PLANE_THREADS, sizeof(T) == 4 ? PLANE_MIN_BLOCKS : 2) k_plane_density(KArgs ka, const double* occ_override) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int z = blockIdx.x - ka.start[p];
  const int n1 = P.n1, n2 = P.n2, n12 = n1 * n2;
  cplx<T>* b0 = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* b1 = b0 + n12;
  cplx<T>* r1 = b1 + n12;
  cplx<T>* r2 = r1 + n1;
  load_roots<T>(r1, P, 0, n1);
  load_roots<T>(r2, P, n1, n2);
  const double* occ = occ_override ? occ_override : P.occ;
  double* acc = reinterpret_cast<double*>(r2 + n2);  // FP64 accumulators of this z-plane
  for (int t = threadIdx.x; t < n12; t += blockDim.x) acc[t] = 0.0;
  const int mx = P.m1max;
  const LineMap rows{mx + 1, n1 - 2 * mx - 1};
  for (int pair = 0; pair < P.npair; ++pair) {
    const double fa = occ[2 * pair];
    const double fb = (2 * pair + 1 < P.nb) ? occ[2 * pair + 1] : 0.0;
    if (fa == 0.0 && fb == 0.0) continue;  // uniform across the block
    const cplx<T>* wcz = reinterpret_cast<const cplx<T>*>(P.Wc) + ((size_t)pair * P.n3 + z) * P.ncol;
    __syncthreads();
    plane_scatter<T>(P, b0, b1, wcz);
    cplx<T>* cur = b0;
    cur = fft_lines<T>(cur, cur == b0 ? b1 : b0, 2 * mx + 1, n2, 1, rows, P.fd[1], r2, T(1));
    cur = fft_lines<T>(cur, cur == b0 ? b1 : b0, n2, 1, n2, contiguous(n2), P.fd[0], r1, T(1));
    for (int t = threadIdx.x; t < n12; t += blockDim.x) {
      const cplx<T> v = cur[t];
      acc[t] += fa * (double)v.x * (double)v.x + fb * (double)v.y * (double)v.y;
    }
  }
  __syncthreads();
  const double io = 1.0 / P.omega;
  double* rho = P.rho_out + (size_t)z * n12;
  for (int t = threadIdx.x; t < n12; t += blockDim.x) rho[t] = acc[t] * io;
}

// ---------------------------------------------------------------------------
// Full FP64 complex grid transforms (in place): plane pass (x and y) and z pass.
// which: 0 = gfft, 1 = gfft2, 2 = gfft3, 3 = gfft4 (the PBE grids).
// ---------------------------------------------------------------------------
// The work grids in the storage precision of a transform: FP64 complex (double and
// float-float), or (FP32) the first half of the same memory viewed as single-precision
// complex.
template <typename T>
__device__ __forceinline__ cplx<typename Work<T>::S>* grid_of(const Prob& P, int which) {
  double2* const g[4] = {P.gfft, P.gfft2, P.gfft3, P.gfft4};
  return reinterpret_cast<cplx<typename Work<T>::S>*>(g[which & 3]);
}

template <typename T>
__global__ void __launch_bounds__(PLANE_THREADS) k_grid_plane_fft(KArgs ka, int which, int sign) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int z = blockIdx.x - ka.start[p];
  const int n1 = P.n1, n2 = P.n2, n12 = n1 * n2;
  cplx<T>* b0 = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* b1 = b0 + n12;
  cplx<T>* r1 = b1 + n12;
  cplx<T>* r2 = r1 + n1;
  load_roots<T>(r1, P, 0, n1);
  load_roots<T>(r2, P, n1, n2);
  auto* g = grid_of<T>(P, which) + (size_t)z * n12;
  for (int t = threadIdx.x; t < n12; t += blockDim.x) b0[t] = Work<T>::in(g[t]);
  __syncthreads();
  const T sg = sign < 0 ? T(-1) : T(1);
  cplx<T>* cur = fft_lines<T>(b0, b1, n1, n2, 1, contiguous(n1), P.fd[1], r2, sg);      // y
  cur = fft_lines<T>(cur, cur == b0 ? b1 : b0, n2, 1, n2, contiguous(n2), P.fd[0], r1, sg);  // x
  for (int t = threadIdx.x; t < n12; t += blockDim.x) g[t] = Work<T>::out(cur[t]);
}

template <typename T>
__global__ void __launch_bounds__(ZCOL_THREADS) k_grid_z_fft(KArgs ka, int which, int sign) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int chunk = blockIdx.x - ka.start[p];
  const int n12 = P.n1 * P.n2, n3 = P.n3;
  const int c0 = chunk * QZ, nc = min(QZ, n12 - c0);
  cplx<T>* lines = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* alt = lines + QZ * n3;
  cplx<T>* roots = alt + QZ * n3;
  load_roots<T>(roots, P, P.n1 + P.n2, n3);
  auto* g = grid_of<T>(P, which);
  for (int t = threadIdx.x; t < nc * n3; t += blockDim.x) {
    int z = t / nc, c = t - z * nc;
    lines[c * n3 + z] = Work<T>::in(g[(size_t)z * n12 + c0 + c]);
  }
  __syncthreads();
  const cplx<T>* res = fft_lines<T>(lines, alt, nc, n3, 1, contiguous(nc), P.fd[2], roots, sign < 0 ? T(-1) : T(1));
  for (int t = threadIdx.x; t < nc * n3; t += blockDim.x) {
    int z = t / nc, c = t - z * nc;
    g[(size_t)z * n12 + c0 + c] = Work<T>::out(res[c * n3 + z]);
  }
}

// Line blocks of the grid transform for planes too large for one CTA: along x (axis 0:
// length N1, element stride N2, lines (z, i2)) or y (axis 1: length N2, contiguous, lines
// (z, i1)), QZ lines per CTA, loads and stores coalesced across the lines' fast index.
template <typename T>
__global__ void __launch_bounds__(ZCOL_THREADS) k_grid_line_fft(KArgs ka, int which, int sign, int axis) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int chunk = blockIdx.x - ka.start[p];
  const int n1 = P.n1, n2 = P.n2, n12 = n1 * n2;
  const int n = axis ? n2 : n1;
  const int nlines = P.n3 * (axis ? n1 : n2);
  const int l0 = chunk * QZ, nc = min(QZ, nlines - l0);
  cplx<T>* lines = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* alt = lines + QZ * n;
  cplx<T>* roots = alt + QZ * n;
  load_roots<T>(roots, P, axis ? n1 : 0, n);
  auto* g = grid_of<T>(P, which);
  auto at = [&](int c, int e) -> size_t {
    const int l = l0 + c;
    if (axis) return (size_t)l * n2 + e;
    const int z = l / n2;
    return (size_t)z * n12 + (size_t)e * n2 + (l - z * n2);
  };
  for (int t = threadIdx.x; t < nc * n; t += blockDim.x) {
    const int c = axis ? t / n : t % nc, e = axis ? t % n : t / nc;
    lines[c * n + e] = Work<T>::in(g[at(c, e)]);
  }
  __syncthreads();
  const cplx<T>* res =
      fft_lines<T>(lines, alt, nc, n, 1, contiguous(nc), P.fd[axis ? 1 : 0], roots, sign < 0 ? T(-1) : T(1));
  for (int t = threadIdx.x; t < nc * n; t += blockDim.x) {
    const int c = axis ? t / n : t % nc, e = axis ? t % n : t / nc;
    g[at(c, e)] = Work<T>::out(res[c * n + e]);
  }
}

// ---------------------------------------------------------------------------
// Plane pass by line blocks through a global buffer, for planes whose two copies do not
// fit in one CTA's shared memory (the FP64 path beyond about 6900 points per plane).
// Gp[pair][z][r][i2] holds the occupied x rows of each band pair's plane between its y
// and x transforms: r = i1 for i1 <= m1max, r = i1 - (n1 - 2 m1max - 1) for the rows
// i1 >= n1 - m1max (|m1| <= m1max); the other rows are zero and never stored.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int big_row_i1(const Prob& P, int r) {
  return r <= P.m1max ? r : r + P.n1 - 2 * P.m1max - 1;
}
__device__ __forceinline__ int big_row_of(const Prob& P, int i1) {
  if (i1 <= P.m1max) return i1;
  if (i1 >= P.n1 - P.m1max) return i1 - (P.n1 - 2 * P.m1max - 1);
  return -1;
}

// dir +1: compact columns of (pair, z) -> inverse y FFT -> rows of Gp; dir -1: rows of Gp
// -> forward y FFT -> compact columns.  CTA = (problem, pair, z, block of QZ rows).
// skip_empty: pairs whose two occupations are zero are skipped (density pass).
template <typename T>
__global__ void __launch_bounds__(ZCOL_THREADS) k_big_y(KArgs ka, int dir, int skip_empty, const double* occ_override) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int nrows = 2 * P.m1max + 1, nrb = (nrows + QZ - 1) / QZ;
  const int local = blockIdx.x - ka.start[p];
  const int rb = local % nrb, pz = local / nrb;
  const int z = pz % P.n3, pair = pz / P.n3;
  if (skip_empty) {
    const double* occ = occ_override ? occ_override : P.occ;
    const double fa = occ[2 * pair], fb = (2 * pair + 1 < P.nb) ? occ[2 * pair + 1] : 0.0;
    if (fa == 0.0 && fb == 0.0) return;
  }
  const int n = P.n2, r0 = rb * QZ, nc = min(QZ, nrows - r0);
  cplx<T>* lines = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* alt = lines + QZ * n;
  cplx<T>* roots = alt + QZ * n;
  load_roots<T>(roots, P, P.n1, n);
  cplx<T>* wcz = reinterpret_cast<cplx<T>*>(P.Wc) + ((size_t)pair * P.n3 + z) * P.ncol;
  cplx<T>* gp = reinterpret_cast<cplx<T>*>(P.Gp) + ((size_t)pair * P.n3 + z) * nrows * n;
  for (int t = threadIdx.x; t < nc * n; t += blockDim.x) {
    const int c = t / n, e = t - c * n;
    if (dir > 0) {
      const int col = P.colmap[big_row_i1(P, r0 + c) * n + e];
      lines[t] = col >= 0 ? wcz[col] : mk(T(0), T(0));
    } else {
      lines[t] = gp[(size_t)(r0 + c) * n + e];
    }
  }
  __syncthreads();
  const cplx<T>* res = fft_lines<T>(lines, alt, nc, n, 1, contiguous(nc), P.fd[1], roots, dir > 0 ? T(1) : T(-1));
  for (int t = threadIdx.x; t < nc * n; t += blockDim.x) {
    const int c = t / n, e = t - c * n;
    if (dir > 0) {
      gp[(size_t)(r0 + c) * n + e] = res[t];
    } else {
      const int col = P.colmap[big_row_i1(P, r0 + c) * n + e];
      if (col >= 0) wcz[col] = res[t];
    }
  }
}

// x lines of (pair, z): inverse x FFT (the unstored rows read as zero), times V_eff/N,
// forward x FFT, occupied rows back to Gp.  CTA = (problem, pair, z, block of QZ columns
// i2); loads and stores coalesced across the block's columns.
template <typename T>
__global__ void __launch_bounds__(ZCOL_THREADS) k_big_x(KArgs ka) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int n1 = P.n1, n2 = P.n2, nrows = 2 * P.m1max + 1, ncb = (n2 + QZ - 1) / QZ;
  const int local = blockIdx.x - ka.start[p];
  const int cb = local % ncb, pz = local / ncb;
  const int z = pz % P.n3, pair = pz / P.n3;
  const int c0 = cb * QZ, nc = min(QZ, n2 - c0);
  cplx<T>* lines = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* alt = lines + QZ * n1;
  cplx<T>* roots = alt + QZ * n1;
  load_roots<T>(roots, P, 0, n1);
  cplx<T>* gp = reinterpret_cast<cplx<T>*>(P.Gp) + ((size_t)pair * P.n3 + z) * nrows * n2;
  for (int t = threadIdx.x; t < nc * n1; t += blockDim.x) {
    const int e = t / nc, c = t - e * nc;
    const int r = big_row_of(P, e);
    lines[c * n1 + e] = r >= 0 ? gp[(size_t)r * n2 + c0 + c] : mk(T(0), T(0));
  }
  __syncthreads();
  cplx<T>* cur = fft_lines<T>(lines, alt, nc, n1, 1, contiguous(nc), P.fd[0], roots, T(1));
  const T* v = reinterpret_cast<const T*>(P.veff) + (size_t)z * n1 * n2;
  for (int t = threadIdx.x; t < nc * n1; t += blockDim.x) {
    const int e = t / nc, c = t - e * nc;
    cur[c * n1 + e] = scale(cur[c * n1 + e], v[(size_t)e * n2 + c0 + c]);
  }
  __syncthreads();
  cur = fft_lines<T>(cur, cur == lines ? alt : lines, nc, n1, 1, contiguous(nc), P.fd[0], roots, T(-1));
  for (int t = threadIdx.x; t < nc * n1; t += blockDim.x) {
    const int e = t / nc, c = t - e * nc;
    const int r = big_row_of(P, e);
    if (r >= 0) gp[(size_t)r * n2 + c0 + c] = cur[c * n1 + e];
  }
}

// Density of the big-plane path: per (problem, z, block of QZ columns i2), every band pair's
// x lines (after k_big_y) transformed to real space and f_a Re^2 + f_b Im^2 accumulated in
// FP64 over the pairs in order; rho_out = sum / Omega.
template <typename T>
__global__ void __launch_bounds__(ZCOL_THREADS) k_big_density(KArgs ka, const double* occ_override) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int p = locate(ka.start, ka.nprob, blockIdx.x);
  if (!ka.active[p]) return;
  const Prob& P = ka.probs[p];
  const int n1 = P.n1, n2 = P.n2, nrows = 2 * P.m1max + 1, ncb = (n2 + QZ - 1) / QZ;
  const int local = blockIdx.x - ka.start[p];
  const int cb = local % ncb, z = local / ncb;
  const int c0 = cb * QZ, nc = min(QZ, n2 - c0);
  cplx<T>* lines = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* alt = lines + QZ * n1;
  cplx<T>* roots = alt + QZ * n1;
  double* acc = reinterpret_cast<double*>(roots + n1);
  load_roots<T>(roots, P, 0, n1);
  for (int t = threadIdx.x; t < nc * n1; t += blockDim.x) acc[t] = 0.0;
  const double* occ = occ_override ? occ_override : P.occ;
  for (int pair = 0; pair < P.npair; ++pair) {
    const double fa = occ[2 * pair], fb = (2 * pair + 1 < P.nb) ? occ[2 * pair + 1] : 0.0;
    if (fa == 0.0 && fb == 0.0) continue;  // uniform across the block
    const cplx<T>* gp = reinterpret_cast<const cplx<T>*>(P.Gp) + ((size_t)pair * P.n3 + z) * nrows * n2;
    __syncthreads();
    for (int t = threadIdx.x; t < nc * n1; t += blockDim.x) {
      const int e = t / nc, c = t - e * nc;
      const int r = big_row_of(P, e);
      lines[c * n1 + e] = r >= 0 ? gp[(size_t)r * n2 + c0 + c] : mk(T(0), T(0));
    }
    __syncthreads();
    const cplx<T>* cur = fft_lines<T>(lines, alt, nc, n1, 1, contiguous(nc), P.fd[0], roots, T(1));
    for (int t = threadIdx.x; t < nc * n1; t += blockDim.x) {
      const cplx<T> v = cur[t];
      acc[t] += fa * (double)v.x * (double)v.x + fb * (double)v.y * (double)v.y;
    }
  }
  __syncthreads();
  const double io = 1.0 / P.omega;
  double* rho = P.rho_out + (size_t)z * n1 * n2;
  for (int t = threadIdx.x; t < nc * n1; t += blockDim.x) {
    const int e = t / nc, c = t - e * nc;
    rho[(size_t)e * n2 + c0 + c] = acc[c * n1 + e] * io;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int big_y_ctas(int npair, int n3, int m1max) { return npair * n3 * ((2 * m1max + 1 + QZ - 1) / QZ); }
int big_x_ctas(int npair, int n3, int n2) { return npair * n3 * ((n2 + QZ - 1) / QZ); }
int big_density_ctas(int n3, int n2) { return n3 * ((n2 + QZ - 1) / QZ); }
size_t big_plane_bytes(int npair, int n3, int m1max, int n2, size_t tsize) {
  return (size_t)npair * n3 * (2 * m1max + 1) * n2 * 2 * tsize;
}
template <typename T>
void launch_big_y(const Launch& L, int dir, int skip_empty, const double* occ_override) {
  if (!L.map.total) return;
  size_t sm = (size_t)(2 * QZ + 1) * L.max_n2 * sizeof(cplx<T>);
  k_big_y<T><<<L.map.total, ZCOL_THREADS, sm, L.stream>>>(L.ka, dir, skip_empty, occ_override);
}
template <typename T>
void launch_big_x(const Launch& L) {
  if (!L.map.total) return;
  size_t sm = (size_t)(2 * QZ + 1) * L.max_n1 * sizeof(cplx<T>);
  k_big_x<T><<<L.map.total, ZCOL_THREADS, sm, L.stream>>>(L.ka);
}
template <typename T>
void launch_big_density(const Launch& L, const double* occ_override) {
  if (!L.map.total) return;
  size_t sm = (size_t)(2 * QZ + 1) * L.max_n1 * sizeof(cplx<T>) + (size_t)QZ * L.max_n1 * sizeof(double);
  k_big_density<T><<<L.map.total, ZCOL_THREADS, sm, L.stream>>>(L.ka, occ_override);
}

template <typename T>
void launch_wave_to_cols(const Launch& L, int src) {
  if (!L.map.total) return;
  size_t sm = (size_t)(4 * QCP + 1) * L.max_n3 * sizeof(cplx<T>);
  k_wave_to_cols<T><<<L.map.total, ZCOL_THREADS, sm, L.stream>>>(L.ka, src);
}
template <typename T>
void launch_cols_to_wave(const Launch& L, int src, int dst) {
  if (!L.map.total) return;
  size_t sm = (size_t)(4 * QCP + 1) * L.max_n3 * sizeof(cplx<T>);
  k_cols_to_wave<T><<<L.map.total, ZCOL_THREADS, sm, L.stream>>>(L.ka, src, dst);
}
template <typename T>
void launch_plane_vpsi(const Launch& L) {
  if (!L.map.total) return;
  size_t sm = (size_t)(2 * L.max_n12 + L.max_n1 + L.max_n2) * sizeof(cplx<T>);
  k_plane_vpsi<T><<<L.map.total, L.plane_threads, sm, L.stream>>>(L.ka);
}
template <typename T>
void launch_plane_density(const Launch& L, const double* occ_override) {
  if (!L.map.total) return;
  size_t sm = (size_t)(2 * L.max_n12 + L.max_n1 + L.max_n2) * sizeof(cplx<T>) + (size_t)L.max_n12 * sizeof(double) + 16;
  k_plane_density<T><<<L.map.total, L.plane_threads, sm, L.stream>>>(L.ka, occ_override);
}
template <typename T>
void launch_grid_line_fft(const Launch& L, int which, int sign, int axis) {
  if (!L.map.total) return;
  const int n = axis ? L.max_n2 : L.max_n1;
  size_t sm = (size_t)(2 * QZ + 1) * n * sizeof(cplx<T>);
  k_grid_line_fft<T><<<L.map.total, ZCOL_THREADS, sm, L.stream>>>(L.ka, which, sign, axis);
}
template <typename T>
void launch_grid_plane_fft(const Launch& L, int which, int sign) {
  if (!L.map.total) return;
  size_t sm = (size_t)(2 * L.max_n12 + L.max_n1 + L.max_n2) * sizeof(cplx<T>);
  k_grid_plane_fft<T><<<L.map.total, L.plane_threads, sm, L.stream>>>(L.ka, which, sign);
}
template <typename T>
void launch_grid_z_fft(const Launch& L, int which, int sign) {
  if (!L.map.total) return;
  size_t sm = (size_t)(2 * QZ + 1) * L.max_n3 * sizeof(cplx<T>);
  k_grid_z_fft<T><<<L.map.total, ZCOL_THREADS, sm, L.stream>>>(L.ka, which, sign);
}

bool fft_reg_init() {
  return plane_vpsi_reg_init() && plane_density_reg_init() && zreg_init() && pair_reg_init() && plane_ms_init();
}

void fft_set_smem_limits(size_t bytes) {
  cudaFuncSetAttribute(k_wave_to_cols<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_wave_to_cols<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_cols_to_wave<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_cols_to_wave<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_plane_vpsi<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_plane_vpsi<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_plane_density<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_plane_density<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_grid_plane_fft<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_grid_z_fft<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_grid_line_fft<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_grid_plane_fft<ff>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_grid_z_fft<ff>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_grid_line_fft<ff>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_grid_plane_fft<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_grid_z_fft<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_grid_line_fft<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_big_y<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_big_y<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_big_x<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_big_x<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_big_density<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  cudaFuncSetAttribute(k_big_density<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  plane_vpsi_reg_set_smem_limits(bytes);
  plane_ms_set_smem_limits(bytes);
  plane_density_reg_set_smem_limits(bytes);
  zreg_set_smem_limits(bytes);
  pair_reg_set_smem_limits(bytes);
}

template void launch_wave_to_cols<float>(const Launch&, int);
template void launch_wave_to_cols<double>(const Launch&, int);
template void launch_cols_to_wave<float>(const Launch&, int, int);
template void launch_cols_to_wave<double>(const Launch&, int, int);
template void launch_grid_line_fft<float>(const Launch&, int, int, int);
template void launch_grid_line_fft<double>(const Launch&, int, int, int);
template void launch_grid_plane_fft<float>(const Launch&, int, int);
template void launch_grid_plane_fft<double>(const Launch&, int, int);
template void launch_grid_z_fft<float>(const Launch&, int, int);
template void launch_grid_z_fft<double>(const Launch&, int, int);
template void launch_grid_line_fft<ff>(const Launch&, int, int, int);
template void launch_grid_plane_fft<ff>(const Launch&, int, int);
template void launch_grid_z_fft<ff>(const Launch&, int, int);
template void launch_plane_vpsi<float>(const Launch&);
template void launch_plane_vpsi<double>(const Launch&);
template void launch_plane_density<float>(const Launch&, const double*);
template void launch_plane_density<double>(const Launch&, const double*);
template void launch_big_y<float>(const Launch&, int, int, const double*);
template void launch_big_y<double>(const Launch&, int, int, const double*);
template void launch_big_x<float>(const Launch&);
template void launch_big_x<double>(const Launch&);
template void launch_big_density<float>(const Launch&, const double*);
template void launch_big_density<double>(const Launch&, const double*);

}  // namespace sgo
