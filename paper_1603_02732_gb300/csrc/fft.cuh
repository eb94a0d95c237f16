// Batched 1D FFTs on lines held in shared memory (device side).
//
// A mixed-radix (2, 3, 4, 5 and composite 6 ... 16) Stockham autosort transform (Stockham, 1966; the
// GPU formulation of Govindaraju et al., SC'08).  Stage s with radix R and span
// Ns (product of the earlier radices) maps, for every butterfly j < n/R of a line,
//   v_r = in[j + r n/R] * w^(r (j mod Ns)),  w = exp(sign 2 pi i / (Ns R)),
//   v = DFT_R(v),  out[(j - j mod Ns) R + j mod Ns + r Ns] = v_r.
// Stages alternate between two shared-memory buffers (out of place, one
// butterfly per thread iteration, so few registers).  No scaling is applied.
//   sign = -1: X(m) = sum_j x(j) exp(-2 pi i m j / n)   (r -> G)
//   sign = +1: x(j) = sum_m X(m) exp(+2 pi i m j / n)   (G -> r)
#pragma once

#include "ff.cuh"
#include "sgo_internal.cuh"

namespace sgo {

// exp(sign 2 pi i / 3) etc. written out: cos/sin of 2pi/3, 2pi/5, 4pi/5 (functions, so that
// the float-float type, not a scalar, can take them in device code too).
template <typename T>
struct Rc {
  static __host__ __device__ __forceinline__ T s3() { return T(0.86602540378443864676); }
  static __host__ __device__ __forceinline__ T c1() { return T(0.30901699437494742410); }   // cos(2 pi/5)
  static __host__ __device__ __forceinline__ T c2() { return T(-0.80901699437494742410); }  // cos(4 pi/5)
  static __host__ __device__ __forceinline__ T s1() { return T(0.95105651629515357212); }   // sin(2 pi/5)
  static __host__ __device__ __forceinline__ T s2() { return T(0.58778525229247312917); }   // sin(4 pi/5)
};

template <typename T, int R>
__device__ __forceinline__ void butterfly(cplx<T>* v, T sg);

template <>
__device__ __forceinline__ void butterfly<float, 2>(cplx<float>* v, float) {
  cplx<float> a = v[0], b = v[1];
  v[0] = a + b;
  v[1] = a - b;
}
template <>
__device__ __forceinline__ void butterfly<double, 2>(cplx<double>* v, double) {
  cplx<double> a = v[0], b = v[1];
  v[0] = a + b;
  v[1] = a - b;
}
template <>
__device__ __forceinline__ void butterfly<ff, 2>(cplx<ff>* v, ff) {
  cplx<ff> a = v[0], b = v[1];
  v[0] = a + b;
  v[1] = a - b;
}

template <typename T>
__device__ __forceinline__ void bfly3(cplx<T>* v, T sg) {
  cplx<T> a = v[0], b = v[1], c = v[2];
  cplx<T> t1 = b + c;
  cplx<T> t2 = mk(a.x - T(0.5) * t1.x, a.y - T(0.5) * t1.y);
  cplx<T> t3 = scale(b - c, sg * Rc<T>::s3());
  v[0] = a + t1;
  v[1] = mk(t2.x - t3.y, t2.y + t3.x);  // t2 + i t3
  v[2] = mk(t2.x + t3.y, t2.y - t3.x);  // t2 - i t3
}
template <>
__device__ __forceinline__ void butterfly<float, 3>(cplx<float>* v, float sg) { bfly3<float>(v, sg); }
template <>
__device__ __forceinline__ void butterfly<double, 3>(cplx<double>* v, double sg) { bfly3<double>(v, sg); }
template <>
__device__ __forceinline__ void butterfly<ff, 3>(cplx<ff>* v, ff sg) { bfly3<ff>(v, sg); }

template <typename T>
__device__ __forceinline__ void bfly4(cplx<T>* v, T sg) {
  cplx<T> a = v[0], b = v[1], c = v[2], d = v[3];
  cplx<T> s0 = a + c, d0 = a - c, s1 = b + d, d1 = mul_is(b - d, sg);
  v[0] = s0 + s1;
  v[2] = s0 - s1;
  v[1] = d0 + d1;
  v[3] = d0 - d1;
}
template <>
__device__ __forceinline__ void butterfly<float, 4>(cplx<float>* v, float sg) { bfly4<float>(v, sg); }
template <>
__device__ __forceinline__ void butterfly<double, 4>(cplx<double>* v, double sg) { bfly4<double>(v, sg); }
template <>
__device__ __forceinline__ void butterfly<ff, 4>(cplx<ff>* v, ff sg) { bfly4<ff>(v, sg); }

template <typename T>
__device__ __forceinline__ void bfly5(cplx<T>* v, T sg) {
  cplx<T> a = v[0];
  cplx<T> t1 = v[1] + v[4], t2 = v[2] + v[3], t3 = v[1] - v[4], t4 = v[2] - v[3];
  const T c1 = Rc<T>::c1(), c2 = Rc<T>::c2(), s1 = Rc<T>::s1(), s2 = Rc<T>::s2();
  cplx<T> u1 = mk(a.x + c1 * t1.x + c2 * t2.x, a.y + c1 * t1.y + c2 * t2.y);
  cplx<T> u2 = mk(a.x + c2 * t1.x + c1 * t2.x, a.y + c2 * t1.y + c1 * t2.y);
  cplx<T> w1 = mul_is(mk(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y), sg);
  cplx<T> w2 = mul_is(mk(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y), sg);
  v[0] = a + t1 + t2;
  v[1] = u1 + w1;
  v[4] = u1 - w1;
  v[2] = u2 + w2;
  v[3] = u2 - w2;
}
template <>
__device__ __forceinline__ void butterfly<float, 5>(cplx<float>* v, float sg) { bfly5<float>(v, sg); }
template <>
__device__ __forceinline__ void butterfly<double, 5>(cplx<double>* v, double sg) { bfly5<double>(v, sg); }
template <>
__device__ __forceinline__ void butterfly<ff, 5>(cplx<ff>* v, ff sg) { bfly5<ff>(v, sg); }

// Composite radix R = R1 R2 in registers (Cooley-Tukey inside the butterfly):
// with m = R2 m1 + m2 and k = k1 + R1 k2,
//   X[k1 + R1 k2] = sum_m2 w_R2^(m2 k2) [ w_R^(m2 k1) sum_m1 x[R2 m1 + m2] w_R1^(m1 k1) ].
// The internal factors w_R^t are read from the line's roots table (t (n/R) entries apart).
template <typename T, int R>
struct Bfly;

template <typename T, int R1, int R2>
__device__ __forceinline__ void bfly_comp(cplx<T>* v, T sg, const cplx<T>* roots, int stride) {
  constexpr int R = R1 * R2;
  cplx<T> y[R2][R1];
#pragma unroll
  for (int m2 = 0; m2 < R2; ++m2) {
    cplx<T> a[R1];
#pragma unroll
    for (int m1 = 0; m1 < R1; ++m1) a[m1] = v[R2 * m1 + m2];
    Bfly<T, R1>::run(a, sg, roots, stride * R2);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) y[m2][k1] = a[k1];
  }
#pragma unroll
  for (int m2 = 1; m2 < R2; ++m2)
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) {
      cplx<T> w = roots[((m2 * k1) % R) * stride];
      w.y = sg < T(0) ? w.y : -w.y;
      y[m2][k1] = y[m2][k1] * w;
    }
#pragma unroll
  for (int k1 = 0; k1 < R1; ++k1) {
    cplx<T> b[R2];
#pragma unroll
    for (int m2 = 0; m2 < R2; ++m2) b[m2] = y[m2][k1];
    Bfly<T, R2>::run(b, sg, roots, stride * R1);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = b[k2];
  }
}

// Bfly<T,R>::run(v, sign, roots, stride): in-register DFT of length R, where
// roots[t * stride] = exp(-2 pi i t / R).
#define SGO_BASE_BFLY(RR)                                                                 \
  template <typename T>                                                                   \
  struct Bfly<T, RR> {                                                                    \
    static __device__ __forceinline__ void run(cplx<T>* v, T sg, const cplx<T>*, int) {    \
      butterfly<T, RR>(v, sg);                                                            \
    }                                                                                     \
  };
SGO_BASE_BFLY(2)
SGO_BASE_BFLY(3)
SGO_BASE_BFLY(4)
SGO_BASE_BFLY(5)
#undef SGO_BASE_BFLY
#define SGO_COMP_BFLY(RR, R1, R2)                                                               \
  template <typename T>                                                                         \
  struct Bfly<T, RR> {                                                                          \
    static __device__ __forceinline__ void run(cplx<T>* v, T sg, const cplx<T>* roots, int st) {  \
      bfly_comp<T, R1, R2>(v, sg, roots, st);                                                   \
    }                                                                                           \
  };
SGO_COMP_BFLY(6, 2, 3)
SGO_COMP_BFLY(8, 2, 4)
SGO_COMP_BFLY(9, 3, 3)
SGO_COMP_BFLY(10, 2, 5)
SGO_COMP_BFLY(12, 4, 3)
SGO_COMP_BFLY(15, 3, 5)
SGO_COMP_BFLY(16, 4, 4)
#undef SGO_COMP_BFLY

// floor(b / d) for b < 2^16, d <= 2^15, with mg = 0xFFFFFFFF / d + 1 (d > 1)
__device__ __forceinline__ unsigned fdiv(unsigned b, unsigned d, unsigned mg) { return d == 1 ? b : __umulhi(b, mg); }

// Line l starts at data + base(l) * ls, base(l) = l < split ? l : l + jump (two runs of lines).
struct LineMap {
  int split;
  int jump;
  __device__ __forceinline__ int operator()(int l) const { return l < split ? l : l + jump; }
};

template <typename T, int R>
__device__ __forceinline__ void fft_stage(const cplx<T>* __restrict__ src, cplx<T>* __restrict__ dst, int nlines,
                                          int ls, int es, LineMap lm, int n, int Ns, const cplx<T>* __restrict__ roots,
                                          T sg) {
  const int nq = n / R;
  const int total = nlines * nq;
  const int rs = n / (Ns * R);
  const unsigned dq = es == 1 ? nq : nlines;
  const unsigned mq = dq > 1 ? 0xFFFFFFFFu / dq + 1u : 0u;
  const unsigned mn = Ns > 1 ? 0xFFFFFFFFu / (unsigned)Ns + 1u : 0u;
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    // contiguous lines: neighbouring threads take neighbouring butterflies of a line;
    // strided lines: neighbouring threads take the same butterfly of neighbouring lines
    const int q = (int)fdiv((unsigned)b, dq, mq);
    const int line = es == 1 ? q : b - q * (int)dq;
    const int j = es == 1 ? b - q * (int)dq : q;
    const int k = j - (int)fdiv((unsigned)j, (unsigned)Ns, mn) * Ns;
    const int lb = lm(line) * ls;
    cplx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      cplx<T> x = src[lb + (j + r * nq) * es];
      if (r > 0 && k > 0) {
        cplx<T> w = roots[r * k * rs];
        w.y = sg < T(0) ? w.y : -w.y;
        x = x * w;
      }
      v[r] = x;
    }
    Bfly<T, R>::run(v, sg, roots, n / R);
    const int d0 = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[lb + (d0 + r * Ns) * es] = v[r];
  }
  __syncthreads();
}

// FFT of nlines lines of length d.n, ping-ponging between buffers a and b (same layout;
// element e of line l at [lm(l)*ls + e*es]).  Returns the buffer that holds the result.
// Only the addressed lines are read and written.  roots[t] = exp(-2 pi i t / n).
// The caller synchronises before the call; the call returns synchronised.
template <typename T>
__device__ __forceinline__ cplx<T>* fft_lines(cplx<T>* a, cplx<T>* b, int nlines, int ls, int es, LineMap lm,
                                              const FftDim& d, const cplx<T>* roots, T sg) {
  int Ns = 1;
  cplx<T>* src = a;
  cplx<T>* dst = b;
  for (int s = 0; s < d.nst; ++s) {
    const int R = d.rad[s];
    switch (R) {
      case 16: fft_stage<T, 16>(src, dst, nlines, ls, es, lm, d.n, Ns, roots, sg); break;
      case 15: fft_stage<T, 15>(src, dst, nlines, ls, es, lm, d.n, Ns, roots, sg); break;
      case 12: fft_stage<T, 12>(src, dst, nlines, ls, es, lm, d.n, Ns, roots, sg); break;
      case 10: fft_stage<T, 10>(src, dst, nlines, ls, es, lm, d.n, Ns, roots, sg); break;
      case 9: fft_stage<T, 9>(src, dst, nlines, ls, es, lm, d.n, Ns, roots, sg); break;
      case 8: fft_stage<T, 8>(src, dst, nlines, ls, es, lm, d.n, Ns, roots, sg); break;
      case 6: fft_stage<T, 6>(src, dst, nlines, ls, es, lm, d.n, Ns, roots, sg); break;
      case 5: fft_stage<T, 5>(src, dst, nlines, ls, es, lm, d.n, Ns, roots, sg); break;
      case 4: fft_stage<T, 4>(src, dst, nlines, ls, es, lm, d.n, Ns, roots, sg); break;
      case 3: fft_stage<T, 3>(src, dst, nlines, ls, es, lm, d.n, Ns, roots, sg); break;
      default: fft_stage<T, 2>(src, dst, nlines, ls, es, lm, d.n, Ns, roots, sg); break;
    }
    Ns *= R;
    cplx<T>* t = src;
    src = dst;
    dst = t;
  }
  return src;
}

__device__ __forceinline__ LineMap contiguous(int nlines) { return LineMap{nlines, 0}; }

}  // namespace sgo
