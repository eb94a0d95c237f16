// Batched 1D FFTs on lines held in shared memory (device side).
//
// A mixed-radix (2, 3, 4, 5) Stockham autosort transform (Stockham, 1966; the
// GPU formulation of Govindaraju et al., SC'08).  Stage s with radix R and span
// Ns (product of the earlier radices) maps, for every butterfly j < n/R of a line,
//   v_r = in[j + r n/R] * w^(r (j mod Ns)),  w = exp(sign 2 pi i / (Ns R)),
//   v = DFT_R(v),  out[(j - j mod Ns) R + j mod Ns + r Ns] = v_r.
// Stages alternate between two shared-memory buffers (out of place, one
// butterfly per thread iteration, so few registers).  No scaling is applied.
//   sign = -1: X(m) = sum_j x(j) exp(-2 pi i m j / n)   (r -> G)
//   sign = +1: x(j) = sum_m X(m) exp(+2 pi i m j / n)   (G -> r)
#pragma once

#include "sgo_internal.cuh"

namespace sgo {

// exp(sign 2 pi i / 3) etc. written out: cos/sin of 2pi/3, 2pi/5, 4pi/5.
template <typename T>
struct Rc {
  static constexpr T s3 = T(0.86602540378443864676);
  static constexpr T c1 = T(0.30901699437494742410);   // cos(2 pi/5)
  static constexpr T c2 = T(-0.80901699437494742410);  // cos(4 pi/5)
  static constexpr T s1 = T(0.95105651629515357212);   // sin(2 pi/5)
  static constexpr T s2 = T(0.58778525229247312917);   // sin(4 pi/5)
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

template <typename T>
__device__ __forceinline__ void bfly3(cplx<T>* v, T sg) {
  cplx<T> a = v[0], b = v[1], c = v[2];
  cplx<T> t1 = b + c;
  cplx<T> t2 = mk(a.x - T(0.5) * t1.x, a.y - T(0.5) * t1.y);
  cplx<T> t3 = scale(b - c, sg * Rc<T>::s3);
  v[0] = a + t1;
  v[1] = mk(t2.x - t3.y, t2.y + t3.x);  // t2 + i t3
  v[2] = mk(t2.x + t3.y, t2.y - t3.x);  // t2 - i t3
}
template <>
__device__ __forceinline__ void butterfly<float, 3>(cplx<float>* v, float sg) { bfly3<float>(v, sg); }
template <>
__device__ __forceinline__ void butterfly<double, 3>(cplx<double>* v, double sg) { bfly3<double>(v, sg); }

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

template <typename T>
__device__ __forceinline__ void bfly5(cplx<T>* v, T sg) {
  cplx<T> a = v[0];
  cplx<T> t1 = v[1] + v[4], t2 = v[2] + v[3], t3 = v[1] - v[4], t4 = v[2] - v[3];
  cplx<T> u1 = mk(a.x + Rc<T>::c1 * t1.x + Rc<T>::c2 * t2.x, a.y + Rc<T>::c1 * t1.y + Rc<T>::c2 * t2.y);
  cplx<T> u2 = mk(a.x + Rc<T>::c2 * t1.x + Rc<T>::c1 * t2.x, a.y + Rc<T>::c2 * t1.y + Rc<T>::c1 * t2.y);
  cplx<T> w1 = mul_is(mk(Rc<T>::s1 * t3.x + Rc<T>::s2 * t4.x, Rc<T>::s1 * t3.y + Rc<T>::s2 * t4.y), sg);
  cplx<T> w2 = mul_is(mk(Rc<T>::s2 * t3.x - Rc<T>::s1 * t4.x, Rc<T>::s2 * t3.y - Rc<T>::s1 * t4.y), sg);
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
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    const int line = b / nq;
    const int j = b - line * nq;
    const int k = j % Ns;
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
    butterfly<T, R>(v, sg);
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
    if (R == 4) fft_stage<T, 4>(src, dst, nlines, ls, es, lm, d.n, Ns, roots, sg);
    else if (R == 2) fft_stage<T, 2>(src, dst, nlines, ls, es, lm, d.n, Ns, roots, sg);
    else if (R == 3) fft_stage<T, 3>(src, dst, nlines, ls, es, lm, d.n, Ns, roots, sg);
    else fft_stage<T, 5>(src, dst, nlines, ls, es, lm, d.n, Ns, roots, sg);
    Ns *= R;
    cplx<T>* t = src;
    src = dst;
    dst = t;
  }
  return src;
}

__device__ __forceinline__ LineMap contiguous(int nlines) { return LineMap{nlines, 0}; }

}  // namespace sgo
