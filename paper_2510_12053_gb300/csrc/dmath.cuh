// Device arithmetic helpers: float-float ("df") numbers and small 3x3 algebra.
//
// A df number is an unevaluated sum hi + lo of two float32 values with
// |lo| <= ulp(hi) / 2, carrying about 48 significant bits.  The operations
// below are built from the classic error-free transformations:
//   * TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s = fl(a + b) and the exact error;
//   * FastTwoSum (Dekker 1971): the same when |a| >= |b|, in three operations;
//   * TwoProduct via fused multiply-add: p = fl(a b), e = fma(a, b, -p) exact.
// Addition uses the "sloppy" variant (one TwoSum on the high parts): its
// absolute error is a few units of 2^-46 times |a| + |b|, i.e. the same
// order as float64 rounding of the operands, which is what the gradient
// sums here need (their cancellation is between operands, not in the error).
// GB300 runs float32 at about 58x the float64 rate, so these are several
// times cheaper than native float64 for the gradient.
#pragma once

#include <cuda_runtime.h>

namespace ccg {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float h, float l) { return df{h, l}; }

__device__ __forceinline__ df df_from_double(double d) {
  float h = __double2float_rn(d);
  float l = __double2float_rn(d - (double)h);
  return df{h, l};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df{s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return df{s, e};
}

__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

// a * b + c
__device__ __forceinline__ df df_fma(df a, df b, df c) { return df_add(df_mul(a, b), c); }

__device__ __forceinline__ df df_scale(df a, float s) {
  float p = __fmul_rn(a.hi, s);
  float e = __fmaf_rn(a.hi, s, -p);
  e = __fmaf_rn(a.lo, s, e);
  return fast_two_sum(p, e);
}

// ---------------------------------------------------------------------------
// 3x3 helpers (row-major 9-arrays), templated on the scalar type
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void mat3_zero(T* a) {
#pragma unroll
  for (int k = 0; k < 9; ++k) a[k] = T(0);
}

// C += A * B
template <typename T>
__device__ __forceinline__ void mat3_mul_acc(const T* A, const T* B, T* C) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T s = C[3 * r + c];
#pragma unroll
      for (int k = 0; k < 3; ++k) s = fma(A[3 * r + k], B[3 * k + c], s);
      C[3 * r + c] = s;
    }
}

// C += A^T * B
template <typename T>
__device__ __forceinline__ void mat3_tmul_acc(const T* A, const T* B, T* C) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T s = C[3 * r + c];
#pragma unroll
      for (int k = 0; k < 3; ++k) s = fma(A[3 * k + r], B[3 * k + c], s);
      C[3 * r + c] = s;
    }
}

// Cholesky of a symmetric 3x3 (lower triangle read).  Returns false when a
// pivot is not above rel * max diagonal (or that maximum is not positive).
// L is stored row-major lower (L[3r+c], c <= r).
__device__ __forceinline__ bool chol3(const double* M, double* L, double rel) {
  double dmax = fmax(M[0], fmax(M[4], M[8]));
  if (!(dmax > 0.0)) return false;
  double thr = rel * dmax;
  double p0 = M[0];
  if (!(p0 > thr)) return false;
  double l00 = sqrt(p0);
  double l10 = M[3] / l00;
  double l20 = M[6] / l00;
  double p1 = M[4] - l10 * l10;
  if (!(p1 > thr)) return false;
  double l11 = sqrt(p1);
  double l21 = (M[7] - l20 * l10) / l11;
  double p2 = M[8] - l20 * l20 - l21 * l21;
  if (!(p2 > thr)) return false;
  double l22 = sqrt(p2);
  L[0] = l00; L[1] = 0; L[2] = 0;
  L[3] = l10; L[4] = l11; L[5] = 0;
  L[6] = l20; L[7] = l21; L[8] = l22;
  return true;
}

// Solve (L L^T) y = b in place.
__device__ __forceinline__ void chol3_solve(const double* L, double* b) {
  double y0 = b[0] / L[0];
  double y1 = (b[1] - L[3] * y0) / L[4];
  double y2 = (b[2] - L[6] * y0 - L[7] * y1) / L[8];
  double z2 = y2 / L[8];
  double z1 = (y1 - L[7] * z2) / L[4];
  double z0 = (y0 - L[3] * z1 - L[6] * z2) / L[0];
  b[0] = z0; b[1] = z1; b[2] = z2;
}

}  // namespace ccg

namespace ccg {

// float-float division a / b (one correction step on the float32 quotient)
__device__ __forceinline__ df df_div(df a, df b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const df r = df_sub(a, df_mul(b, df{q1, 0.0f}));
  const float q2 = __fdiv_rn(r.hi, b.hi);
  return fast_two_sum(q1, q2);
}

// Scalar arithmetic used by the batched 3x3 condensation, for float64 and
// for float-float.
template <typename T>
struct Arith;

template <>
struct Arith<double> {
  using V = double;
  static __device__ __forceinline__ V mk(double a) { return a; }
  static __device__ __forceinline__ V mkf(float a) { return (double)a; }
  static __device__ __forceinline__ V add(V a, V b) { return a + b; }
  static __device__ __forceinline__ V sub(V a, V b) { return a - b; }
  static __device__ __forceinline__ V mul(V a, V b) { return a * b; }
  static __device__ __forceinline__ V fma(V a, V b, V c) { return ::fma(a, b, c); }
  static __device__ __forceinline__ V div(V a, V b) { return a / b; }
  static __device__ __forceinline__ V neg(V a) { return -a; }
  static __device__ __forceinline__ bool gt(V a, V b) { return a > b; }
  static __device__ __forceinline__ double to_double(V a) { return a; }
};

template <>
struct Arith<df> {
  using V = df;
  static __device__ __forceinline__ V mk(double a) { return df_from_double(a); }
  static __device__ __forceinline__ V mkf(float a) { return df{a, 0.0f}; }
  static __device__ __forceinline__ V add(V a, V b) { return df_add(a, b); }
  static __device__ __forceinline__ V sub(V a, V b) { return df_sub(a, b); }
  static __device__ __forceinline__ V mul(V a, V b) { return df_mul(a, b); }
  static __device__ __forceinline__ V fma(V a, V b, V c) { return df_fma(a, b, c); }
  static __device__ __forceinline__ V div(V a, V b) { return df_div(a, b); }
  static __device__ __forceinline__ V neg(V a) { return df_neg(a); }
  static __device__ __forceinline__ bool gt(V a, V b) {
    const df d = df_sub(a, b);
    return d.hi > 0.0f || (d.hi == 0.0f && d.lo > 0.0f);
  }
  static __device__ __forceinline__ double to_double(V a) { return df_to_double(a); }
};

// Symmetric 3x3 (lower triangle of M read): adjugate in s[6] = (00 01 02 11 12 22)
// and determinant.  Returns false when M is not SPD by the pivot test: the
// Cholesky pivots M00, det2 / M00, det3 / det2 must all exceed rel * max diag.
template <typename T>
__device__ __forceinline__ bool sym3_adj(const typename Arith<T>::V* M, typename Arith<T>::V rel,
                                         typename Arith<T>::V* adj, typename Arith<T>::V* det) {
  using A = Arith<T>;
  using V = typename A::V;
  const V m00 = M[0], m10 = M[3], m20 = M[6], m11 = M[4], m21 = M[7], m22 = M[8];
  V dmax = m00;
  if (A::gt(m11, dmax)) dmax = m11;
  if (A::gt(m22, dmax)) dmax = m22;
  if (!A::gt(dmax, A::mkf(0.0f))) return false;
  const V thr = A::mul(rel, dmax);
  const V c00 = A::sub(A::mul(m11, m22), A::mul(m21, m21));
  const V c01 = A::sub(A::mul(m21, m20), A::mul(m10, m22));
  const V c02 = A::sub(A::mul(m10, m21), A::mul(m11, m20));
  const V c11 = A::sub(A::mul(m00, m22), A::mul(m20, m20));
  const V c12 = A::sub(A::mul(m10, m20), A::mul(m00, m21));
  const V c22 = A::sub(A::mul(m00, m11), A::mul(m10, m10));
  const V d3 = A::fma(m00, c00, A::fma(m10, c01, A::mul(m20, c02)));
  // pivots: p0 = m00, p1 = c22 / m00, p2 = d3 / c22
  if (!A::gt(m00, thr)) return false;
  if (!A::gt(c22, A::mul(thr, m00))) return false;
  if (!A::gt(d3, A::mul(thr, c22))) return false;
  adj[0] = c00; adj[1] = c01; adj[2] = c02; adj[3] = c11; adj[4] = c12; adj[5] = c22;
  *det = d3;
  return true;
}

}  // namespace ccg
