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

// o = a^{-1} (3x3 row-major, adjugate over determinant); returns det a.
template <typename T>
__device__ __forceinline__ T inv3t(const T* a, T* o) {
  const T c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
  const T det = a[0] * c00 + a[1] * c01 + a[2] * c02;
  const T id = T(1) / det;
  o[0] = c00 * id; o[3] = c01 * id; o[6] = c02 * id;
  o[1] = (a[2] * a[7] - a[1] * a[8]) * id;
  o[4] = (a[0] * a[8] - a[2] * a[6]) * id;
  o[7] = (a[1] * a[6] - a[0] * a[7]) * id;
  o[2] = (a[1] * a[5] - a[2] * a[4]) * id;
  o[5] = (a[2] * a[3] - a[0] * a[5]) * id;
  o[8] = (a[0] * a[4] - a[1] * a[3]) * id;
  return det;
}

// Orthogonal polar factor R of F (F = R S, S symmetric positive definite)
// for det F > 0, by Newton's iteration Y <- (g Y + (g Y)^{-T}) / 2 with
// Higham's scaling g = sqrt(|Y^{-1}|_F / |Y|_F), stopped when the update is
// below 64 units of roundoff of T (at most 40 steps).  Returns false (R
// untouched) when det F <= 0.
template <typename T>
__device__ __forceinline__ bool polar_newton(const T* F, T* R) {
  T Y[9], Yi[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) Y[q] = F[q];
  if (!(inv3t(Y, Yi) > T(0))) return false;
  const T tol = T(64) * (sizeof(T) == 8 ? T(1.1102230246251565e-16) : T(5.9604645e-08));
  for (int it = 0; it < 40; ++it) {
    T ny = 0, ni = 0;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      ny += Y[q] * Y[q];
      ni += Yi[q] * Yi[q];
    }
    const T g = sqrt(sqrt(ni / ny));
    T dn = 0, yn = 0;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T v = T(0.5) * (g * Y[3 * r + c] + Yi[3 * c + r] / g);
        dn += (v - Y[3 * r + c]) * (v - Y[3 * r + c]);
        yn += v * v;
        Y[3 * r + c] = v;
      }
    if (dn <= tol * tol * yn) break;
    inv3t(Y, Yi);
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) R[q] = Y[q];
  return true;
}

// Refines a float32 polar factor R0 of F to float-float accuracy.  R0 is
// near the polar factor R but neither exactly orthogonal nor exactly aligned:
// write R = R0 (I + X).  To first order, R^T R = I fixes the symmetric part
// of X at -D/2 with D = R0^T R0 - I, and R^T F symmetric fixes its skew part
// [w]x by
//   (tr(S) I - S) w = axial(S0 - S0^T) - axial(D S - S D) / 2,
// S0 = R0^T F, S = sym(S0) (with the identity [w]x S + S [w]x =
// [(tr(S) I - S) w]x for symmetric S).  D and the right side are float-float
// sums (their leading terms cancel); w and X, about float32 roundoff in size,
// are formed in float32, and R = R0 + R0 X in float-float: the error left is
// second order in R0's, about 1e-13.
__device__ __forceinline__ void polar_refine_df(const float* R32, const df* F, df* R) {
  df S[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      S[3 * r + c] = df_fma(df{R32[6 + r], 0.0f}, F[6 + c],
                            df_fma(df{R32[3 + r], 0.0f}, F[3 + c], df_mul(df{R32[r], 0.0f}, F[c])));
  float D[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      df d = df_fma(df{R32[6 + r], 0.0f}, df{R32[6 + c], 0.0f},
                    df_fma(df{R32[3 + r], 0.0f}, df{R32[3 + c], 0.0f}, df_mul(df{R32[r], 0.0f}, df{R32[c], 0.0f})));
      if (r == c) d = df_add(d, df{-1.0f, 0.0f});
      D[3 * r + c] = d.hi + d.lo;
    }
  float Ss[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) Ss[3 * r + c] = 0.5f * (S[3 * r + c].hi + S[3 * c + r].hi);
  // DS - SD is skew (D, S symmetric): its axial vector from the lower entries
  float DS[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      DS[3 * r + c] = (D[3 * r] * Ss[c] + D[3 * r + 1] * Ss[3 + c] + D[3 * r + 2] * Ss[6 + c]) -
                      (Ss[3 * r] * D[c] + Ss[3 * r + 1] * D[3 + c] + Ss[3 * r + 2] * D[6 + c]);
  const df a0 = df_sub(S[7], S[5]), a1 = df_sub(S[2], S[6]), a2 = df_sub(S[3], S[1]);
  const float rhs[3] = {(a0.hi + a0.lo) - 0.5f * DS[7], (a1.hi + a1.lo) - 0.5f * DS[2],
                        (a2.hi + a2.lo) - 0.5f * DS[3]};
  const float tr = Ss[0] + Ss[4] + Ss[8];
  float K[9], Ki[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) K[q] = -Ss[q];
  K[0] += tr;
  K[4] += tr;
  K[8] += tr;
  inv3t(K, Ki);
  float w[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) w[r] = Ki[3 * r] * rhs[0] + Ki[3 * r + 1] * rhs[1] + Ki[3 * r + 2] * rhs[2];
  const float X[9] = {-0.5f * D[0], -0.5f * D[1] - w[2], -0.5f * D[2] + w[1],
                      -0.5f * D[3] + w[2], -0.5f * D[4], -0.5f * D[5] - w[0],
                      -0.5f * D[6] - w[1], -0.5f * D[7] + w[0], -0.5f * D[8]};
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float d = R32[3 * r] * X[c] + R32[3 * r + 1] * X[3 + c] + R32[3 * r + 2] * X[6 + c];
      R[3 * r + c] = two_sum(R32[3 * r + c], d);
    }
}

// Fixed Corotational Hessian blocks (Sec. 4.1 material):
//   dP[dF] = 2 mu (dF - dR) + lam (C : dF) C + lam (J - 1) d2J/dF2 : dF,
//   dR = R [w]_x,  (tr(S) I - S) w = axial(R^T dF - dF^T R),  S = R^T F,
// evaluated for the nine unit directions E_cd and contracted with the shape
// vectors: block (v, w)[a][c] = V sum_{b,d} dP(E_cd)[a][b] G_v[b] G_w[d];
// the 10 upper blocks (pairs a <= b) into dst[9 pair + q].
template <typename T>
__device__ __forceinline__ void fcr_hess_blocks(const T* F, const T* R, const T* C, T J, T mu, T lam, T V,
                                                const T (&G)[4][3], T* __restrict__ dst) {
  T S[9], K[9], Ki[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) S[3 * r + c] = R[r] * F[c] + R[3 + r] * F[3 + c] + R[6 + r] * F[6 + c];
  const T tr = S[0] + S[4] + S[8];
#pragma unroll
  for (int q = 0; q < 9; ++q) K[q] = -S[q];
  K[0] += tr;
  K[4] += tr;
  K[8] += tr;
  inv3t(K, Ki);
#pragma unroll
  for (int q = 0; q < 90; ++q) dst[q] = T(0);
  const T s = lam * (J - T(1));
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      // R^T E_cd has column d = row c of R; its skew part's axial vector
      T ax[3];
      ax[0] = (d == 1 ? R[3 * c + 2] : T(0)) - (d == 2 ? R[3 * c + 1] : T(0));
      ax[1] = (d == 2 ? R[3 * c + 0] : T(0)) - (d == 0 ? R[3 * c + 2] : T(0));
      ax[2] = (d == 0 ? R[3 * c + 1] : T(0)) - (d == 1 ? R[3 * c + 0] : T(0));
      T w[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) w[i] = Ki[3 * i] * ax[0] + Ki[3 * i + 1] * ax[1] + Ki[3 * i + 2] * ax[2];
      // dR = R [w]_x, [w]_x = [[0, -w2, w1], [w2, 0, -w0], [-w1, w0, 0]]
      T dP[9];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const T r0 = R[3 * a], r1 = R[3 * a + 1], r2 = R[3 * a + 2];
        const T dR0 = r1 * w[2] - r2 * w[1];
        const T dR1 = r2 * w[0] - r0 * w[2];
        const T dR2 = r0 * w[1] - r1 * w[0];
        dP[3 * a + 0] = T(-2) * mu * dR0;
        dP[3 * a + 1] = T(-2) * mu * dR1;
        dP[3 * a + 2] = T(-2) * mu * dR2;
      }
      dP[3 * c + d] += T(2) * mu;
      const T cc = lam * C[3 * c + d];
#pragma unroll
      for (int q = 0; q < 9; ++q) dP[q] += cc * C[q];
      // d2J/dF_ab dF_cd = eps_ace eps_bdf F_ef: nonzero for a != c, b != d
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (a == c) continue;
        const int e = 3 - a - c;
        const T sa = ((c - a + 3) % 3 == 1) ? T(1) : T(-1);  // eps_ace
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          if (b == d) continue;
          const int f = 3 - b - d;
          const T sb = ((d - b + 3) % 3 == 1) ? T(1) : T(-1);  // eps_bdf
          dP[3 * a + b] += s * sa * sb * F[3 * e + f];
        }
      }
      T y[4][3];
#pragma unroll
      for (int v = 0; v < 4; ++v)
#pragma unroll
        for (int a = 0; a < 3; ++a) y[v][a] = dP[3 * a] * G[v][0] + dP[3 * a + 1] * G[v][1] + dP[3 * a + 2] * G[v][2];
      int pair = 0;
#pragma unroll
      for (int va = 0; va < 4; ++va)
#pragma unroll
        for (int vb = va; vb < 4; ++vb) {
          const T gw = V * G[vb][d];
#pragma unroll
          for (int a = 0; a < 3; ++a) dst[9 * pair + 3 * a + c] += y[va][a] * gw;
          ++pair;
        }
    }
}

}  // namespace ccg
