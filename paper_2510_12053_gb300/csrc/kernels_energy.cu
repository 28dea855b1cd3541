// Per-tet stable Neo-Hookean derivatives, vertex gathers and reductions.
//
// Energy (Eq. 2): E = 1/2 (x - xt)^T M (x - xt) + w sum_t V_t Psi(F_t),
// w = h^2 (dynamic) or 1 (quasistatic), F_t = D_s D_m^{-1}.
// With C = cof F, J = det F, s = lam_hat (J - 1) - mu:
//   P            = mu F + s C                                 (dPsi/dF)
//   dE_t/dx_v    = w V P G_v
//   d2E_t/dx_v dx_w = w V [ mu (G_v . G_w) I + lam_hat (C G_v)(C G_w)^T
//                           + s [F (G_v x G_w)]_skew ]
// where G_1..G_3 are the rows of D_m^{-1}, G_0 = -(G_1 + G_2 + G_3), and
// [q]_skew[a][c] = sum_e eps_ace q_e (the contraction of d2J/dF2 with G_v, G_w).
// Fixed Corotational (the paper's material, Sec. 4.1), with (mu, lam) in
// place of (mu, lam_hat) and R the polar rotation of F:
//   Psi = mu |F - R|^2 + lam/2 (J - 1)^2,  P = 2 mu (F - R) + lam (J - 1) C,
// Hessian blocks from fcr_hess_blocks.  An inverted tet (det F <= 0) has no
// rotation to extract here: its gradient entries become NaN, which the
// condensation reports as a non-finite update.
#include "cc_internal.cuh"
#include "dmath.cuh"

namespace ccg {

namespace {

constexpr int kBlock = 256;

inline unsigned grid_for(int64_t count, int block = kBlock) {
  int64_t g = (count + block - 1) / block;
  return (unsigned)(g < 1 ? 1 : g);
}

// ---- float64 per-tet kinematics ------------------------------------------
struct TetF64 {
  double F[9], C[9], J, G[4][3];
};

__device__ __forceinline__ void tet_kinematics_f64(const double (&p)[4][3], const double* B, TetF64& k) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double e0 = p[1][a] - p[0][a], e1 = p[2][a] - p[0][a], e2 = p[3][a] - p[0][a];
#pragma unroll
    for (int b = 0; b < 3; ++b) k.F[3 * a + b] = e0 * B[b] + e1 * B[3 + b] + e2 * B[6 + b];
  }
  // column b of C is (column b+1 of F) x (column b+2 of F)
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    int b1 = (b + 1) % 3, b2 = (b + 2) % 3;
    k.C[0 + b] = k.F[3 + b1] * k.F[6 + b2] - k.F[6 + b1] * k.F[3 + b2];
    k.C[3 + b] = k.F[6 + b1] * k.F[0 + b2] - k.F[0 + b1] * k.F[6 + b2];
    k.C[6 + b] = k.F[0 + b1] * k.F[3 + b2] - k.F[3 + b1] * k.F[0 + b2];
  }
  k.J = k.F[0] * k.C[0] + k.F[3] * k.C[3] + k.F[6] * k.C[6];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    k.G[1][b] = B[b];
    k.G[2][b] = B[3 + b];
    k.G[3][b] = B[6 + b];
    k.G[0][b] = -(B[b] + B[3 + b] + B[6 + b]);
  }
}

// Hessian block (v, w) without the w V factor.
template <typename T>
__device__ __forceinline__ void hess_block(const T* F, const T (&a_v)[3], const T (&a_w)[3],
                                           const T* Gv, const T* Gw, T mu, T lh, T s, T* K) {
  T gg = Gv[0] * Gw[0] + Gv[1] * Gw[1] + Gv[2] * Gw[2];
  T cr0 = Gv[1] * Gw[2] - Gv[2] * Gw[1];
  T cr1 = Gv[2] * Gw[0] - Gv[0] * Gw[2];
  T cr2 = Gv[0] * Gw[1] - Gv[1] * Gw[0];
  T q0 = F[0] * cr0 + F[1] * cr1 + F[2] * cr2;
  T q1 = F[3] * cr0 + F[4] * cr1 + F[5] * cr2;
  T q2 = F[6] * cr0 + F[7] * cr1 + F[8] * cr2;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) K[3 * r + c] = lh * a_v[r] * a_w[c];
  K[0] += mu * gg;
  K[4] += mu * gg;
  K[8] += mu * gg;
  K[1] += s * q2;
  K[2] -= s * q1;
  K[3] -= s * q2;
  K[5] += s * q0;
  K[6] += s * q1;
  K[7] -= s * q0;
}

// The tet's upper Hessian blocks V K_ab (corner pairs a <= b, order (0,0),
// (0,1), (0,2), (0,3), (1,1), (1,2), (1,3), (2,2), (2,3), (3,3)) in the
// per-tet store's layout (a diagonal block's upper triangle, the others 3x3
// row-major): pairs P0 <= pair < P1 from dst[0] on.
template <typename T, int P0 = 0, int P1 = 10>
__device__ __forceinline__ void tet_hess_blocks(const T* F, const T* C, T s, T mu, T lh, T V, const T (&G)[4][3],
                                                T* __restrict__ dst) {
  T a[4][3];
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int r = 0; r < 3; ++r) a[v][r] = C[3 * r] * G[v][0] + C[3 * r + 1] * G[v][1] + C[3 * r + 2] * G[v][2];
  int pair = 0;
#pragma unroll
  for (int va = 0; va < 4; ++va)
#pragma unroll
    for (int vb = va; vb < 4; ++vb) {
      if (pair >= P0 && pair < P1) {
        T K[9];
        hess_block<T>(F, a[va], a[vb], G[va], G[vb], mu, lh, s, K);
        T* d = dst + (tet_pair_offset(pair) - tet_pair_offset(P0));
        if (va == vb) {
          d[0] = V * K[0];
          d[1] = V * K[1];
          d[2] = V * K[2];
          d[3] = V * K[4];
          d[4] = V * K[5];
          d[5] = V * K[8];
        } else {
#pragma unroll
          for (int q = 0; q < 9; ++q) d[q] = V * K[q];
        }
      }
      ++pair;
    }
}

// Hessian staging.  Each thread stages its tet's blocks in shared memory at a
// per-thread pitch, then the warp copies every live tet's staged values to
// the per-tet store with coalesced stores (flush).  The SNH blocks are formed
// in the store's layout and flushed in two halves of five pairs (39 values,
// half the shared memory per thread, so more warps stay resident); FCR forms
// all ten 3x3 blocks at once (they accumulate over the nine directions of dF)
// and the flush keeps the diagonal blocks' upper triangles.  The pitches are
// odd so that the 32 lanes' k-th values fall in distinct banks.
template <bool kFCR>
struct TetStage {
  static constexpr int kVals = kFCR ? 90 : 39;  // staged values per tet (part)
  static constexpr int kPitch = kFCR ? 91 : 39;
};

// Staged index (full 3x3 blocks, 9 per pair) of value e of the store layout.
__device__ __forceinline__ int full_block_index(int e) {
  int pair = 0;
#pragma unroll
  for (int p = 1; p < 10; ++p) pair += e >= tet_pair_offset(p) ? 1 : 0;
  const int i = e - tet_pair_offset(pair);
  const int q = !tet_pair_is_diag(pair) ? i : (i < 3 ? i : (i < 5 ? i + 1 : 8));  // upper triangle 0 1 2 4 5 8
  return 9 * pair + q;
}

// Copies the warp's staged values (part `part` of each tet's record; with
// kFromFull the ten staged 3x3 blocks, compacted to the store's layout) to
// the per-tet store; t is this lane's tet (-1: none).  Every lane of the warp
// calls it.
template <typename T, int kVals, int kPitch, bool kFromFull = false>
__device__ __forceinline__ void flush_stage(const T* hstage, int t, int part, T* __restrict__ hten) {
  __syncwarp();
  const int lane = threadIdx.x & 31, wbase = threadIdx.x & ~31;
  constexpr int kOut = kFromFull ? tet_pair_offset(10) : kVals;
  for (int u = 0; u < 32; ++u) {
    const int tu = __shfl_sync(0xffffffffu, t, u);
    if (tu < 0) continue;
    const T* src = hstage + (wbase + u) * kPitch;
#pragma unroll
    for (int e = lane; e < kOut; e += 32)
      hten[(int64_t)tu * kTetStore + part * kVals + e] = src[kFromFull ? full_block_index(e) : e];
  }
  __syncwarp();
}

// ---- phase A: per-tet gradients and Hessian blocks of the tets whose vertices moved
__device__ __forceinline__ void tet_grad_f64_body(const int4* __restrict__ tets, const int4* __restrict__ tslot,
                                                  const double* __restrict__ Bm, const double* __restrict__ vol,
                                                  const uint8_t* __restrict__ pinned, const double* __restrict__ x,
                                                  int64_t n, int t, double mu, double lh, double weight,
                                                  double* __restrict__ gcon, double* __restrict__ hstage,
                                                  bool fcr, bool live, int t_store, double* __restrict__ hten) {
  const int4 tv = tets[t], ts = tslot[t];
  const int vid[4] = {tv.x, tv.y, tv.z, tv.w};
  const int ent[4] = {ts.x, ts.y, ts.z, ts.w};
  double p[4][3];
#pragma unroll
  for (int v = 0; v < 4; ++v)
#pragma unroll
    for (int a = 0; a < 3; ++a) p[v][a] = x[a * n + vid[v]];
  double B[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) B[q] = Bm[9 * (int64_t)t + q];
  TetF64 kin;
  tet_kinematics_f64(p, B, kin);
  const double s = lh * (kin.J - 1.0) - mu;
  const double V = vol[t] * weight;
  double P[9], R[9];
  if (fcr) {
    // lh holds lam for this material
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    if (!polar_newton<double>(kin.F, R))
      for (int q = 0; q < 9; ++q) R[q] = nan;
    const double sl = lh * (kin.J - 1.0);
#pragma unroll
    for (int q = 0; q < 9; ++q) P[q] = 2.0 * mu * (kin.F[q] - R[q]) + sl * kin.C[q];
  } else {
#pragma unroll
    for (int q = 0; q < 9; ++q) P[q] = mu * kin.F[q] + s * kin.C[q];
  }
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    if (!live || pinned[vid[v]]) continue;
    const int64_t e = ent[v];
#pragma unroll
    for (int r = 0; r < 3; ++r)
      gcon[3 * e + r] = V * (P[3 * r] * kin.G[v][0] + P[3 * r + 1] * kin.G[v][1] + P[3 * r + 2] * kin.G[v][2]);
  }
  double* hdst = hstage + threadIdx.x * (fcr ? TetStage<true>::kPitch : TetStage<false>::kPitch);
  if (fcr) {
    fcr_hess_blocks<double>(kin.F, R, kin.C, kin.J, mu, lh, V, kin.G, hdst);
    flush_stage<double, TetStage<true>::kVals, TetStage<true>::kPitch, true>(hstage, t_store, 0, hten);
  } else {
    tet_hess_blocks<double, 0, 5>(kin.F, kin.C, s, mu, lh, V, kin.G, hdst);
    flush_stage<double, TetStage<false>::kVals, TetStage<false>::kPitch>(hstage, t_store, 0, hten);
    tet_hess_blocks<double, 5, 10>(kin.F, kin.C, s, mu, lh, V, kin.G, hdst);
    flush_stage<double, TetStage<false>::kVals, TetStage<false>::kPitch>(hstage, t_store, 1, hten);
  }
}

// Float64 per-tet kernel; the Hessian blocks go through the shared-memory
// staging above.  Lanes past the list evaluate the list's first tet and store
// nothing (every lane takes part in the warp's flushes).
template <bool kFCR>
__global__ void k_tet_grad_f64(const int4* __restrict__ tets, const int4* __restrict__ tslot,
                               const double* __restrict__ Bm, const double* __restrict__ vol,
                               const uint8_t* __restrict__ pinned, const double* __restrict__ x, int64_t n,
                               const int32_t* __restrict__ list, int64_t count, const double2* __restrict__ mat,
                               double weight, double* __restrict__ gcon, double* __restrict__ hten) {
  pdl_entry();
  extern __shared__ __align__(16) double hstage64[];
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool live = k < count;
  const int t = live ? list[k] : -1;
  const int tc = live ? t : list[0];
  const double2 ml = mat[tc];
  tet_grad_f64_body(tets, tslot, Bm, vol, pinned, x, n, tc, ml.x, ml.y, weight, gcon, hstage64, kFCR, live, t,
                    hten);
}

__device__ __forceinline__ void tet_grad_mixed_body(const int4* __restrict__ tets, const int4* __restrict__ tslot,
                                                    const float2* __restrict__ Bm_df, const float2* __restrict__ volw,
                                                    const uint8_t* __restrict__ pinned, const float4* __restrict__ x_hi,
                                                    const float4* __restrict__ x_lo, int t, df mu_d, df lh_d,
                                                    float mu_f, float lh_f, const float* __restrict__ volw32,
                                                    float2* __restrict__ gcon, float* __restrict__ hstage, bool fcr,
                                                    bool live, int t_store, float* __restrict__ hten,
                                                    bool hess = true) {
  const int4 tv = tets[t], ts = tslot[t];
  const int vid[4] = {tv.x, tv.y, tv.z, tv.w};
  const int ent[4] = {ts.x, ts.y, ts.z, ts.w};
  df p[4][3];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    float4 h = x_hi[vid[v]], l = x_lo[vid[v]];
    p[v][0] = df{h.x, l.x};
    p[v][1] = df{h.y, l.y};
    p[v][2] = df{h.z, l.z};
  }
  df B[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    float2 b = Bm_df[9 * (int64_t)t + q];
    B[q] = df{b.x, b.y};
  }
  df F[9];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    df e0 = df_sub(p[1][a], p[0][a]), e1 = df_sub(p[2][a], p[0][a]), e2 = df_sub(p[3][a], p[0][a]);
#pragma unroll
    for (int b = 0; b < 3; ++b) F[3 * a + b] = df_fma(e2, B[6 + b], df_fma(e1, B[3 + b], df_mul(e0, B[b])));
  }
  df C[9];
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    int b1 = (b + 1) % 3, b2 = (b + 2) % 3;
    C[0 + b] = df_sub(df_mul(F[3 + b1], F[6 + b2]), df_mul(F[6 + b1], F[3 + b2]));
    C[3 + b] = df_sub(df_mul(F[6 + b1], F[0 + b2]), df_mul(F[0 + b1], F[6 + b2]));
    C[6 + b] = df_sub(df_mul(F[0 + b1], F[3 + b2]), df_mul(F[3 + b1], F[0 + b2]));
  }
  df J = df_fma(F[6], C[6], df_fma(F[3], C[3], df_mul(F[0], C[0])));
  df Jm1 = df_add(J, df{-1.0f, 0.0f});
  df s = df_sub(df_mul(lh_d, Jm1), mu_d);
  const float2 vw = volw[t];
  const df V{vw.x, vw.y};
  df P[9];
  float R32[9];
  if (fcr) {
    // lh holds lam for this material; R to float32 by Newton, then one
    // float-float correction against the full F
    float Fh[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) Fh[q] = F[q].hi;
    df R[9];
    if (polar_newton<float>(Fh, R32)) {
      polar_refine_df(R32, F, R);
    } else {
      const float nan = __int_as_float(0x7fc00000);
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        R32[q] = nan;
        R[q] = df{nan, 0.0f};
      }
    }
    const df sl = df_mul(lh_d, Jm1), mu2 = df_scale(mu_d, 2.0f);
#pragma unroll
    for (int q = 0; q < 9; ++q) P[q] = df_mul(V, df_fma(mu2, df_sub(F[q], R[q]), df_mul(sl, C[q])));
  } else {
#pragma unroll
    for (int q = 0; q < 9; ++q) P[q] = df_mul(V, df_fma(mu_d, F[q], df_mul(s, C[q])));
  }
  df g[4][3];
#pragma unroll
  for (int v = 1; v < 4; ++v)
#pragma unroll
    for (int r = 0; r < 3; ++r)
      g[v][r] = df_fma(P[3 * r + 2], B[3 * (v - 1) + 2],
                       df_fma(P[3 * r + 1], B[3 * (v - 1) + 1], df_mul(P[3 * r], B[3 * (v - 1)])));
#pragma unroll
  for (int r = 0; r < 3; ++r) g[0][r] = df_neg(df_add(df_add(g[1][r], g[2][r]), g[3][r]));
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    if (!live || pinned[vid[v]]) continue;
    const int64_t e = ent[v];
#pragma unroll
    for (int r = 0; r < 3; ++r) gcon[3 * e + r] = make_float2(g[v][r].hi, g[v][r].lo);
  }
  if (!hess) return;  // the rows are built from the positions (k_row_build)
  // float32 Hessian blocks from the high parts
  float Ff[9], Cf[9], G[4][3];
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    Ff[q] = F[q].hi;
    Cf[q] = C[q].hi;
  }
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    G[1][b] = B[b].hi;
    G[2][b] = B[3 + b].hi;
    G[3][b] = B[6 + b].hi;
    G[0][b] = -(G[1][b] + G[2][b] + G[3][b]);
  }
  float* hdst = hstage + threadIdx.x * (fcr ? TetStage<true>::kPitch : TetStage<false>::kPitch);
  const float V32 = volw32[t];
  if (fcr) {
    fcr_hess_blocks<float>(Ff, R32, Cf, J.hi, mu_f, lh_f, V32, G, hdst);
    flush_stage<float, TetStage<true>::kVals, TetStage<true>::kPitch, true>(hstage, t_store, 0, hten);
  } else {
    tet_hess_blocks<float, 0, 5>(Ff, Cf, s.hi, mu_f, lh_f, V32, G, hdst);
    flush_stage<float, TetStage<false>::kVals, TetStage<false>::kPitch>(hstage, t_store, 0, hten);
    tet_hess_blocks<float, 5, 10>(Ff, Cf, s.hi, mu_f, lh_f, V32, G, hdst);
    flush_stage<float, TetStage<false>::kVals, TetStage<false>::kPitch>(hstage, t_store, 1, hten);
  }
}

// Float-float per-tet kernel (gradient in float-float, Hessian blocks in
// float32 through the shared-memory staging above).  Lanes past the list
// evaluate the list's first tet and store nothing.
template <bool kFCR, bool kHess = true>
__global__ void k_tet_grad_mixed(const int4* __restrict__ tets, const int4* __restrict__ tslot,
                                 const float2* __restrict__ Bm_df, const float2* __restrict__ volw,
                                 const uint8_t* __restrict__ pinned, const float4* __restrict__ x_hi,
                                 const float4* __restrict__ x_lo, const int32_t* __restrict__ list, int64_t count,
                                 const float4* __restrict__ matdf, const float* __restrict__ volw32,
                                 float2* __restrict__ gcon, float* __restrict__ hten) {
  pdl_entry();
  extern __shared__ __align__(16) float hstage[];
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool live = k < count;
  const int t = live ? list[k] : -1;
  const int tc = live ? t : list[0];
  const float4 ml = matdf[tc];  // (mu hi, mu lo, lam_hat hi, lam_hat lo)
  tet_grad_mixed_body(tets, tslot, Bm_df, volw, pinned, x_hi, x_lo, tc, df{ml.x, ml.y}, df{ml.z, ml.w}, ml.x, ml.z,
                      volw32, gcon, hstage, kFCR, live, t, hten, kHess);
}

// Gradient of free row j from its per-(vertex, slot) entries e0 .. e0 + val - 1
// (plus the inertial term of dynamic solves).
template <bool kMixed>
__device__ __forceinline__ void row_gradient(int j, int e0, int val, int lane, const double* __restrict__ gcon64,
                                             const float2* __restrict__ gcon_df, const double* __restrict__ mass64,
                                             const float2* __restrict__ mass_df, const double* __restrict__ x,
                                             const float4* __restrict__ x_hi, const float4* __restrict__ x_lo,
                                             const double* __restrict__ xt, const float4* __restrict__ xt_hi,
                                             const float4* __restrict__ xt_lo, int64_t n, bool dynamic,
                                             double* __restrict__ g64, float* __restrict__ g_hi,
                                             float* __restrict__ g_lo) {
  // gradient: lane 8a + p (component a < 3, p < 8) sums the entries p, p + 8,
  // ... of component a in order, then a fixed butterfly over its eight lanes
  // finishes the sum (lanes 24..31 carry zeros through the shuffles)
  const int ga = lane >> 3, gp = lane & 7;
  if (kMixed) {
    df gd{0.0f, 0.0f};
    if (ga < 3)
      for (int k = gp; k < val; k += 8) {
        const float2 cc = gcon_df[3 * (int64_t)(e0 + k) + ga];
        gd = df_add(gd, df{cc.x, cc.y});
      }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      const df other{__shfl_xor_sync(0xffffffffu, gd.hi, o), __shfl_xor_sync(0xffffffffu, gd.lo, o)};
      gd = df_add(gd, other);
    }
    if (ga < 3 && gp == 0) {
      if (dynamic) {
        const df mj{mass_df[j].x, mass_df[j].y};
        const float xh = reinterpret_cast<const float*>(x_hi + j)[ga];
        const float xl = reinterpret_cast<const float*>(x_lo + j)[ga];
        const float th = reinterpret_cast<const float*>(xt_hi + j)[ga];
        const float tl = reinterpret_cast<const float*>(xt_lo + j)[ga];
        gd = df_fma(mj, df_sub(df{xh, xl}, df{th, tl}), gd);
      }
      g_hi[3 * (int64_t)j + ga] = gd.hi;
      g_lo[3 * (int64_t)j + ga] = gd.lo;
    }
  } else {
    double gs = 0.0;
    if (ga < 3)
      for (int k = gp; k < val; k += 8) gs += gcon64[3 * (int64_t)(e0 + k) + ga];
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) gs += __shfl_xor_sync(0xffffffffu, gs, o);
    if (ga < 3 && gp == 0) {
      if (dynamic) gs += mass64[j] * (x[ga * n + j] - xt[ga * n + j]);
      g64[3 * (int64_t)j + ga] = gs;
    }
  }
}

// ---- phase B: one warp per free row j ---------------------------------------
// Every upper block (j, l) of the row sums its sources -- the stored blocks of
// the incident tets, transposed where the tet lists l before j -- in a fixed
// order, one lane per (block, component): the diagonal block's 24-odd
// sources (the tets' diagonal blocks, stored as upper triangles) are split
// over three groups of nine lanes, the other blocks take nine lanes each,
// three per round.  Blocks are written padded to 3 x 4.  The
// row's gradient is the fixed-butterfly sum of its per-(vertex, slot) entries.
// A row starts from its 32-byte record (row id, block and source ranges,
// entry range), so the index chain before the stored blocks are read is two
// loads deep; the gradient, which needs only the record, is summed first.
template <typename HT, bool kMixed>
__global__ void k_row_gather(const int4* __restrict__ row_hdr, int64_t nrows, const int32_t* __restrict__ rs_ptr,
                             const int32_t* __restrict__ rs_src, const HT* __restrict__ hten,
                             const HT* __restrict__ massh, const double* __restrict__ mass64,
                             const float2* __restrict__ mass_df, const double* __restrict__ gcon64,
                             const float2* __restrict__ gcon_df, const double* __restrict__ x,
                             const float4* __restrict__ x_hi, const float4* __restrict__ x_lo,
                             const double* __restrict__ xt, const float4* __restrict__ xt_hi,
                             const float4* __restrict__ xt_lo, int64_t n, bool dynamic, int max_rs, int max_up,
                             HT* __restrict__ bsr, double* __restrict__ g64, float* __restrict__ g_hi,
                             float* __restrict__ g_lo) {
  pdl_entry();
  extern __shared__ int rsh[];
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5, warp = threadIdx.x >> 5;
  const int64_t wid = (int64_t)blockIdx.x * wpb + warp;
  if (wid >= nrows) return;
  const int4 h0 = __ldg(row_hdr + 2 * wid), h1 = __ldg(row_hdr + 2 * wid + 1);
  const int j = h0.x, p0 = h0.y, nup = h0.z, rb = h0.w, rcount = h1.x;
  row_gradient<kMixed>(j, h1.y, h1.z, lane, gcon64, gcon_df, mass64, mass_df, x, x_hi, x_lo, xt, xt_hi, xt_lo, n,
                       dynamic, g64, g_hi, g_lo);
  const int c = lane % 9, grp = lane / 9, r = c / 3, col = c % 3;
  const int tidx = 3 * col + r;
  // element (r, col) of a stored diagonal block (its upper triangle)
  const int lo = min(r, col), hi = max(r, col);
  const int sym = lo == 0 ? hi : (lo == 1 ? hi + 2 : 5);
  // the row's source offsets and per-block ranges, one coalesced pass
  int* roff = rsh + warp * (max_rs + max_up + 1);
  int* rsrc = roff + max_up + 1;
  for (int q = lane; q <= nup; q += 32) roff[q] = rs_ptr[p0 + q] - rb;
  for (int k = lane; k < rcount; k += 32) rsrc[k] = rs_src[rb + k];
  __syncwarp();

  // diagonal block
  {
    HT acc = HT(0);
    if (grp < 3) {
      const int s1 = roff[1];
#pragma unroll 4
      for (int s = grp; s < s1; s += 3) acc += hten[rsrc[s] + sym];  // diagonal pairs: never transposed
    }
    const HT a1 = __shfl_down_sync(0xffffffffu, acc, 9);
    const HT a2 = __shfl_down_sync(0xffffffffu, acc, 18);
    if (lane < 9) {
      HT d = (acc + a1) + a2;
      if (dynamic && r == col) d += massh[j];
      HT* dst = bsr + (int64_t)p0 * 12 + 4 * r;
      dst[col] = d;
      if (col == 2) dst[3] = HT(0);
    }
  }
  // off-diagonal upper blocks, three per round
  for (int base = 1; base < nup; base += 3) {
    const int q = base + grp;
    if (grp < 3 && q < nup) {
      HT acc = HT(0);
      const int s1 = roff[q + 1];
#pragma unroll 4
      for (int s = roff[q]; s < s1; ++s) {
        const int v = rsrc[s];
        acc += hten[(v & 0x7fffffff) + (v < 0 ? tidx : c)];
      }
      HT* dst = bsr + (int64_t)(p0 + q) * 12 + 4 * r;
      dst[col] = acc;
      if (col == 2) dst[3] = HT(0);
    }
  }
}

// ---- phase B without the per-tet store (mixed path, stable Neo-Hookean) ----
// One warp per free row j.  The gradient is summed from the per-(vertex,
// slot) entries exactly as in k_row_gather.  The upper block row is formed
// from the positions instead of a stored Hessian: lane k takes the row's k-th
// incident tet (ascending tet id), forms F = D_s D_m^{-1} in float32 (edge
// vectors from the float-float position mirror, so they carry full float32
// accuracy), cof F and J, and the blocks K_{cj,w} = d2E_t/dx_j dx_w of every
// corner w whose vertex id is >= j (float32, the formula of hess_block),
// staged in shared memory.  Lanes (block, component) then sum each block's
// sources -- the row-local codes k * 4 + w of the upper blocks, ascending --
// in the same fixed order as the gather.  Each tet's kinematics are formed
// by its four rows, but no Hessian value goes through global memory.
template <int kMaxVal>
__global__ void __launch_bounds__(128) k_row_build(
    const int4* __restrict__ row_hdr, int64_t nrows, const int32_t* __restrict__ rs_ptr,
    const uint16_t* __restrict__ rs_loc, const int32_t* __restrict__ vt_tet, const uint8_t* __restrict__ vt_corner,
    const int4* __restrict__ vt_ids, const float4* __restrict__ Bm32p, const float* __restrict__ volw32,
    const float4* __restrict__ matdf, const float4* __restrict__ x_hi, const float4* __restrict__ x_lo,
    const float* __restrict__ mass32, const float2* __restrict__ mass_df, const float2* __restrict__ gcon_df,
    const float4* __restrict__ xt_hi, const float4* __restrict__ xt_lo, bool dynamic, int max_rs, int max_up,
    float* __restrict__ bsr, float* __restrict__ g_hi, float* __restrict__ g_lo) {
  pdl_entry();
  constexpr int kPitch = 37;  // odd: the lanes' staged blocks start in distinct banks
  extern __shared__ __align__(16) float rb_smem[];
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5, warp = threadIdx.x >> 5;
  const int64_t wid = (int64_t)blockIdx.x * wpb + warp;
  if (wid >= nrows) return;
  float* stage = rb_smem + warp * (kMaxVal * kPitch);
  int* roff = reinterpret_cast<int*>(rb_smem + wpb * (kMaxVal * kPitch)) + warp * (max_up + 1 + (max_rs + 1) / 2);
  uint16_t* rloc = reinterpret_cast<uint16_t*>(roff + max_up + 1);
  const int4 h0 = __ldg(row_hdr + 2 * wid), h1 = __ldg(row_hdr + 2 * wid + 1);
  const int j = h0.x, p0 = h0.y, nup = h0.z, rb = h0.w, rcount = h1.x, e0 = h1.y, val = h1.z;
  row_gradient<true>(j, e0, val, lane, nullptr, gcon_df, nullptr, mass_df, nullptr, x_hi, x_lo, nullptr, xt_hi,
                     xt_lo, 0, dynamic, nullptr, g_hi, g_lo);
  for (int q = lane; q <= nup; q += 32) roff[q] = rs_ptr[p0 + q] - rb;
  for (int k = lane; k < rcount; k += 32) rloc[k] = rs_loc[rb + k];
  for (int k = lane; k < val; k += 32) {
    const int t = vt_tet[e0 + k];
    const int cj = vt_corner[e0 + k];
    const int4 tv = vt_ids[e0 + k];  // the tet's vertex ids, stored per entry: no load waits for t
    const int vid[4] = {tv.x, tv.y, tv.z, tv.w};
    float4 ph[4], pl[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      ph[v] = x_hi[vid[v]];
      pl[v] = x_lo[vid[v]];
    }
    const float4 b0 = Bm32p[3 * (int64_t)t], b1 = Bm32p[3 * (int64_t)t + 1], b2 = Bm32p[3 * (int64_t)t + 2];
    float G[4][3] = {{-(b0.x + b1.x + b2.x), -(b0.y + b1.y + b2.y), -(b0.z + b1.z + b2.z)},
                     {b0.x, b0.y, b0.z}, {b1.x, b1.y, b1.z}, {b2.x, b2.y, b2.z}};
    float F[9];
    {
      float e[3][3];  // e[v - 1][a]: edge x_v - x_0
#pragma unroll
      for (int v = 1; v < 4; ++v) {
        e[v - 1][0] = (ph[v].x - ph[0].x) + (pl[v].x - pl[0].x);
        e[v - 1][1] = (ph[v].y - ph[0].y) + (pl[v].y - pl[0].y);
        e[v - 1][2] = (ph[v].z - ph[0].z) + (pl[v].z - pl[0].z);
      }
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) F[3 * a + b] = fmaf(e[2][a], G[3][b], fmaf(e[1][a], G[2][b], e[0][a] * G[1][b]));
    }
    float C[9];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int b1i = (b + 1) % 3, b2i = (b + 2) % 3;
      C[0 + b] = F[3 + b1i] * F[6 + b2i] - F[6 + b1i] * F[3 + b2i];
      C[3 + b] = F[6 + b1i] * F[0 + b2i] - F[0 + b1i] * F[6 + b2i];
      C[6 + b] = F[0 + b1i] * F[3 + b2i] - F[3 + b1i] * F[0 + b2i];
    }
    const float J = F[0] * C[0] + F[3] * C[3] + F[6] * C[6];
    const float4 ml = matdf[t];  // (mu hi, mu lo, lam_hat hi, lam_hat lo)
    const float mu = ml.x, lh = ml.z, V = volw32[t];
    const float sJ = lh * (J - 1.0f) - mu;
    float a[4][3];
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int r = 0; r < 3; ++r) a[v][r] = C[3 * r] * G[v][0] + C[3 * r + 1] * G[v][1] + C[3 * r + 2] * G[v][2];
    float aj[3], Gj[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      aj[r] = cj == 0 ? a[0][r] : cj == 1 ? a[1][r] : cj == 2 ? a[2][r] : a[3][r];
      Gj[r] = cj == 0 ? G[0][r] : cj == 1 ? G[1][r] : cj == 2 ? G[2][r] : G[3][r];
    }
    float* dst = stage + k * kPitch;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      if (vid[w] < j) continue;
      float K[9];
      hess_block<float>(F, aj, a[w], Gj, G[w], mu, lh, sJ, K);
#pragma unroll
      for (int q = 0; q < 9; ++q) dst[9 * w + q] = V * K[q];
    }
  }
  __syncwarp();
  const int c = lane % 9, grp = lane / 9, r = c / 3, col = c % 3;
  // diagonal block: one source per incident tet, three interleaved partial sums
  {
    float acc = 0.0f;
    if (grp < 3) {
      const int s1 = roff[1];
      for (int s = grp; s < s1; s += 3) {
        const int code = rloc[s];
        acc += stage[(code >> 2) * kPitch + 9 * (code & 3) + c];
      }
    }
    const float a1 = __shfl_down_sync(0xffffffffu, acc, 9);
    const float a2 = __shfl_down_sync(0xffffffffu, acc, 18);
    if (lane < 9) {
      float d = (acc + a1) + a2;
      if (dynamic && r == col) d += mass32[j];
      float* dst = bsr + (int64_t)p0 * 12 + 4 * r;
      dst[col] = d;
      if (col == 2) dst[3] = 0.0f;
    }
  }
  // off-diagonal upper blocks, three per round
  for (int base = 1; base < nup; base += 3) {
    const int q = base + grp;
    if (grp < 3 && q < nup) {
      float acc = 0.0f;
      const int s1 = roff[q + 1];
      for (int s = roff[q]; s < s1; ++s) {
        const int code = rloc[s];
        acc += stage[(code >> 2) * kPitch + 9 * (code & 3) + c];
      }
      float* dst = bsr + (int64_t)(p0 + q) * 12 + 4 * r;
      dst[col] = acc;
      if (col == 2) dst[3] = 0.0f;
    }
  }
}

// ---- reductions --------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (wid == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  __syncthreads();
  return v;
}

// Stage 2: sums `count` partials in a fixed order, out[0] = result.
__global__ void k_reduce_final(const double* __restrict__ part, int64_t count, double* __restrict__ out) {
  pdl_entry();
  double v = 0.0;
  for (int64_t k = threadIdx.x; k < count; k += blockDim.x) v += part[k];
  v = block_sum(v);
  if (threadIdx.x == 0) out[0] = v;
}

template <bool kFCR>
__global__ void k_energy_tets(const int4* __restrict__ tets, const double* __restrict__ Bm,
                              const double* __restrict__ vol, const double* __restrict__ x, int64_t n,
                              int64_t T, const double2* __restrict__ mat, double weight, double* __restrict__ part) {
  pdl_entry();
  double e = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < T; t += (int64_t)gridDim.x * blockDim.x) {
    const int4 tv = tets[t];
    const int vid[4] = {tv.x, tv.y, tv.z, tv.w};
    double p[4][3];
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int a = 0; a < 3; ++a) p[v][a] = x[a * n + vid[v]];
    double B[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) B[q] = Bm[9 * t + q];
    TetF64 kin;
    tet_kinematics_f64(p, B, kin);
    const double Jm1 = kin.J - 1.0;
    const double mu = mat[t].x, lh = mat[t].y;
    if (kFCR) {
      double R[9];
      double d2 = 0.0;
      if (polar_newton<double>(kin.F, R)) {
#pragma unroll
        for (int q = 0; q < 9; ++q) d2 += (kin.F[q] - R[q]) * (kin.F[q] - R[q]);
      } else {
        d2 = __longlong_as_double(0x7ff8000000000000ll);
      }
      e += weight * vol[t] * (mu * d2 + 0.5 * lh * Jm1 * Jm1);
    } else {
      double I = 0.0;
#pragma unroll
      for (int q = 0; q < 9; ++q) I += kin.F[q] * kin.F[q];
      e += weight * vol[t] * (0.5 * mu * (I - 3.0) - mu * Jm1 + 0.5 * lh * Jm1 * Jm1);
    }
  }
  e = block_sum(e);
  if (threadIdx.x == 0) part[blockIdx.x] = e;
}

// Energy of every mesh of a batch (Eq. 2 per mesh): one CTA per mesh over its
// tets [tptr[b], tptr[b+1]) and, when dynamic, its vertices, in a fixed order.
template <bool kFCR>
__global__ void k_energy_mesh(const int64_t* __restrict__ tptr, const int64_t* __restrict__ vptr,
                              const int4* __restrict__ tets, const double* __restrict__ Bm,
                              const double* __restrict__ vol, const double* __restrict__ x, int64_t n,
                              const double2* __restrict__ mat, double weight, const double* __restrict__ mass,
                              const double* __restrict__ xt, double* __restrict__ out) {
  pdl_entry();
  const int b = blockIdx.x;
  double e = 0.0;
  for (int64_t t = tptr[b] + threadIdx.x; t < tptr[b + 1]; t += blockDim.x) {
    const int4 tv = tets[t];
    const int vid[4] = {tv.x, tv.y, tv.z, tv.w};
    double p[4][3];
#pragma unroll
    for (int v = 0; v < 4; ++v)
#pragma unroll
      for (int a = 0; a < 3; ++a) p[v][a] = x[a * n + vid[v]];
    double B[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) B[q] = Bm[9 * t + q];
    TetF64 kin;
    tet_kinematics_f64(p, B, kin);
    const double Jm1 = kin.J - 1.0;
    const double mu = mat[t].x, lh = mat[t].y;
    if (kFCR) {
      double R[9];
      double d2 = 0.0;
      if (polar_newton<double>(kin.F, R)) {
#pragma unroll
        for (int q = 0; q < 9; ++q) d2 += (kin.F[q] - R[q]) * (kin.F[q] - R[q]);
      } else {
        d2 = __longlong_as_double(0x7ff8000000000000ll);
      }
      e += weight * vol[t] * (mu * d2 + 0.5 * lh * Jm1 * Jm1);
    } else {
      double I = 0.0;
#pragma unroll
      for (int q = 0; q < 9; ++q) I += kin.F[q] * kin.F[q];
      e += weight * vol[t] * (0.5 * mu * (I - 3.0) - mu * Jm1 + 0.5 * lh * Jm1 * Jm1);
    }
  }
  if (xt)
    for (int64_t j = vptr[b] + threadIdx.x; j < vptr[b + 1]; j += blockDim.x) {
      const double d0 = x[j] - xt[j], d1 = x[n + j] - xt[n + j], d2 = x[2 * n + j] - xt[2 * n + j];
      e += 0.5 * mass[j] * (d0 * d0 + d1 * d1 + d2 * d2);
    }
  e = block_sum(e);
  if (threadIdx.x == 0) out[b] = e;
}

// x = x0 + alpha[mesh of the vertex] (x1 - x0), all 3n entries.
__global__ void k_line_point_mesh(const double* __restrict__ x0, const double* __restrict__ x1, int64_t n,
                                  const int32_t* __restrict__ vert_mesh, const double* __restrict__ alpha,
                                  double* __restrict__ x) {
  pdl_entry();
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= 3 * n) return;
  const double a = alpha[vert_mesh[k % n]];
  x[k] = x0[k] + a * (x1[k] - x0[k]);
}

__global__ void k_energy_inertia(const double* __restrict__ mass, const double* __restrict__ x,
                                 const double* __restrict__ xt, int64_t n, double* __restrict__ part) {
  pdl_entry();
  double e = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    double d0 = x[j] - xt[j], d1 = x[n + j] - xt[n + j], d2 = x[2 * n + j] - xt[2 * n + j];
    e += 0.5 * mass[j] * (d0 * d0 + d1 * d1 + d2 * d2);
  }
  e = block_sum(e);
  if (threadIdx.x == 0) part[blockIdx.x] = e;
}

template <bool kMixed>
__global__ void k_gnorm(const int32_t* __restrict__ free_rows, int64_t nfree, const double* __restrict__ g64,
                        const float* __restrict__ g_hi, const float* __restrict__ g_lo, int64_t n,
                        double* __restrict__ grad_out, double* __restrict__ part) {
  pdl_entry();
  double acc = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nfree; k += (int64_t)gridDim.x * blockDim.x) {
    const int j = free_rows[k];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double v = kMixed ? (double)g_hi[3 * (int64_t)j + a] + (double)g_lo[3 * (int64_t)j + a]
                        : g64[3 * (int64_t)j + a];
      acc += v * v;
      if (grad_out) grad_out[a * n + j] = v;
    }
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// Squared free gradient norm of every mesh of a batch: one CTA per mesh over
// its contiguous range of free rows, fixed-order block reduction.
template <bool kMixed>
__global__ void k_gnorm_mesh(const int32_t* __restrict__ fptr, const int32_t* __restrict__ free_rows,
                             const double* __restrict__ g64, const float* __restrict__ g_hi,
                             const float* __restrict__ g_lo, double* __restrict__ gsq) {
  pdl_entry();
  const int b = blockIdx.x;
  double acc = 0.0;
  for (int k = fptr[b] + threadIdx.x; k < fptr[b + 1]; k += blockDim.x) {
    const int j = free_rows[k];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double v = kMixed ? (double)g_hi[3 * (int64_t)j + a] + (double)g_lo[3 * (int64_t)j + a]
                              : g64[3 * (int64_t)j + a];
      acc += v * v;
    }
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) gsq[b] = acc;
}

__global__ void k_split_df(const double* __restrict__ x, int64_t n, float4* __restrict__ hi,
                           float4* __restrict__ lo) {
  pdl_entry();
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  df a = df_from_double(x[j]), b = df_from_double(x[n + j]), c = df_from_double(x[2 * n + j]);
  hi[j] = make_float4(a.hi, b.hi, c.hi, 0.f);
  lo[j] = make_float4(a.lo, b.lo, c.lo, 0.f);
}

__global__ void k_inertial_target(const double* __restrict__ x, const double* __restrict__ v, int64_t n,
                                  double h, double g0, double g1, double g2, double* __restrict__ xt) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double gg[3] = {g0, g1, g2};
#pragma unroll
  for (int a = 0; a < 3; ++a) xt[a * n + j] = x[a * n + j] + h * v[a * n + j] + h * h * gg[a];
}

__global__ void k_velocity(const double* __restrict__ x, const double* __restrict__ xold, int64_t n, double h,
                           double* __restrict__ v) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= 3 * n) return;
  v[k] = (x[k] - xold[k]) / h;
}

__global__ void k_line_point(const double* __restrict__ x0, const double* __restrict__ x1, int64_t n, double alpha,
                             double* __restrict__ x) {
  pdl_entry();
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= 3 * n) return;
  x[k] = x0[k] + alpha * (x1[k] - x0[k]);
}

constexpr int kRedBlocks = 1024;

}  // namespace

// ---------------------------------------------------------------------------
void launch_tet_grad_f64(Mesh& m, const double* x, const int32_t* list, int64_t count, double weight,
                         cudaStream_t s) {
  if (count <= 0) return;
  constexpr int kThreads = 64;
  const bool fcr = m.model == CC_MODEL_FCR;
  const size_t smem =
      (size_t)kThreads * (fcr ? TetStage<true>::kPitch : TetStage<false>::kPitch) * sizeof(double);
  auto kern = fcr ? k_tet_grad_f64<true> : k_tet_grad_f64<false>;
  set_smem_limit(reinterpret_cast<const void*>(kern), smem);
  pdl_launch(kern, grid_for(count, kThreads), kThreads, smem, s, (const int4*)m.d_tets.p, (const int4*)m.d_tslot.p,
             (const double*)m.d_Bm.p, (const double*)m.d_vol.p, (const uint8_t*)m.d_pinned.p, x, m.n, list, count,
             (const double2*)m.d_mat64.p, weight, m.f64.gcon.p, m.f64.hten.p);
}

void launch_tet_grad_mixed(Mesh& m, const int32_t* list, int64_t count, double weight, cudaStream_t s) {
  if (count <= 0) return;
  (void)weight;
  constexpr int kThreads = 128;
  const bool fcr = m.model == CC_MODEL_FCR;
  if (rows_from_positions(m)) {
    pdl_launch(k_tet_grad_mixed<false, false>, grid_for(count, kThreads), kThreads, 0, s, (const int4*)m.d_tets.p,
               (const int4*)m.d_tslot.p, (const float2*)m.d_Bm_df.p, (const float2*)m.d_volw_df.p,
               (const uint8_t*)m.d_pinned.p, (const float4*)m.mx.x_hi.p, (const float4*)m.mx.x_lo.p, list, count,
               (const float4*)m.d_matdf.p, (const float*)m.d_volw32.p, m.mx.gcon.p, (float*)nullptr);
    return;
  }
  const size_t smem = (size_t)kThreads * (fcr ? TetStage<true>::kPitch : TetStage<false>::kPitch) * sizeof(float);
  auto kern = fcr ? k_tet_grad_mixed<true> : k_tet_grad_mixed<false>;
  set_smem_limit(reinterpret_cast<const void*>(kern), smem);
  pdl_launch(kern, grid_for(count, kThreads), kThreads, smem, s, (const int4*)m.d_tets.p, (const int4*)m.d_tslot.p,
             (const float2*)m.d_Bm_df.p, (const float2*)m.d_volw_df.p, (const uint8_t*)m.d_pinned.p,
             (const float4*)m.mx.x_hi.p, (const float4*)m.mx.x_lo.p, list, count, (const float4*)m.d_matdf.p,
             (const float*)m.d_volw32.p, m.mx.gcon.p, m.mx.hten.p);
}

template <typename HT, bool kMixed>
static void launch_rows(Mesh& m, const double* x, const double* xt, HT* bsr, const HT* hten, const HT* massh,
                        cudaStream_t s) {
  if (m.n_free <= 0) return;  // every vertex pinned: no rows
  const bool dyn = m.h > 0.0;
  const int wpb = m.tune_gather_wpb > 0 ? m.tune_gather_wpb : 4;
  const int64_t blocks = (m.n_free + wpb - 1) / wpb;
  const size_t smem = (size_t)wpb * (m.max_rs + m.max_up + 1) * sizeof(int);
  set_smem_limit(reinterpret_cast<const void*>(k_row_gather<HT, kMixed>), smem);
  pdl_launch(k_row_gather<HT, kMixed>, (unsigned)blocks, 32 * wpb, smem, s,
      (const int4*)m.d_row_hdr.p, m.n_free, m.d_rs_ptr.p, m.d_rs_src.p, hten, massh, m.d_mass.p,
      m.d_mass_df.p, kMixed ? nullptr : m.f64.gcon.p, kMixed ? m.mx.gcon.p : nullptr, x,
      kMixed ? m.mx.x_hi.p : nullptr, kMixed ? m.mx.x_lo.p : nullptr, dyn ? xt : nullptr,
      kMixed ? m.mx.xt_hi.p : nullptr, kMixed ? m.mx.xt_lo.p : nullptr, m.n, dyn, m.max_rs, m.max_up, bsr,
      kMixed ? nullptr : m.f64.g.p, kMixed ? m.mx.g_hi.p : nullptr, kMixed ? m.mx.g_lo.p : nullptr);
}

void launch_rows_f64(Mesh& m, const double* x, const double* xt, double weight, cudaStream_t s) {
  (void)weight;
  launch_rows<double, false>(m, x, xt, m.f64.bsr.p, m.f64.hten.p, m.d_mass.p, s);
}

void launch_rows_mixed(Mesh& m, double weight, cudaStream_t s) {
  (void)weight;
  if (!rows_from_positions(m)) {
    launch_rows<float, true>(m, nullptr, nullptr, m.mx.bsr.p, m.mx.hten.p, m.d_mass32.p, s);
    return;
  }
  if (m.n_free <= 0) return;
  const bool dyn = m.h > 0.0;
  constexpr int kWpb = 4;
  const int64_t blocks = (m.n_free + kWpb - 1) / kWpb;
  const int maxval = m.max_valence <= 32 ? 32 : 64;
  const size_t smem = (size_t)kWpb * ((size_t)maxval * 37 * sizeof(float) +
                                      (size_t)(m.max_up + 1 + (m.max_rs + 1) / 2) * sizeof(int));
  auto kern = maxval == 32 ? k_row_build<32> : k_row_build<64>;
  set_smem_limit(reinterpret_cast<const void*>(kern), smem);
  pdl_launch(kern, (unsigned)blocks, 32 * kWpb, smem, s, (const int4*)m.d_row_hdr.p, m.n_free,
             (const int32_t*)m.d_rs_ptr.p, (const uint16_t*)m.d_rs_loc.p, (const int32_t*)m.d_vt_tet.p,
             (const uint8_t*)m.d_vt_corner.p, (const int4*)m.d_vt_ids.p, (const float4*)m.d_Bm32p.p,
             (const float*)m.d_volw32.p, (const float4*)m.d_matdf.p, (const float4*)m.mx.x_hi.p,
             (const float4*)m.mx.x_lo.p, (const float*)m.d_mass32.p, (const float2*)m.d_mass_df.p,
             (const float2*)m.mx.gcon.p, (const float4*)m.mx.xt_hi.p, (const float4*)m.mx.xt_lo.p, dyn, m.max_rs,
             m.max_up, m.mx.bsr.p, m.mx.g_hi.p, m.mx.g_lo.p);
}

void launch_energy(Mesh& m, const double* x, const double* xt, double* out, cudaStream_t s) {
  const double w = m.h > 0.0 ? m.h * m.h : 1.0;
  pdl_launch(m.model == CC_MODEL_FCR ? k_energy_tets<true> : k_energy_tets<false>, kRedBlocks, kBlock, 0, s,
             (const int4*)m.d_tets.p, (const double*)m.d_Bm.p, (const double*)m.d_vol.p, x, m.n, m.T,
             (const double2*)m.d_mat64.p, w, m.d_red.p);
  if (m.h > 0.0 && xt) {
    pdl_launch(k_energy_inertia, kRedBlocks, kBlock, 0, s, m.d_mass.p, x, xt, m.n, m.d_red.p + kRedBlocks);
    pdl_launch(k_reduce_final, 1, 1024, 0, s, m.d_red.p, (int64_t)(2 * kRedBlocks), out);
  } else {
    pdl_launch(k_reduce_final, 1, 1024, 0, s, m.d_red.p, (int64_t)kRedBlocks, out);
  }
}

void launch_energy_mesh(Mesh& m, const double* x, const double* xt, double* out, cudaStream_t s) {
  const double w = m.h > 0.0 ? m.h * m.h : 1.0;
  const unsigned B = (unsigned)(m.mesh_vptr.size() - 1);
  pdl_launch(m.model == CC_MODEL_FCR ? k_energy_mesh<true> : k_energy_mesh<false>, B, kBlock, 0, s,
             (const int64_t*)m.d_mesh_tptr.p, (const int64_t*)m.d_mesh_vptr.p, (const int4*)m.d_tets.p,
             (const double*)m.d_Bm.p, (const double*)m.d_vol.p, x, m.n, (const double2*)m.d_mat64.p, w,
             (const double*)m.d_mass.p, m.h > 0.0 ? xt : nullptr, out);
}

void launch_line_point_mesh(Mesh& m, const double* x0, const double* x1, const double* alpha, double* x,
                            cudaStream_t s) {
  pdl_launch(k_line_point_mesh, grid_for(3 * m.n), kBlock, 0, s, x0, x1, m.n, (const int32_t*)m.d_vert_mesh.p, alpha,
             x);
}

void launch_gnorm_f64(Mesh& m, double* grad_out, double* out, cudaStream_t s) {
  pdl_launch(k_gnorm<false>, kRedBlocks, kBlock, 0, s, m.d_free_rows.p, m.n_free, (const double*)m.f64.g.p,
             (const float*)nullptr, (const float*)nullptr, m.n, grad_out, m.d_red.p);
  pdl_launch(k_reduce_final, 1, 1024, 0, s, m.d_red.p, (int64_t)kRedBlocks, out);
}

void launch_gnorm_mixed(Mesh& m, double* grad_out, double* out, cudaStream_t s) {
  pdl_launch(k_gnorm<true>, kRedBlocks, kBlock, 0, s, m.d_free_rows.p, m.n_free, (const double*)nullptr,
             (const float*)m.mx.g_hi.p, (const float*)m.mx.g_lo.p, m.n, grad_out, m.d_red.p);
  pdl_launch(k_reduce_final, 1, 1024, 0, s, m.d_red.p, (int64_t)kRedBlocks, out);
}

void launch_gnorm_mesh(Mesh& m, bool mixed, cudaStream_t s) {
  const unsigned B = (unsigned)(m.mesh_vptr.size() - 1);
  if (mixed)
    pdl_launch(k_gnorm_mesh<true>, B, 256, 0, s, m.d_mesh_fptr.p, m.d_free_rows.p, (const double*)nullptr,
               (const float*)m.mx.g_hi.p, (const float*)m.mx.g_lo.p, m.d_mesh_gsq.p);
  else
    pdl_launch(k_gnorm_mesh<false>, B, 256, 0, s, m.d_mesh_fptr.p, m.d_free_rows.p, (const double*)m.f64.g.p,
               (const float*)nullptr, (const float*)nullptr, m.d_mesh_gsq.p);
}

void launch_split_df(const double* x, int64_t n, float4* hi, float4* lo, cudaStream_t s) {
  pdl_launch(k_split_df, grid_for(n), kBlock, 0, s, x, n, hi, lo);
}

void launch_inertial_target(const double* x, const double* v, int64_t n, double h, const double* grav, double* xt,
                            cudaStream_t s) {
  k_inertial_target<<<grid_for(n), kBlock, 0, s>>>(x, v, n, h, grav[0], grav[1], grav[2], xt);
}

void launch_line_point(const double* x0, const double* x1, int64_t n, double alpha, double* x, cudaStream_t s) {
  pdl_launch(k_line_point, grid_for(3 * n), kBlock, 0, s, x0, x1, n, alpha, x);
}

void launch_velocity(const double* x, const double* xold, int64_t n, double h, double* v, cudaStream_t s) {
  k_velocity<<<grid_for(3 * n), kBlock, 0, s>>>(x, xold, n, h, v);
}

}  // namespace ccg
