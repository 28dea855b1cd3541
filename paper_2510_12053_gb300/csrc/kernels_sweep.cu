// Fused subspace-coupling products and Schur-condensed local solve
// (Eq. 9-12), one warp per free vertex i of the current colour.
//
// For vertex i with support S (|S| = m) and basis blocks U[s] (3x3):
//   A  = sum_{l in row i, l in S} H_il U[l]                 (= H_iC U_i)
//   Y_j = sum_{l in row j, l in S} H_jl U[l],   j in S
//   Ht = sum_{j in S} U[j]^T Y_j                             (= U^T H_CC U)
//   b  = sum_{j in S} U[j]^T g_j                             (= U^T g_C)
// then, in float64 on lane 0:
//   S = A Ht^{-1} A^T,  gt = g_i - A Ht^{-1} b,  dx_i = -(H_ii - S)^{-1} gt
// and x_i += dx_i (the subspace part U dalpha is discarded, Sec. 3.1).
// The warp stages U_i in shared memory and indexes it through an open
// addressing hash (vertex id -> support slot), so any mesh works.
// Same-coloured vertices share no tet, and this kernel reads only g, H and U,
// so writing x in place is race-free for both schedules.
#include "cc_internal.cuh"
#include "dmath.cuh"

namespace ccg {

namespace {

constexpr double kPivotRel = 1e-12;

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

template <typename HT>
__host__ __device__ inline size_t warp_smem_bytes(int sup_max, int hash_size) {
  return align16((size_t)sup_max * 9 * sizeof(HT)) + (size_t)hash_size * 4 + align16((size_t)hash_size * 2);
}

__device__ __forceinline__ unsigned hash_slot(int id, int bits) {
  return ((unsigned)id * 2654435761u) >> (32 - bits);
}

__device__ __forceinline__ int hash_find(const int* keys, const short* vals, int id, int bits) {
  const unsigned mask = (1u << bits) - 1u;
  unsigned h = hash_slot(id, bits);
  while (true) {
    const int k = keys[h];
    if (k == id) return vals[h];
    if (k == -1) return -1;
    h = (h + 1) & mask;
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename HT, bool kMixed, int kUpd>
__global__ void k_local_solve(const int32_t* __restrict__ verts, int64_t count, const int32_t* __restrict__ sup_ptr,
                              const int32_t* __restrict__ sup_idx, const HT* __restrict__ U,
                              const int32_t* __restrict__ bsr_ptr, const int32_t* __restrict__ bsr_col,
                              const HT* __restrict__ bsr, const double* __restrict__ g64,
                              const float* __restrict__ g_hi, const float* __restrict__ g_lo, int64_t n,
                              int hash_bits, int sup_max, double* __restrict__ x, float4* __restrict__ x_hi,
                              float4* __restrict__ x_lo, unsigned long long* __restrict__ fallback,
                              unsigned long long* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int hs = 1 << hash_bits;
  unsigned char* base = smem + (size_t)warp * warp_smem_bytes<HT>(sup_max, hs);
  HT* Us = reinterpret_cast<HT*>(base);
  int* keys = reinterpret_cast<int*>(base + align16((size_t)sup_max * 9 * sizeof(HT)));
  short* vals = reinterpret_cast<short*>(keys + hs);

  const int64_t wid = (int64_t)blockIdx.x * wpb + warp;
  if (wid >= count) return;  // uniform per warp
  const int i = verts[wid];
  const int s0 = sup_ptr[i];
  const int m = sup_ptr[i + 1] - s0;

  if (kUpd != CC_UPDATE_CD) {
    for (int k = lane; k < hs; k += 32) keys[k] = -1;
    for (int k = lane; k < 9 * m; k += 32) Us[k] = U[(int64_t)s0 * 9 + k];
    __syncwarp();
    for (int s = lane; s < m; s += 32) {
      const int id = sup_idx[s0 + s];
      unsigned h = hash_slot(id, hash_bits);
      while (true) {
        const int prev = atomicCAS(&keys[h], -1, id);
        if (prev == -1) {
          vals[h] = (short)s;
          break;
        }
        h = (h + 1) & (unsigned)(hs - 1);
      }
    }
    __syncwarp();
  }

  HT Hii[9], A[9], Ht[9], b[3];
  mat3_zero(Hii);
  mat3_zero(A);
  mat3_zero(Ht);
  b[0] = b[1] = b[2] = HT(0);

  // row i: diagonal block and A = H_iC U
  const int r0 = bsr_ptr[i], r1 = bsr_ptr[i + 1];
  for (int p = r0 + lane; p < r1; p += 32) {
    const int l = bsr_col[p];
    const HT* Hb = bsr + (int64_t)p * 9;
    if (l == i) {
#pragma unroll
      for (int q = 0; q < 9; ++q) Hii[q] = Hb[q];
    } else if (kUpd == CC_UPDATE_CC) {
      const int t = hash_find(keys, vals, l, hash_bits);
      if (t >= 0) {
        HT Hl[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) Hl[q] = Hb[q];
        mat3_mul_acc(Hl, Us + 9 * t, A);
      }
    }
  }

  // Ht = U^T H_CC U and b = U^T g_C over the support rows
  if (kUpd != CC_UPDATE_CD) {
    for (int s = lane; s < m; s += 32) {
      const int j = sup_idx[s0 + s];
      HT Y[9];
      mat3_zero(Y);
      const int p1 = bsr_ptr[j + 1];
      for (int p = bsr_ptr[j]; p < p1; ++p) {
        const int t = hash_find(keys, vals, bsr_col[p], hash_bits);
        if (t >= 0) {
          HT Hl[9];
          const HT* Hb = bsr + (int64_t)p * 9;
#pragma unroll
          for (int q = 0; q < 9; ++q) Hl[q] = Hb[q];
          mat3_mul_acc(Hl, Us + 9 * t, Y);
        }
      }
      const HT* Uj = Us + 9 * s;
      mat3_tmul_acc(Uj, Y, Ht);
      HT gj[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) gj[a] = kMixed ? (HT)g_hi[3 * (int64_t)j + a] : (HT)g64[3 * (int64_t)j + a];
#pragma unroll
      for (int c = 0; c < 3; ++c) b[c] += Uj[c] * gj[0] + Uj[3 + c] * gj[1] + Uj[6 + c] * gj[2];
    }
  }

#pragma unroll
  for (int q = 0; q < 9; ++q) {
    Hii[q] = warp_sum(Hii[q]);
    A[q] = warp_sum(A[q]);
    Ht[q] = warp_sum(Ht[q]);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) b[c] = warp_sum(b[c]);

  if (lane != 0) return;

  double gi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    gi[a] = kMixed ? (double)g_hi[3 * (int64_t)i + a] + (double)g_lo[3 * (int64_t)i + a] : g64[3 * (int64_t)i + a];
  double H[9], L[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) H[q] = (double)Hii[q];

  double dx[3] = {-gi[0], -gi[1], -gi[2]};
  int fb = -1;
  bool done = false;
  if (kUpd != CC_UPDATE_CD) {
    if (m == 0) {
      fb = 0;
    } else {
      double Htd[9], Ad[9], bd[3] = {(double)b[0], (double)b[1], (double)b[2]};
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        Htd[q] = (double)Ht[q];
        Ad[q] = (double)A[q];
      }
      if (kUpd == CC_UPDATE_JGS2) {
        double M[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) M[q] = H[q] + Htd[q];
        if (chol3(M, L, kPivotRel)) {
          double r[3] = {-(gi[0] + bd[0]), -(gi[1] + bd[1]), -(gi[2] + bd[2])};
          chol3_solve(L, r);
          dx[0] = r[0]; dx[1] = r[1]; dx[2] = r[2];
          done = true;
        } else {
          fb = 1;
        }
      } else {
        double Lt[9];
        if (chol3(Htd, Lt, kPivotRel)) {
          // Z = Ht^{-1} A^T (columns = rows of A), y = Ht^{-1} b
          double Z[9];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            double col[3] = {Ad[3 * c], Ad[3 * c + 1], Ad[3 * c + 2]};
            chol3_solve(Lt, col);
            Z[c] = col[0]; Z[3 + c] = col[1]; Z[6 + c] = col[2];
          }
          chol3_solve(Lt, bd);
          double M[9], gt[3];
#pragma unroll
          for (int r = 0; r < 3; ++r) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
              M[3 * r + c] = H[3 * r + c] - (Ad[3 * r] * Z[c] + Ad[3 * r + 1] * Z[3 + c] + Ad[3 * r + 2] * Z[6 + c]);
            gt[r] = gi[r] - (Ad[3 * r] * bd[0] + Ad[3 * r + 1] * bd[1] + Ad[3 * r + 2] * bd[2]);
          }
          if (chol3(M, L, kPivotRel)) {
            double r[3] = {-gt[0], -gt[1], -gt[2]};
            chol3_solve(L, r);
            dx[0] = r[0]; dx[1] = r[1]; dx[2] = r[2];
            done = true;
          } else {
            fb = 2;
          }
        } else {
          fb = 1;
        }
      }
    }
  }
  if (!done) {
    // coordinate descent step: one Newton step on vertex i
    if (chol3(H, L, 0.0)) {
      double r[3] = {-gi[0], -gi[1], -gi[2]};
      chol3_solve(L, r);
      dx[0] = r[0]; dx[1] = r[1]; dx[2] = r[2];
    } else {
      dx[0] = dx[1] = dx[2] = __longlong_as_double(0x7ff8000000000000LL);
    }
  }
  if (fb >= 0) atomicAdd(&fallback[fb], 1ull);
  if (!(isfinite(dx[0]) && isfinite(dx[1]) && isfinite(dx[2]))) {
    atomicOr(err, 1ull);
    return;
  }
  double xn[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    xn[a] = x[a * n + i] + dx[a];
    x[a * n + i] = xn[a];
  }
  if (kMixed) {
    df a0 = df_from_double(xn[0]), a1 = df_from_double(xn[1]), a2 = df_from_double(xn[2]);
    x_hi[i] = make_float4(a0.hi, a1.hi, a2.hi, 0.f);
    x_lo[i] = make_float4(a0.lo, a1.lo, a2.lo, 0.f);
  }
}

template <typename HT, bool kMixed, int kUpd>
void launch_one(Mesh& m, const int32_t* verts, int64_t count, const HT* U, const HT* bsr, const double* g64,
                const float* g_hi, const float* g_lo, double* x, SweepCounters c, cudaStream_t s) {
  const int wpb = 4;
  const int hs = m.hash_size > 0 ? m.hash_size : 32;
  int bits = 0;
  while ((1 << bits) < hs) ++bits;
  const int supm = m.sup_max > 0 ? m.sup_max : 1;
  const size_t smem = (size_t)wpb * warp_smem_bytes<HT>(supm, hs);
  auto kern = k_local_solve<HT, kMixed, kUpd>;
  CCG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t blocks = (count + wpb - 1) / wpb;
  kern<<<(unsigned)blocks, wpb * 32, smem, s>>>(verts, count, m.d_sup_ptr.p, m.d_sup_idx.p, U, m.d_bsr_ptr.p,
                                                m.d_bsr_col.p, bsr, g64, g_hi, g_lo, m.n, bits, supm, x,
                                                kMixed ? m.mx.x_hi.p : nullptr, kMixed ? m.mx.x_lo.p : nullptr,
                                                c.fallback, c.error);
  CCG_CUDA(cudaGetLastError());
}

}  // namespace

void launch_local_solve_f64(Mesh& m, cc_update upd, const int32_t* verts, int64_t count, double* x,
                            SweepCounters c, cudaStream_t s) {
  if (count <= 0) return;
  switch (upd) {
    case CC_UPDATE_CC:
      launch_one<double, false, CC_UPDATE_CC>(m, verts, count, m.f64.U.p, m.f64.bsr.p, m.f64.g.p, nullptr, nullptr, x, c, s);
      break;
    case CC_UPDATE_CD:
      launch_one<double, false, CC_UPDATE_CD>(m, verts, count, m.f64.U.p, m.f64.bsr.p, m.f64.g.p, nullptr, nullptr, x, c, s);
      break;
    default:
      launch_one<double, false, CC_UPDATE_JGS2>(m, verts, count, m.f64.U.p, m.f64.bsr.p, m.f64.g.p, nullptr, nullptr, x, c, s);
  }
}

void launch_local_solve_mixed(Mesh& m, cc_update upd, const int32_t* verts, int64_t count, double* x,
                              SweepCounters c, cudaStream_t s) {
  if (count <= 0) return;
  switch (upd) {
    case CC_UPDATE_CC:
      launch_one<float, true, CC_UPDATE_CC>(m, verts, count, m.mx.U.p, m.mx.bsr.p, nullptr, m.mx.g_hi.p, m.mx.g_lo.p, x, c, s);
      break;
    case CC_UPDATE_CD:
      launch_one<float, true, CC_UPDATE_CD>(m, verts, count, m.mx.U.p, m.mx.bsr.p, nullptr, m.mx.g_hi.p, m.mx.g_lo.p, x, c, s);
      break;
    default:
      launch_one<float, true, CC_UPDATE_JGS2>(m, verts, count, m.mx.U.p, m.mx.bsr.p, nullptr, m.mx.g_hi.p, m.mx.g_lo.p, x, c, s);
  }
}

}  // namespace ccg
