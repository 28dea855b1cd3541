// Learned perturbation bases on the GPU (no counterpart in the paper, whose
// bases come from the patch solve of Eq. 5, Sec. 3.1):
//
//  * the network: float32 master parameters, BF16 weight copies in both
//    orientations, forward and backward passes made of tcgen05 GEMMs with
//    fused bias / GELU / GELU-gradient epilogues, split-K weight gradients
//    reduced in a fixed order, Adam;
//  * per-vertex inputs from the rest geometry of the 2-ring (64 stencil
//    slots of the Kuhn lattice) and the material, targets from computed
//    bases, assembly of predicted bases;
//  * the Eq. 5 residual rho_i = ||H_PP U_i + H_Pi|| / ||H_Pi|| of every basis
//    at the rest Hessian, and the per-vertex fallback to the patch solve.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "cc_internal.cuh"
#include "mlp.cuh"

namespace ccg {

using bf16 = __nv_bfloat16;

namespace {

int round8(int64_t v) { return (int)((v + 7) / 8 * 8); }

// ---------------------------------------------------------------------------
// Stencil of the Kuhn lattice (consistent (1,1,1) diagonals).  Its 1-ring
// offsets are the seven nonzero 0/1 vectors and their negatives; the 2-ring
// adds every sum of two 1-ring offsets that is neither 0 nor a 1-ring offset.
// Slots: the 14 1-ring offsets in lexicographic order, then the others in
// lexicographic order (64 in all).
// ---------------------------------------------------------------------------
struct SlotTable {
  int8_t s[128];  // index (dx + 2) * 25 + (dy + 2) * 5 + (dz + 2); -1 off the stencil
};

SlotTable make_slot_table() {
  using V = std::array<int, 3>;
  std::vector<V> one;
  for (int b = 1; b < 8; ++b) {
    const V a = {b & 1, (b >> 1) & 1, (b >> 2) & 1};
    one.push_back(a);
    one.push_back({-a[0], -a[1], -a[2]});
  }
  std::sort(one.begin(), one.end());
  std::vector<V> two;
  for (const V& u : one)
    for (const V& w : one) {
      const V c = {u[0] + w[0], u[1] + w[1], u[2] + w[2]};
      if (c == V{0, 0, 0} || std::binary_search(one.begin(), one.end(), c)) continue;
      two.push_back(c);
    }
  std::sort(two.begin(), two.end());
  two.erase(std::unique(two.begin(), two.end()), two.end());
  CCG_CHECK(one.size() == 14 && two.size() == 50, CC_ERR_STATE, "stencil construction");
  SlotTable t;
  std::memset(t.s, -1, sizeof(t.s));
  int slot = 0;
  for (const auto* list : {&one, &two})
    for (const V& o : *list) t.s[(o[0] + 2) * 25 + (o[1] + 2) * 5 + (o[2] + 2)] = (int8_t)slot++;
  return t;
}

// Cell size estimate of free vertex i: mean over the 1-ring of the largest
// coordinate difference (ascending neighbour order).  0 when i has none.
__device__ double lattice_spacing(int i, int64_t n, const double* __restrict__ X,
                                  const int32_t* __restrict__ nbr_ptr, const int32_t* __restrict__ nbr_idx) {
  const int p0 = nbr_ptr[i], p1 = nbr_ptr[i + 1];
  if (p1 == p0) return 0.0;
  const double xi = X[i], yi = X[n + i], zi = X[2 * n + i];
  double acc = 0.0;
  for (int p = p0; p < p1; ++p) {
    const int j = nbr_idx[p];
    acc += fmax(fabs(X[j] - xi), fmax(fabs(X[n + j] - yi), fabs(X[2 * n + j] - zi)));
  }
  return acc / (double)(p1 - p0);
}

// Slot of j in the stencil of i (and the deviation q - o), or -1.
__device__ int stencil_slot(const SlotTable& tab, int i, int j, int64_t n, const double* __restrict__ X, double ell,
                            double dev[3]) {
  int o[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double q = (X[a * n + j] - X[a * n + i]) / ell;
    const double f = floor(q + 0.5);
    o[a] = (int)f;
    dev[a] = q - f;
  }
  if (o[0] < -2 || o[0] > 2 || o[1] < -2 || o[1] > 2 || o[2] < -2 || o[2] > 2) return -1;
  return tab.s[(o[0] + 2) * 25 + (o[1] + 2) * 5 + (o[2] + 2)];
}

__device__ __forceinline__ bf16 to_bf16(double v) { return __float2bfloat16_rn(__double2float_rn(v)); }

// One thread per free row: the 258 input channels (and zero padding up to ld).
__global__ void k_features(int nrows, const int32_t* __restrict__ rows, int64_t n, const double* __restrict__ X,
                           const int32_t* __restrict__ nbr_ptr, const int32_t* __restrict__ nbr_idx,
                           const uint8_t* __restrict__ pinned, const double2* __restrict__ vmat, SlotTable tab,
                           bf16* __restrict__ out, int64_t ld, int* __restrict__ err) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const int i = rows[r];
  bf16* row = out + (int64_t)r * ld;
  const double ell = lattice_spacing(i, n, X, nbr_ptr, nbr_idx);
  int slotv[64];
#pragma unroll
  for (int s = 0; s < 64; ++s) slotv[s] = -1;
  bool bad = !(ell > 0.0);
  if (!bad) {
    const int p0 = nbr_ptr[i], p1 = nbr_ptr[i + 1];
    for (int p = p0; p < p1 && !bad; ++p) {
      // the 1-ring neighbour a itself (q = start - 1), then a's own 1-ring
      const int a = nbr_idx[p];
      for (int q = nbr_ptr[a] - 1; q < nbr_ptr[a + 1]; ++q) {
        const int j = q < nbr_ptr[a] ? a : nbr_idx[q];
        if (j == i) continue;
        double dev[3];
        const int s = stencil_slot(tab, i, j, n, X, ell, dev);
        if (s < 0) {
          bad = true;
          break;
        }
        if (slotv[s] < 0) slotv[s] = j;
        else if (slotv[s] != j) {
          bad = true;
          break;
        }
      }
    }
  }
  if (bad) {
    atomicExch(err, 1);
    for (int64_t c = 0; c < ld; ++c) row[c] = __float2bfloat16_rn(0.0f);
    return;
  }
  for (int s = 0; s < 64; ++s) {
    const int j = slotv[s];
    if (j < 0) {
#pragma unroll
      for (int c = 0; c < 4; ++c) row[4 * s + c] = __float2bfloat16_rn(0.0f);
      continue;
    }
    double dev[3];
    stencil_slot(tab, i, j, n, X, ell, dev);
#pragma unroll
    for (int c = 0; c < 3; ++c) row[4 * s + c] = to_bf16(8.0 * dev[c]);
    row[4 * s + 3] = __float2bfloat16_rn(pinned[j] ? -1.0f : 1.0f);
  }
  const double2 em = vmat[i];
  row[256] = to_bf16((log10(em.x) - 5.5) / 1.5);
  row[257] = to_bf16(10.0 * (em.y - 0.4));
  for (int64_t c = 258; c < ld; ++c) row[c] = __float2bfloat16_rn(0.0f);
}

// One thread per free row: the slot of every support entry.
__global__ void k_support_slots(int nrows, const int32_t* __restrict__ rows, int64_t n, const double* __restrict__ X,
                                const int32_t* __restrict__ nbr_ptr, const int32_t* __restrict__ nbr_idx,
                                const int32_t* __restrict__ sup_ptr, const int32_t* __restrict__ sup_idx,
                                SlotTable tab, int8_t* __restrict__ sup_slot, int* __restrict__ err) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const int i = rows[r];
  const double ell = lattice_spacing(i, n, X, nbr_ptr, nbr_idx);
  for (int p = sup_ptr[i]; p < sup_ptr[i + 1]; ++p) {
    double dev[3];
    const int s = ell > 0.0 ? stencil_slot(tab, i, sup_idx[p], n, X, ell, dev) : -1;
    if (s < 0) atomicExch(err, 1);
    sup_slot[p] = (int8_t)s;
  }
}

// One warp per free row: target row from the float64 bases (rows pre-zeroed).
__global__ void k_targets(int nrows, const int32_t* __restrict__ rows, const int32_t* __restrict__ sup_ptr,
                          const int8_t* __restrict__ sup_slot, const double* __restrict__ U, float* __restrict__ T,
                          int64_t ldt) {
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= nrows) return;
  const int i = rows[r];
  const int p0 = sup_ptr[i], m = sup_ptr[i + 1] - p0;
  for (int k = lane; k < 9 * m; k += 32) {
    const int a = k / 9, q = k % 9;
    const int s = sup_slot[p0 + a];
    if (s >= 0) T[(int64_t)r * ldt + 9 * s + q] = (float)U[(int64_t)(p0 + a) * 9 + q];
  }
}

// One warp per free row: bases from the predictions.
__global__ void k_assemble(int nrows, const int32_t* __restrict__ rows, const int32_t* __restrict__ sup_ptr,
                           const int8_t* __restrict__ sup_slot, const float* __restrict__ Y, int64_t ldy,
                           double* __restrict__ U64, float* __restrict__ U32) {
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= nrows) return;
  const int i = rows[r];
  const int p0 = sup_ptr[i], m = sup_ptr[i + 1] - p0;
  for (int k = lane; k < 9 * m; k += 32) {
    const int a = k / 9, q = k % 9;
    const int s = sup_slot[p0 + a];
    const float v = s >= 0 ? Y[(int64_t)r * ldy + 9 * s + q] : 0.0f;
    U64[(int64_t)(p0 + a) * 9 + q] = (double)v;
    U32[(int64_t)(p0 + a) * 9 + q] = v;
  }
}

__device__ int find_sorted_i32(const int32_t* a, int m, int key) {
  int lo = 0, hi = m - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int v = a[mid];
    if (v == key) return mid;
    if (v < key) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

// acc (3x3) += Hb (3x3 in a 3x4 padded block, transposed when tr) * Ub (3x3)
__device__ __forceinline__ void acc_hu(double* acc, const double* Hb, bool tr, const double* Ub) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double s = acc[3 * r + d];
#pragma unroll
      for (int c = 0; c < 3; ++c) s = fma(tr ? Hb[4 * c + r] : Hb[4 * r + c], Ub[3 * c + d], s);
      acc[3 * r + d] = s;
    }
}

// One warp per free row i: rho_i = ||H_PP U_i + H_Pi||_F / ||H_Pi||_F from the
// upper 3x3 blocks of the float64 Hessian rows.  Lane a takes support vertex
// j = S[a]: blocks (j, l), l >= j from row j, blocks (l, j), l < j from row l
// (transposed).  Fixed summation order; fixed shuffle reduction.
__global__ void k_basis_residual(int nrows, const int32_t* __restrict__ rows, const int32_t* __restrict__ sup_ptr,
                                 const int32_t* __restrict__ sup_idx, const int32_t* __restrict__ up_ptr,
                                 const int32_t* __restrict__ up_col, const int32_t* __restrict__ nbr_ptr,
                                 const int32_t* __restrict__ nbr_idx, const double* __restrict__ bsr,
                                 const double* __restrict__ U, double* __restrict__ rho) {
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= nrows) return;
  const int i = rows[r];
  const int s0 = sup_ptr[i], m = sup_ptr[i + 1] - s0;
  const int32_t* S = sup_idx + s0;
  double res2 = 0.0, base2 = 0.0;
  for (int a = lane; a < m; a += 32) {
    const int j = S[a];
    double acc[9], hji[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = hji[k] = 0.0;
    for (int p = up_ptr[j]; p < up_ptr[j + 1]; ++p) {
      const int l = up_col[p];
      const double* Hb = bsr + (int64_t)p * 12;
      if (l == i) {
#pragma unroll
        for (int rr = 0; rr < 3; ++rr)
#pragma unroll
          for (int c = 0; c < 3; ++c) hji[3 * rr + c] = Hb[4 * rr + c];
      } else {
        const int t = (l == j) ? a : find_sorted_i32(S, m, l);
        if (t >= 0) acc_hu(acc, Hb, false, U + (int64_t)(s0 + t) * 9);
      }
    }
    // neighbours l < j of j that lie in the patch (or are i), ascending:
    // block (l, j), stored in row l, is H_jl^T
    for (int e = nbr_ptr[j]; e < nbr_ptr[j + 1]; ++e) {
      const int l = nbr_idx[e];
      if (l >= j) break;
      const int b = l == i ? -1 : find_sorted_i32(S, m, l);
      if (l != i && b < 0) continue;
      const int q0 = up_ptr[l] + 1, q1 = up_ptr[l + 1];  // diagonal first, then ascending
      const int pos = find_sorted_i32(up_col + q0, q1 - q0, j);
      if (pos < 0) continue;
      const double* Hb = bsr + (int64_t)(q0 + pos) * 12;
      if (b < 0) {
#pragma unroll
        for (int rr = 0; rr < 3; ++rr)
#pragma unroll
          for (int c = 0; c < 3; ++c) hji[3 * rr + c] = Hb[4 * c + rr];
      } else {
        acc_hu(acc, Hb, true, U + (int64_t)(s0 + b) * 9);
      }
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double v = acc[k] + hji[k];
      res2 = fma(v, v, res2);
      base2 = fma(hji[k], hji[k], base2);
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    res2 += __shfl_xor_sync(0xffffffffu, res2, off);
    base2 += __shfl_xor_sync(0xffffffffu, base2, off);
  }
  if (lane == 0) rho[r] = base2 > 0.0 ? sqrt(res2 / base2) : 0.0;
}

// ---------------------------------------------------------------------------
// Network kernels
// ---------------------------------------------------------------------------
// dst row b = src row idx[b] (BF16 rows of `cols` elements, 16-byte chunks).
// Training minibatch rows: row b of step *step is idx[*step * B + b] (the
// step counter lives on the device, so one captured step replays for all).
__global__ void k_gather_rows_bf16(const bf16* __restrict__ src, int64_t lds, const int32_t* __restrict__ idx,
                                   const int* __restrict__ step, int B, int chunks, bf16* __restrict__ dst,
                                   int64_t ldd) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= (int64_t)B * chunks) return;
  const int b = (int)(k / chunks), c = (int)(k % chunks);
  const int32_t row = idx[(int64_t)*step * B + b];
  reinterpret_cast<uint4*>(dst + (int64_t)b * ldd)[c] = reinterpret_cast<const uint4*>(src + (int64_t)row * lds)[c];
}

// vec = 4: cols, lds and ldd multiples of 4 and both bases 16-byte aligned
// (float4 copies); else vec = 1.
template <int vec>
__global__ void k_gather_rows_f32(const float* __restrict__ src, int64_t lds, const int32_t* __restrict__ idx,
                                  const int* __restrict__ step, int B, int cols, float* __restrict__ dst,
                                  int64_t ldd) {
  const int per = cols / vec;
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= (int64_t)B * per) return;
  const int b = (int)(k / per), c = (int)(k % per) * vec;
  const float* s = src + (int64_t)idx[(int64_t)*step * B + b] * lds + c;
  float* d = dst + (int64_t)b * ldd + c;
  if constexpr (vec == 4) *reinterpret_cast<float4*>(d) = *reinterpret_cast<const float4*>(s);
  else *d = *s;
}

// end of a training step: the next step's number and beta^t
__global__ void k_step_advance(int* __restrict__ step, double* __restrict__ pw, double b1, double b2) {
  ++*step;
  pw[0] *= b1;
  pw[1] *= b2;
}

// dst [cols x ldd] = src [rows x cols]^T (BF16), 32 x 32 tiles through shared memory.
__global__ void k_transpose_bf16(const bf16* __restrict__ src, int64_t lds, int rows, int cols, bf16* __restrict__ dst,
                                 int64_t ldd) {
  __shared__ bf16 tile[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = r0 + k, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[k][threadIdx.x] = src[(int64_t)r * lds + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = c0 + k, r = r0 + threadIdx.x;
    if (r < rows && c < cols) dst[(int64_t)c * ldd + r] = tile[threadIdx.x][k];
  }
}

// Output gradient of the mean squared error: dY = 2 (Y - T) / (B d_out) in
// BF16, row-major and transposed, and per-block float64 partial sums of
// (Y - T)^2.  32 x 32 tiles; block partials at part[blockIdx.y * gridDim.x + blockIdx.x].
__global__ void k_loss_dy(const float* __restrict__ Y, int64_t ldy, const float* __restrict__ T, int64_t ldt, int B,
                          int D, float scale, bf16* __restrict__ dy, int64_t lddy, bf16* __restrict__ dyt,
                          int64_t lddt, double* __restrict__ part) {
  __shared__ bf16 tile[32][33];
  __shared__ double red[8];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  float acc = 0.0f;  // a thread's four squares in float32; the block's warps' sums in float64
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = r0 + k, c = c0 + threadIdx.x;
    if (r < B && c < D) {
      const float d = Y[(int64_t)r * ldy + c] - T[(int64_t)r * ldt + c];
      acc = fmaf(d, d, acc);
      const bf16 g = __float2bfloat16_rn(d * scale);
      dy[(int64_t)r * lddy + c] = g;
      tile[k][threadIdx.x] = g;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (threadIdx.x == 0) red[threadIdx.y] = (double)acc;
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = c0 + k, r = r0 + threadIdx.x;
    if (r < B && c < D) dyt[(int64_t)c * lddt + r] = tile[threadIdx.x][k];
  }
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    double sum = 0.0;
    for (int w = 0; w < (int)blockDim.y; ++w) sum += red[w];
    part[blockIdx.y * gridDim.x + blockIdx.x] = sum;
  }
}

// out[0] = scale * sum of part[0..count) in a fixed order (one block).
// out[step ? *step : 0] = scale * sum of part[0 .. count)
__global__ void k_sum_partials(const double* __restrict__ part, int count, double scale, double* __restrict__ out,
                               const int* __restrict__ step) {
  __shared__ double red[256];
  double a = 0.0;
  for (int k = threadIdx.x; k < count; k += 256) a += part[k];
  red[threadIdx.x] = a;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[step ? *step : 0] = red[0] * scale;
}

// out[row] = sum over the first `cols` entries of a BF16 row (one warp per row).
// One block of 256 threads per row (blockIdx.x): thread t sums columns
// t, t + 256, ... (pairs of columns when the row start and length allow),
// then warps and the block reduce in a fixed order.
__global__ void k_rowsum_bf16(const bf16* __restrict__ src, int64_t lds, int rows, int cols, float* __restrict__ out) {
  __shared__ float wsum[8];
  const int r = blockIdx.x;
  if (r >= rows) return;
  const bf16* row = src + (int64_t)r * lds;
  float a = 0.0f;
  if ((lds & 1) == 0 && (cols & 1) == 0 && (reinterpret_cast<uintptr_t>(src) & 3) == 0) {
    const __nv_bfloat162* row2 = reinterpret_cast<const __nv_bfloat162*>(row);
    for (int c = threadIdx.x; c < cols / 2; c += 256) {
      const float2 f = __bfloat1622float2(row2[c]);
      a += f.x + f.y;
    }
  } else {
    for (int c = threadIdx.x; c < cols; c += 256) a += __bfloat162float(row[c]);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < 8; ++w) t += wsum[w];
    out[r] = t;
  }
}

// out[k] = sum_s P[s * stride + k], s ascending.
__global__ void k_sum_slices(const float* __restrict__ P, int S, int64_t stride, int64_t count, float* __restrict__ out,
                             int64_t ldo, int cols, int64_t ldp) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= count) return;
  const int64_t r = k / cols, c = k % cols;
  float a = 0.0f;
  for (int s = 0; s < S; ++s) a += P[s * stride + r * ldp + c];
  out[r * ldo + c] = a;
}

// Adam (Kingma and Ba 2015, Algorithm 1) on the float32 master parameters.
// Adam with the bias corrections bc1, bc2, or 1 - pw[0], 1 - pw[1] when pw
// (this step's beta1^t, beta2^t, kept on the device) is given.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t count, float lr, float b1, float b2, float eps, float bc1, float bc2,
                       const double* __restrict__ pw) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= count) return;
  if (pw) {
    bc1 = (float)(1.0 - pw[0]);
    bc2 = (float)(1.0 - pw[1]);
  }
  const float gk = g[k];
  const float mk = b1 * m[k] + (1.0f - b1) * gk;
  const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  const float mh = mk / bc1, vh = vk / bc2;
  p[k] -= lr * mh / (sqrtf(vh) + eps);
}

// BF16 copies of one weight matrix W [N x K]: W16 [N x ldk], W16^T [K x ldn].
__global__ void k_refresh_bf16(const float* __restrict__ W, int N, int K, bf16* __restrict__ w16, int64_t ldk,
                               bf16* __restrict__ wt16, int64_t ldn) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= (int64_t)N * K) return;
  const int n = (int)(k / K), c = (int)(k % K);
  const bf16 b = __float2bfloat16_rn(W[k]);
  w16[(int64_t)n * ldk + c] = b;
  wt16[(int64_t)c * ldn + n] = b;
}

unsigned blocks_for(int64_t count, int threads) { return (unsigned)((count + threads - 1) / threads); }

}  // namespace

// ---------------------------------------------------------------------------
// The network
// ---------------------------------------------------------------------------
struct MlpNet {
  std::vector<int> dims;           // d_in, hidden..., d_out
  int L = 0;                       // layers (hidden + output)
  std::vector<int64_t> off_w, off_b;
  int64_t nparams = 0;
  std::vector<int> ldk, ldn;       // leading dims of W16 [N x ldk] and W16^T [K x ldn]
  int max_batch = 0, ldB = 0;
  cudaStream_t stream = nullptr;
  DBuf<float> params, grad, adam_m, adam_v;
  std::vector<DBuf<bf16>> w16, wt16;
  std::vector<DBuf<float>> z32;    // [B x N_l] pre-activations of hidden layers
  std::vector<DBuf<bf16>> h16, ht16;
  DBuf<float> y32;
  DBuf<bf16> dy16, dyt16, dz16[2], dzt16[2];
  DBuf<float> partial;
  DBuf<bf16> xb, xbt;
  DBuf<float> tb;
  DBuf<double> loss_part, loss_hist;
  DBuf<int> step_dev;  // training step within a cc_mlp_train call
  DBuf<double> adam_pw;     // that step's beta1^t, beta2^t
  double adam_pw_host[2] = {0.0, 0.0};
  DBuf<int> err;
  int64_t adam_t = 0;
  DBuf<bf16> inf_h[2];
  int64_t inf_rows = 0;
  int fused_inference = 1;  // 0: one GEMM per layer; 1, 2: one kernel for every layer (2: SM-pair MMAs)

  int d_in() const { return dims.front(); }
  int d_out() const { return dims.back(); }

  void check_err() {
    int h = 0;
    CCG_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, stream));
    CCG_CUDA(cudaStreamSynchronize(stream));
    CCG_CHECK(h == 0, CC_ERR_TIMEOUT, "a bounded wait in a GEMM kernel expired");
  }

  void refresh_bf16() {
    for (int l = 0; l < L; ++l) {
      const int N = dims[l + 1], K = dims[l];
      k_refresh_bf16<<<blocks_for((int64_t)N * K, 256), 256, 0, stream>>>(params.p + off_w[l], N, K, w16[l].p, ldk[l],
                                                                          wt16[l].p, ldn[l]);
      CCG_CUDA(cudaGetLastError());
    }
  }

  // Forward over a training batch held in xb (B rows, leading dim ldx):
  // keeps pre-activations and activations (both orientations) for backward.
  void forward_train(const bf16* X, int64_t ldx, int B) {
    for (int l = 0; l < L; ++l) {
      const int N = dims[l + 1], K = dims[l];
      const bf16* A = l == 0 ? X : h16[l - 1].p;
      const int64_t lda = l == 0 ? ldx : dims[l];
      GemmEpilogue ep;
      ep.bias = params.p + off_b[l];
      if (l < L - 1) {
        ep.z32 = z32[l].p;
        ep.ldz = N;
        ep.h16 = h16[l].p;
        ep.ldh = N;
        ep.ht16 = ht16[l].p;
        ep.ldt = ldB;
        gemm_tn(A, lda, w16[l].p, ldk[l], B, N, K, kEpiBiasGelu, ep, err.p, stream,
                gemm_pick_shape(B, N, K, false));
      } else {
        ep.c32 = y32.p;
        ep.ldc = N;
        gemm_tn(A, lda, w16[l].p, ldk[l], B, N, K, kEpiBiasF32, ep, err.p, stream, gemm_pick_shape(B, N, K, false));
      }
    }
  }

  // Loss into loss_dev[step ? *step : 0], gradient into `grad` (all
  // parameters).  xbt holds X^T.
  void backward(const float* T, int64_t ldt, int B, double* loss_dev, const int* step = nullptr) {
    const int D = d_out();
    {
      const dim3 grid((unsigned)((D + 31) / 32), (unsigned)((B + 31) / 32));
      k_loss_dy<<<grid, dim3(32, 8), 0, stream>>>(y32.p, D, T, ldt, B, D, 2.0f / ((float)B * (float)D), dy16.p, D,
                                                  dyt16.p, ldB, loss_part.p);
      CCG_CUDA(cudaGetLastError());
      k_sum_partials<<<1, 256, 0, stream>>>(loss_part.p, (int)(grid.x * grid.y), 1.0 / ((double)B * D), loss_dev,
                                            step);
      CCG_CUDA(cudaGetLastError());
    }
    const bf16* dz = dy16.p;
    const bf16* dzt = dyt16.p;
    int cur = 0;
    for (int l = L - 1; l >= 0; --l) {
      const int N = dims[l + 1], K = dims[l];
      // weight gradient dW_l = dZ^T H_{l-1}: [N x K], contraction over the batch
      const bf16* Ht = l == 0 ? xbt.p : ht16[l - 1].p;
      const GemmShape sh = gemm_pick_shape(N, K, B, true);
      GemmEpilogue ep;
      ep.c32 = partial.p;
      ep.ldc = K;
      ep.split_stride = (int64_t)N * K;
      CCG_CHECK((int64_t)sh.splits * N * K <= (int64_t)partial.count, CC_ERR_STATE, "split-K workspace too small");
      gemm_tn(dzt, ldB, Ht, ldB, N, K, B, kEpiF32, ep, err.p, stream, sh);
      const int kt = (B + 63) / 64, per = (kt + sh.splits - 1) / sh.splits, S = (kt + per - 1) / per;
      k_sum_slices<<<blocks_for((int64_t)N * K, 256), 256, 0, stream>>>(partial.p, S, (int64_t)N * K, (int64_t)N * K,
                                                                        grad.p + off_w[l], K, K, K);
      CCG_CUDA(cudaGetLastError());
      // bias gradient: row sums of dZ^T
      k_rowsum_bf16<<<(unsigned)N, 256, 0, stream>>>(dzt, ldB, N, B, grad.p + off_b[l]);
      CCG_CUDA(cudaGetLastError());
      if (l == 0) break;
      // input gradient dH_{l-1} = dZ W_l, times gelu'(Z_{l-1}) in the epilogue
      GemmEpilogue eg;
      eg.z32 = z32[l - 1].p;
      eg.ldz = K;
      eg.h16 = dz16[cur].p;
      eg.ldh = K;
      eg.ht16 = dzt16[cur].p;
      eg.ldt = ldB;
      gemm_tn(dz, N, wt16[l].p, ldn[l], B, K, N, kEpiGeluGrad, eg, err.p, stream, gemm_pick_shape(B, K, N, false));
      dz = dz16[cur].p;
      dzt = dzt16[cur].p;
      cur ^= 1;
    }
  }

  void adam(const float* g, const cc_adam& o) {
    ++adam_t;
    const double bc1 = 1.0 - std::pow((double)o.beta1, (double)adam_t);
    const double bc2 = 1.0 - std::pow((double)o.beta2, (double)adam_t);
    k_adam<<<blocks_for(nparams, 256), 256, 0, stream>>>(params.p, g, adam_m.p, adam_v.p, nparams, o.lr, o.beta1,
                                                         o.beta2, o.eps, (float)bc1, (float)bc2, nullptr);
    CCG_CUDA(cudaGetLastError());
    refresh_bf16();
  }

  // Adam with this step's beta^t from the device (the training loop)
  void adam_dev(const float* g, const cc_adam& o) {
    k_adam<<<blocks_for(nparams, 256), 256, 0, stream>>>(params.p, g, adam_m.p, adam_v.p, nparams, o.lr, o.beta1,
                                                         o.beta2, o.eps, 1.0f, 1.0f, adam_pw.p);
    CCG_CUDA(cudaGetLastError());
    refresh_bf16();
  }

  void transpose_input(const bf16* X, int64_t ldx, int B) {
    const dim3 grid((unsigned)((d_in() + 31) / 32), (unsigned)((B + 31) / 32));
    k_transpose_bf16<<<grid, dim3(32, 8), 0, stream>>>(X, ldx, B, d_in(), xbt.p, ldB);
    CCG_CUDA(cudaGetLastError());
  }

  // Inference over any number of rows: Y = net(X).
  void forward_rows(const bf16* X, int64_t ldx, int64_t rows, float* Y, int64_t ldy) {
    if (fused_inference && mlp_fused_supported(dims)) {
      std::vector<const bf16*> w(L);
      std::vector<const float*> b(L);
      for (int l = 0; l < L; ++l) {
        w[l] = w16[l].p;
        b[l] = params.p + off_b[l];
      }
      mlp_forward_fused(X, ldx, (int)rows, dims, w, ldk, b, Y, ldy, err.p, stream, fused_inference == 2);
      return;
    }
    int hmax = 8;
    for (int l = 1; l < L; ++l) hmax = std::max(hmax, dims[l]);
    if (rows > inf_rows) {
      inf_h[0].alloc((size_t)rows * hmax);
      inf_h[1].alloc((size_t)rows * hmax);
      inf_rows = rows;
    }
    for (int l = 0; l < L; ++l) {
      const int N = dims[l + 1], K = dims[l];
      const bf16* A = l == 0 ? X : inf_h[(l - 1) & 1].p;
      const int64_t lda = l == 0 ? ldx : dims[l];
      GemmEpilogue ep;
      ep.bias = params.p + off_b[l];
      if (l < L - 1) {
        ep.h16 = inf_h[l & 1].p;
        ep.ldh = N;
        gemm_tn(A, lda, w16[l].p, ldk[l], (int)rows, N, K, kEpiBiasGelu, ep, err.p, stream,
                gemm_pick_shape((int)rows, N, K, false));
      } else {
        ep.c32 = Y;
        ep.ldc = ldy;
        gemm_tn(A, lda, w16[l].p, ldk[l], (int)rows, N, K, kEpiBiasF32, ep, err.p, stream,
                gemm_pick_shape((int)rows, N, K, false));
      }
    }
  }
};

// Eq. 5 residual rho_i = ||H_PP U_i + H_Pi|| / ||H_Pi|| (float64 bases and
// block rows) of a device list of free vertices, into rho[count].
void basis_residuals(Mesh& m, const int32_t* d_rows, int64_t count, double* rho, cudaStream_t s) {
  if (count <= 0) return;
  k_basis_residual<<<blocks_for(count * 32, 256), 256, 0, s>>>((int)count, d_rows, m.d_sup_ptr.p, m.d_sup_idx.p,
                                                              m.d_up_ptr.p, m.d_up_col.p, m.d_nbr_ptr.p,
                                                              m.d_nbr_idx.p, m.f64.bsr.p, m.f64.U.p, rho);
  CCG_CUDA(cudaGetLastError());
}

}  // namespace ccg

using namespace ccg;

struct cc_mlp : public ccg::MlpNet {};
struct cc_mesh : public ccg::Mesh {};

namespace {

void require_bf16_operand(const void* p, int64_t ld, int64_t cols, const char* what) {
  CCG_CHECK(p != nullptr, CC_ERR_INVALID_ARG, std::string(what) + " is NULL");
  CCG_CHECK((reinterpret_cast<uintptr_t>(p) & 15) == 0, CC_ERR_INVALID_ARG,
            std::string(what) + " must be 16-byte aligned");
  CCG_CHECK(ld % 8 == 0 && ld >= cols, CC_ERR_INVALID_ARG,
            std::string(what) + ": leading dimension must be a multiple of 8 and cover the row");
}

double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// Rest positions (SoA) and per-vertex (E, nu) of the vertex's first tet.
void upload_rest_inputs(Mesh& m, DBuf<double>& Xs, DBuf<double2>& vmat) {
  const int64_t n = m.n;
  std::vector<double> soa(3 * n);
  for (int64_t j = 0; j < n; ++j)
    for (int a = 0; a < 3; ++a) soa[a * n + j] = m.X[3 * j + a];
  Xs.upload(soa, m.stream);
  std::vector<double2> vm(n, make_double2(1.0, 0.0));
  for (int64_t v = 0; v < n; ++v)
    if (m.vt_ptr[v + 1] > m.vt_ptr[v]) {
      const int32_t t = m.vt_tet[m.vt_ptr[v]];
      vm[v] = make_double2(m.tet_E[t], m.tet_nu[t]);
    }
  vmat.upload(vm, m.stream);
}

void read_err(DBuf<int>& err, cudaStream_t s, const char* msg) {
  int h = 0;
  CCG_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  CCG_CUDA(cudaStreamSynchronize(s));
  CCG_CHECK(h == 0, CC_ERR_INVALID_ARG, msg);
}

}  // namespace

extern "C" {

cc_status cc_gemm_bf16_tn(const void* A, int64_t lda, const void* B, int64_t ldb, int32_t M, int32_t N, int32_t K,
                          float* C, int64_t ldc, int32_t n_tile, int32_t k_splits, int32_t flags, void* stream) {
  CC_API_BODY("cc_gemm_bf16_tn", {
    CCG_CHECK(A && B && C && ldc >= N, CC_ERR_INVALID_ARG, "bad GEMM arguments");
    CCG_CHECK(k_splits >= 0 && n_tile >= 0, CC_ERR_INVALID_ARG, "bad GEMM launch shape");
    cudaStream_t s = (cudaStream_t)stream;
    DBuf<int> err;
    err.alloc(1);
    CCG_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    GemmShape sh = gemm_pick_shape(M, N, K, false);
    if (n_tile) sh.bn = n_tile;
    sh.splits = std::max(1, (int)k_splits);
    sh.persistent = (flags & CC_GEMM_ONE_TILE_PER_CTA) == 0;
    GemmEpilogue ep;
    if (sh.splits == 1) {
      ep.c32 = C;
      ep.ldc = ldc;
      gemm_tn(A, lda, B, ldb, M, N, K, kEpiF32, ep, err.p, s, sh);
    } else {
      DBuf<float> part;
      part.alloc((size_t)sh.splits * M * N);
      ep.c32 = part.p;
      ep.ldc = N;
      ep.split_stride = (int64_t)M * N;
      gemm_tn(A, lda, B, ldb, M, N, K, kEpiF32, ep, err.p, s, sh);
      const int kt = (K + 63) / 64, per = (kt + sh.splits - 1) / sh.splits, S = (kt + per - 1) / per;
      k_sum_slices<<<blocks_for((int64_t)M * N, 256), 256, 0, s>>>(part.p, S, (int64_t)M * N, (int64_t)M * N, C, ldc,
                                                                  N, N);
      CCG_CUDA(cudaGetLastError());
      CCG_CUDA(cudaStreamSynchronize(s));
    }
    int h = 0;
    CCG_CUDA(cudaMemcpyAsync(&h, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CCG_CUDA(cudaStreamSynchronize(s));
    CCG_CHECK(h == 0, CC_ERR_TIMEOUT, "a bounded wait in the GEMM kernel expired");
  })
}

cc_status cc_mlp_activation(const float* x, int32_t n, float* out, void* stream) {
  CC_API_BODY("cc_mlp_activation", {
    CCG_CHECK(x && out && n >= 0, CC_ERR_INVALID_ARG, "bad arguments");
    if (n == 0) return CC_OK;
    gelu_check(x, n, out, (cudaStream_t)stream);
    CCG_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  })
}

cc_status cc_mlp_create(const cc_mlp_config* cfg, void* stream, cc_mlp** out) {
  cc_mlp* net = nullptr;
  try {
    ccg::clear_error();
    CCG_CHECK(cfg && out, CC_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    CCG_CHECK(cfg->d_in >= 1 && cfg->hidden >= 8 && cfg->hidden % 8 == 0 && cfg->layers >= 1 && cfg->d_out >= 8 &&
                  cfg->d_out % 8 == 0 && cfg->max_batch >= 1 && cfg->max_batch <= (1 << 20) && cfg->d_in <= 65536 &&
                  cfg->hidden <= 65536 && cfg->d_out <= 65536,
              CC_ERR_INVALID_ARG, "bad network shape (hidden and d_out multiples of 8)");
    net = new cc_mlp();
    net->stream = (cudaStream_t)stream;
    net->dims.push_back(cfg->d_in);
    for (int l = 0; l < cfg->layers; ++l) net->dims.push_back(cfg->hidden);
    net->dims.push_back(cfg->d_out);
    net->L = (int)net->dims.size() - 1;
    int64_t o = 0;
    for (int l = 0; l < net->L; ++l) {
      const int N = net->dims[l + 1], K = net->dims[l];
      net->off_w.push_back(o);
      o += (int64_t)N * K;
      net->off_b.push_back(o);
      o += N;
      net->ldk.push_back(round8(K));
      net->ldn.push_back(round8(N));
    }
    net->nparams = o;
    net->max_batch = cfg->max_batch;
    net->ldB = round8(cfg->max_batch);
    cudaStream_t s = net->stream;
    net->params.alloc(o);
    net->grad.alloc(o);
    net->adam_m.alloc(o);
    net->adam_v.alloc(o);
    CCG_CUDA(cudaMemsetAsync(net->params.p, 0, o * sizeof(float), s));
    CCG_CUDA(cudaMemsetAsync(net->grad.p, 0, o * sizeof(float), s));
    CCG_CUDA(cudaMemsetAsync(net->adam_m.p, 0, o * sizeof(float), s));
    CCG_CUDA(cudaMemsetAsync(net->adam_v.p, 0, o * sizeof(float), s));
    net->w16.resize(net->L);
    net->wt16.resize(net->L);
    int64_t part = 1;
    for (int l = 0; l < net->L; ++l) {
      const int N = net->dims[l + 1], K = net->dims[l];
      net->w16[l].alloc((size_t)N * net->ldk[l]);
      net->wt16[l].alloc((size_t)K * net->ldn[l]);
      CCG_CUDA(cudaMemsetAsync(net->w16[l].p, 0, (size_t)N * net->ldk[l] * sizeof(bf16), s));
      CCG_CUDA(cudaMemsetAsync(net->wt16[l].p, 0, (size_t)K * net->ldn[l] * sizeof(bf16), s));
      const GemmShape sh = gemm_pick_shape(N, K, net->max_batch, true);
      part = std::max<int64_t>(part, (int64_t)sh.splits * N * K);
    }
    const int B = net->max_batch, ldB = net->ldB;
    net->z32.resize(net->L - 1);
    net->h16.resize(net->L - 1);
    net->ht16.resize(net->L - 1);
    int hmax = 8;
    for (int l = 0; l + 1 < net->L; ++l) {
      const int N = net->dims[l + 1];
      hmax = std::max(hmax, N);
      net->z32[l].alloc((size_t)B * N);
      net->h16[l].alloc((size_t)B * N);
      net->ht16[l].alloc((size_t)N * ldB);
    }
    net->y32.alloc((size_t)B * cfg->d_out);
    net->dy16.alloc((size_t)B * cfg->d_out);
    net->dyt16.alloc((size_t)cfg->d_out * ldB);
    for (int c = 0; c < 2; ++c) {
      net->dz16[c].alloc((size_t)B * hmax);
      net->dzt16[c].alloc((size_t)hmax * ldB);
    }
    net->partial.alloc((size_t)part);
    net->xb.alloc((size_t)B * round8(cfg->d_in));
    net->xbt.alloc((size_t)cfg->d_in * ldB);
    net->tb.alloc((size_t)B * cfg->d_out);
    net->loss_part.alloc((size_t)((cfg->d_out + 31) / 32) * ((B + 31) / 32));
    net->loss_hist.alloc(1);
    net->step_dev.alloc(1);
    net->adam_pw.alloc(2);
    net->err.alloc(1);
    CCG_CUDA(cudaMemsetAsync(net->err.p, 0, sizeof(int), s));
    CCG_CUDA(cudaStreamSynchronize(s));
    *out = net;
    return CC_OK;
  } catch (const ccg::Fail& f) {
    cc_mlp_destroy(net);
    return f.st;
  } catch (...) {
    cc_mlp_destroy(net);
    ccg::set_error("cc_mlp_create: unexpected error");
    return CC_ERR_STATE;
  }
}

void cc_mlp_destroy(cc_mlp* net) {
  if (!net) return;
  if (net->stream) cudaStreamSynchronize(net->stream);
  else cudaDeviceSynchronize();
  delete net;  // device buffers are released by their destructors
}

int64_t cc_mlp_param_count(const cc_mlp* net) { return net ? net->nparams : 0; }

cc_status cc_mlp_set_params(cc_mlp* net, const float* params, int64_t count) {
  CC_API_BODY("cc_mlp_set_params", {
    CCG_CHECK(net && params && count == net->nparams, CC_ERR_INVALID_ARG, "parameter count mismatch");
    cudaStream_t s = net->stream;
    CCG_CUDA(cudaMemcpyAsync(net->params.p, params, count * sizeof(float), cudaMemcpyHostToDevice, s));
    CCG_CUDA(cudaMemsetAsync(net->adam_m.p, 0, count * sizeof(float), s));
    CCG_CUDA(cudaMemsetAsync(net->adam_v.p, 0, count * sizeof(float), s));
    net->adam_t = 0;
    net->refresh_bf16();
    CCG_CUDA(cudaStreamSynchronize(s));
  })
}

cc_status cc_mlp_get_params(const cc_mlp* net, float* params, int64_t count) {
  CC_API_BODY("cc_mlp_get_params", {
    CCG_CHECK(net && params && count == net->nparams, CC_ERR_INVALID_ARG, "parameter count mismatch");
    CCG_CUDA(cudaStreamSynchronize(net->stream));
    CCG_CUDA(cudaMemcpy(params, net->params.p, count * sizeof(float), cudaMemcpyDeviceToHost));
  })
}

// File layout: 8-byte tag "CCMLP01\0", int32 count of widths, the widths
// (d_in, hidden..., d_out), int64 parameter count, the float32 parameters in
// the cc_mlp_set_params order; all little-endian as written by this host.
static const char kMlpTag[8] = {'C', 'C', 'M', 'L', 'P', '0', '1', '\0'};

cc_status cc_mlp_save(const cc_mlp* net, const char* path) {
  CC_API_BODY("cc_mlp_save", {
    CCG_CHECK(net && path, CC_ERR_INVALID_ARG, "NULL argument");
    std::vector<float> p(net->nparams);
    CCG_CUDA(cudaStreamSynchronize(net->stream));
    CCG_CUDA(cudaMemcpy(p.data(), net->params.p, p.size() * sizeof(float), cudaMemcpyDeviceToHost));
    FILE* f = std::fopen(path, "wb");
    CCG_CHECK(f, CC_ERR_INVALID_ARG, std::string("cannot open ") + path + " for writing");
    const int32_t nd = (int32_t)net->dims.size();
    const int64_t np = net->nparams;
    bool ok = std::fwrite(kMlpTag, 1, 8, f) == 8 && std::fwrite(&nd, sizeof(nd), 1, f) == 1;
    for (int d : net->dims) {
      const int32_t v = d;
      ok = ok && std::fwrite(&v, sizeof(v), 1, f) == 1;
    }
    ok = ok && std::fwrite(&np, sizeof(np), 1, f) == 1 && std::fwrite(p.data(), sizeof(float), p.size(), f) == p.size();
    ok = (std::fclose(f) == 0) && ok;
    CCG_CHECK(ok, CC_ERR_STATE, std::string("write to ") + path + " failed");
  })
}

cc_status cc_mlp_load(cc_mlp* net, const char* path) {
  CC_API_BODY("cc_mlp_load", {
    CCG_CHECK(net && path, CC_ERR_INVALID_ARG, "NULL argument");
    FILE* f = std::fopen(path, "rb");
    CCG_CHECK(f, CC_ERR_INVALID_ARG, std::string("cannot open ") + path);
    char tag[8] = {0};
    int32_t nd = 0;
    int64_t np = 0;
    bool ok = std::fread(tag, 1, 8, f) == 8 && std::memcmp(tag, kMlpTag, 8) == 0 &&
              std::fread(&nd, sizeof(nd), 1, f) == 1 && nd == (int32_t)net->dims.size();
    for (int k = 0; ok && k < nd; ++k) {
      int32_t v = 0;
      ok = std::fread(&v, sizeof(v), 1, f) == 1 && v == net->dims[k];
    }
    ok = ok && std::fread(&np, sizeof(np), 1, f) == 1 && np == net->nparams;
    std::vector<float> p(ok ? np : 0);
    ok = ok && std::fread(p.data(), sizeof(float), p.size(), f) == p.size();
    std::fclose(f);
    CCG_CHECK(ok, CC_ERR_INVALID_ARG, std::string(path) + " is not a parameter file of this network's shape");
    const cc_status st = cc_mlp_set_params(net, p.data(), np);
    CCG_CHECK(st == CC_OK, st, "cc_mlp_load: setting the parameters failed");
  })
}

cc_status cc_mlp_forward(cc_mlp* net, const void* X, int64_t ldx, int64_t rows, float* Y, int64_t ldy) {
  CC_API_BODY("cc_mlp_forward", {
    CCG_CHECK(net && Y, CC_ERR_INVALID_ARG, "NULL argument");
    CCG_CHECK(rows >= 1 && rows < (int64_t(1) << 31), CC_ERR_INVALID_ARG, "bad row count");
    CCG_CHECK(ldy >= net->d_out(), CC_ERR_INVALID_ARG, "ldy too small");
    require_bf16_operand(X, ldx, net->d_in(), "X");
    CCG_CUDA(cudaMemsetAsync(net->err.p, 0, sizeof(int), net->stream));
    net->forward_rows(static_cast<const bf16*>(X), ldx, rows, Y, ldy);
    net->check_err();
  })
}

cc_status cc_mlp_set_fused(cc_mlp* net, int32_t on) {
  CC_API_BODY("cc_mlp_set_fused", {
    CCG_CHECK(net, CC_ERR_INVALID_ARG, "NULL argument");
    CCG_CHECK(on >= 0 && on <= 2, CC_ERR_INVALID_ARG, "inference kernel must be 0, 1 or 2");
    net->fused_inference = on;
  })
}

cc_status cc_mlp_loss_grad(cc_mlp* net, const void* X, int64_t ldx, const float* T, int64_t ldt, int32_t rows,
                           double* loss, float* grad) {
  CC_API_BODY("cc_mlp_loss_grad", {
    CCG_CHECK(net && T, CC_ERR_INVALID_ARG, "NULL argument");
    CCG_CHECK(rows >= 1 && rows <= net->max_batch, CC_ERR_INVALID_ARG, "rows must be in [1, max_batch]");
    CCG_CHECK(ldt >= net->d_out(), CC_ERR_INVALID_ARG, "ldt too small");
    require_bf16_operand(X, ldx, net->d_in(), "X");
    cudaStream_t s = net->stream;
    CCG_CUDA(cudaMemsetAsync(net->err.p, 0, sizeof(int), s));
    const bf16* Xb = static_cast<const bf16*>(X);
    net->transpose_input(Xb, ldx, rows);
    net->forward_train(Xb, ldx, rows);
    net->backward(T, ldt, rows, net->loss_hist.p);
    if (grad) CCG_CUDA(cudaMemcpyAsync(grad, net->grad.p, net->nparams * sizeof(float), cudaMemcpyDeviceToDevice, s));
    double h = 0.0;
    CCG_CUDA(cudaMemcpyAsync(&h, net->loss_hist.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    net->check_err();
    if (loss) *loss = h;
  })
}

cc_status cc_mlp_adam_step(cc_mlp* net, const float* grad, const cc_adam* opt) {
  CC_API_BODY("cc_mlp_adam_step", {
    CCG_CHECK(net && grad && opt, CC_ERR_INVALID_ARG, "NULL argument");
    net->adam(grad, *opt);
    CCG_CUDA(cudaStreamSynchronize(net->stream));
  })
}

cc_status cc_mlp_train(cc_mlp* net, const void* X, int64_t ldx, const float* T, int64_t ldt, int64_t n_samples,
                       const int32_t* idx, int32_t steps, int32_t batch, const cc_adam* opt, double* losses) {
  CC_API_BODY("cc_mlp_train", {
    CCG_CHECK(net && T && idx && opt, CC_ERR_INVALID_ARG, "NULL argument");
    CCG_CHECK(batch >= 1 && batch <= net->max_batch && steps >= 0 && n_samples >= 1, CC_ERR_INVALID_ARG,
              "bad batch, step or sample count");
    CCG_CHECK(ldt >= net->d_out(), CC_ERR_INVALID_ARG, "ldt too small");
    require_bf16_operand(X, ldx, net->d_in(), "X");
    cudaStream_t s = net->stream;
    CCG_CUDA(cudaMemsetAsync(net->err.p, 0, sizeof(int), s));
    if (steps == 0) return CC_OK;
    net->loss_hist.alloc(steps);
    const int ldxb = round8(net->d_in());
    const int chunks = ldxb / 8;
    const int64_t t0 = net->adam_t;
    int* step = net->step_dev.p;
    CCG_CUDA(cudaMemsetAsync(step, 0, sizeof(int), s));
    const bool vec4 = net->d_out() % 4 == 0 && ldt % 4 == 0 && (reinterpret_cast<uintptr_t>(T) & 15) == 0 &&
                      (reinterpret_cast<uintptr_t>(net->tb.p) & 15) == 0;
    // beta^t of the first step; each step's advance multiplies them by beta
    net->adam_pw_host[0] = std::pow((double)opt->beta1, (double)(t0 + 1));
    net->adam_pw_host[1] = std::pow((double)opt->beta2, (double)(t0 + 1));
    CCG_CUDA(cudaMemcpyAsync(net->adam_pw.p, net->adam_pw_host, 2 * sizeof(double), cudaMemcpyHostToDevice, s));
    // one training step; its minibatch, loss slot and Adam step number come
    // from the device step counter, which the step advances last
    auto one_step = [&]() {
      cudaStream_t q = net->stream;
      k_gather_rows_bf16<<<blocks_for((int64_t)batch * chunks, 256), 256, 0, q>>>(
          static_cast<const bf16*>(X), ldx, idx, step, batch, chunks, net->xb.p, ldxb);
      CCG_CUDA(cudaGetLastError());
      if (vec4)
        k_gather_rows_f32<4><<<blocks_for((int64_t)batch * net->d_out() / 4, 256), 256, 0, q>>>(
            T, ldt, idx, step, batch, net->d_out(), net->tb.p, net->d_out());
      else
        k_gather_rows_f32<1><<<blocks_for((int64_t)batch * net->d_out(), 256), 256, 0, q>>>(
            T, ldt, idx, step, batch, net->d_out(), net->tb.p, net->d_out());
      CCG_CUDA(cudaGetLastError());
      net->transpose_input(net->xb.p, ldxb, batch);
      net->forward_train(net->xb.p, ldxb, batch);
      net->backward(net->tb.p, net->d_out(), batch, net->loss_hist.p, step);
      net->adam_dev(net->grad.p, *opt);
      k_step_advance<<<1, 1, 0, q>>>(step, net->adam_pw.p, (double)opt->beta1, (double)opt->beta2);
      CCG_CUDA(cudaGetLastError());
    };
    // the first step runs directly (it also fills every host-side cache the
    // launches use); the others replay one captured step (about 30 launches).
    // The legacy default stream cannot be captured: the step is then recorded
    // on a private stream, and the graph still runs on the network's stream.
    one_step();
    if (steps > 1) {
      cudaStream_t cap = s, own = nullptr;
      if (s == nullptr || s == cudaStreamLegacy) {
        CCG_CUDA(cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
        cap = own;
      }
      cudaGraph_t g = nullptr;
      cudaGraphExec_t exec = nullptr;
      cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      if (ce == cudaSuccess) {
        net->stream = cap;
        try {
          one_step();
        } catch (...) {
          net->stream = s;
          cudaStreamEndCapture(cap, &g);
          if (g) cudaGraphDestroy(g);
          if (own) cudaStreamDestroy(own);
          throw;
        }
        net->stream = s;
        ce = cudaStreamEndCapture(cap, &g);
      }
      if (ce == cudaSuccess) {
        ce = cudaGraphInstantiate(&exec, g, 0);
        cudaGraphDestroy(g);
      }
      for (int st = 1; st < steps && ce == cudaSuccess; ++st) ce = cudaGraphLaunch(exec, s);
      if (exec) cudaGraphExecDestroy(exec);
      if (own) cudaStreamDestroy(own);
      CCG_CUDA(ce);
    }
    net->adam_t += steps;
    if (losses) CCG_CUDA(cudaMemcpyAsync(losses, net->loss_hist.p, steps * sizeof(double), cudaMemcpyDeviceToHost, s));
    net->check_err();
  })
}

cc_status cc_learned_inputs(cc_mesh* m, void* X, int64_t ldx, float* T, int64_t ldt, int64_t rows_cap,
                            int64_t* rows) {
  CC_API_BODY("cc_learned_inputs", {
    CCG_CHECK(m && X, CC_ERR_INVALID_ARG, "NULL argument");
    CCG_CHECK(ldx >= CC_LEARNED_LDX && ldx % 8 == 0, CC_ERR_INVALID_ARG, "ldx must be >= 264 and a multiple of 8");
    CCG_CHECK(rows_cap >= m->n_free, CC_ERR_INVALID_ARG, "rows_cap below the number of free vertices");
    CCG_CHECK(!T || ldt >= CC_LEARNED_D_OUT, CC_ERR_INVALID_ARG, "ldt too small");
    CCG_CHECK(!T || m->k_ring == 2, CC_ERR_STATE, "targets need computed k = 2 bases (cc_build_subspace(mesh, 2))");
    cudaStream_t s = m->stream;
    const SlotTable tab = make_slot_table();
    DBuf<double> Xs;
    DBuf<double2> vmat;
    upload_rest_inputs(*m, Xs, vmat);
    DBuf<int> err;
    err.alloc(1);
    CCG_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    const int nf = (int)m->n_free;
    k_features<<<blocks_for(nf, 128), 128, 0, s>>>(nf, m->d_free_rows.p, m->n, Xs.p, m->d_nbr_ptr.p, m->d_nbr_idx.p,
                                                   m->d_pinned.p, vmat.p, tab, static_cast<bf16*>(X), ldx, err.p);
    CCG_CUDA(cudaGetLastError());
    if (T) {
      DBuf<int8_t> slots;
      slots.alloc(std::max<size_t>(1, m->sup_idx.size()));
      k_support_slots<<<blocks_for(nf, 128), 128, 0, s>>>(nf, m->d_free_rows.p, m->n, Xs.p, m->d_nbr_ptr.p,
                                                          m->d_nbr_idx.p, m->d_sup_ptr.p, m->d_sup_idx.p, tab, slots.p,
                                                          err.p);
      CCG_CUDA(cudaGetLastError());
      CCG_CUDA(cudaMemsetAsync(T, 0, (size_t)nf * ldt * sizeof(float), s));
      k_targets<<<blocks_for((int64_t)nf * 32, 256), 256, 0, s>>>(nf, m->d_free_rows.p, m->d_sup_ptr.p, slots.p,
                                                                  m->f64.U.p, T, ldt);
      CCG_CUDA(cudaGetLastError());
      read_err(err, s, "cc_learned_inputs: a vertex within 2 hops is off the lattice stencil");
    } else {
      read_err(err, s, "cc_learned_inputs: a vertex within 2 hops is off the lattice stencil");
    }
    if (rows) *rows = m->n_free;
  })
}

cc_status cc_build_learned_subspace(cc_mesh* m, cc_mlp* net, double tau, double* rho_out, cc_learned_stats* st) {
  CC_API_BODY("cc_build_learned_subspace", {
    const auto t_all = std::chrono::steady_clock::now();
    CCG_CHECK(m && net, CC_ERR_INVALID_ARG, "NULL argument");
    CCG_CHECK(net->d_in() == CC_LEARNED_D_IN && net->d_out() == CC_LEARNED_D_OUT, CC_ERR_INVALID_ARG,
              "network must map 258 inputs to 576 outputs");
    CCG_CHECK(m->num_colors > 0, CC_ERR_STATE, "cc_color must run before building bases");
    CCG_CHECK(m->h == 0.0, CC_ERR_INVALID_ARG, "learned bases are for quasistatic meshes (h = 0)");
    CCG_CHECK(std::isfinite(tau) && tau > 0.0, CC_ERR_INVALID_ARG, "tau must be positive");
    cudaStream_t s = m->stream;
    cc_learned_stats out{};
    ensure_state(*m, CC_PREC_FP64);
    drop_graph(*m);
    // the network runs on the mesh's stream for this call
    struct StreamSwap {
      MlpNet* n;
      cudaStream_t old;
      ~StreamSwap() { n->stream = old; }
    } swap{net, net->stream};
    net->stream = s;

    auto t0 = std::chrono::steady_clock::now();
    build_supports(*m, 2);
    CCG_CUDA(cudaStreamSynchronize(s));
    out.ms_supports = ms_since(t0);

    t0 = std::chrono::steady_clock::now();
    const SlotTable tab = make_slot_table();
    DBuf<double> Xs;
    DBuf<double2> vmat;
    upload_rest_inputs(*m, Xs, vmat);
    const int nf = (int)m->n_free;
    DBuf<bf16> Xin;
    Xin.alloc((size_t)nf * CC_LEARNED_LDX);
    DBuf<int> err;
    err.alloc(1);
    CCG_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    k_features<<<blocks_for(nf, 128), 128, 0, s>>>(nf, m->d_free_rows.p, m->n, Xs.p, m->d_nbr_ptr.p, m->d_nbr_idx.p,
                                                   m->d_pinned.p, vmat.p, tab, Xin.p, CC_LEARNED_LDX, err.p);
    CCG_CUDA(cudaGetLastError());
    DBuf<int8_t> slots;
    slots.alloc(std::max<size_t>(1, m->sup_idx.size()));
    k_support_slots<<<blocks_for(nf, 128), 128, 0, s>>>(nf, m->d_free_rows.p, m->n, Xs.p, m->d_nbr_ptr.p,
                                                        m->d_nbr_idx.p, m->d_sup_ptr.p, m->d_sup_idx.p, tab, slots.p,
                                                        err.p);
    CCG_CUDA(cudaGetLastError());
    read_err(err, s, "cc_build_learned_subspace: a vertex within 2 hops is off the lattice stencil");
    out.ms_inputs = ms_since(t0);

    t0 = std::chrono::steady_clock::now();
    DBuf<float> Y;
    Y.alloc((size_t)nf * CC_LEARNED_D_OUT);
    CCG_CUDA(cudaMemsetAsync(net->err.p, 0, sizeof(int), s));
    net->forward_rows(Xin.p, CC_LEARNED_LDX, nf, Y.p, CC_LEARNED_D_OUT);
    net->check_err();
    out.ms_infer = ms_since(t0);

    t0 = std::chrono::steady_clock::now();
    k_assemble<<<blocks_for((int64_t)nf * 32, 256), 256, 0, s>>>(nf, m->d_free_rows.p, m->d_sup_ptr.p, slots.p, Y.p,
                                                                 CC_LEARNED_D_OUT, m->f64.U.p, m->mx.U.p);
    CCG_CUDA(cudaGetLastError());
    CCG_CUDA(cudaStreamSynchronize(s));
    out.ms_assemble = ms_since(t0);

    t0 = std::chrono::steady_clock::now();
    rest_hessian_f64(*m);
    DBuf<double> rho;
    rho.alloc(nf);
    k_basis_residual<<<blocks_for((int64_t)nf * 32, 256), 256, 0, s>>>(nf, m->d_free_rows.p, m->d_sup_ptr.p,
                                                                       m->d_sup_idx.p, m->d_up_ptr.p, m->d_up_col.p,
                                                                       m->d_nbr_ptr.p, m->d_nbr_idx.p, m->f64.bsr.p,
                                                                       m->f64.U.p, rho.p);
    CCG_CUDA(cudaGetLastError());
    std::vector<double> hr(nf);
    CCG_CUDA(cudaMemcpyAsync(hr.data(), rho.p, nf * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (rho_out) CCG_CUDA(cudaMemcpyAsync(rho_out, rho.p, nf * sizeof(double), cudaMemcpyDeviceToDevice, s));
    std::vector<int32_t> frows(nf);
    CCG_CUDA(cudaMemcpyAsync(frows.data(), m->d_free_rows.p, nf * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CCG_CUDA(cudaStreamSynchronize(s));
    std::vector<int32_t> fall;
    double rmax = 0.0, rsum = 0.0;
    for (int r = 0; r < nf; ++r) {
      const int32_t v = frows[r];
      const bool has = m->sup_ptr[v + 1] > m->sup_ptr[v];
      CCG_CHECK(std::isfinite(hr[r]), CC_ERR_NUMERIC, "non-finite basis residual");
      rsum += hr[r];
      if (has && hr[r] >= tau) fall.push_back(v);
      else rmax = std::max(rmax, hr[r]);
    }
    out.ms_residual = ms_since(t0);

    t0 = std::chrono::steady_clock::now();
    if (!fall.empty()) {
      DBuf<int32_t> fl;
      fl.upload(fall, s);
      patch_solves(*m, fl.p, (int64_t)fall.size(), true);
      bases_to_f32(*m);
    }
    CCG_CUDA(cudaStreamSynchronize(s));
    out.ms_fallback = ms_since(t0);

    out.n_free = nf;
    out.n_fallback = (int64_t)fall.size();
    out.rho_max = rmax;
    out.rho_mean = nf ? rsum / nf : 0.0;
    out.ms_total = ms_since(t_all);
    if (st) *st = out;
  })
}

}  // extern "C"
