// Fused subspace-coupling products and Schur-condensed local solve
// (Eq. 9-12), one CTA per free vertex i of the current colour.
//
// For vertex i with support S (|S| = m) and basis blocks U[s] (3x3):
//   A  = sum_{l in S} H_il U[l]                              (= H_iC U_i)
//   Ht = sum_{j, l in S} U[j]^T H_jl U[l]                    (= U^T H_CC U)
//   b  = sum_{j in S} U[j]^T g_j                             (= U^T g_C)
// then, in float64 on one thread:
//   S = A Ht^{-1} A^T,  gt = g_i - A Ht^{-1} b,  dx_i = -(H_ii - S)^{-1} gt
// and x_i += dx_i (the subspace part U dalpha is discarded, Sec. 3.1).
// H is stored as its upper 3x3 blocks (l >= j, diagonal first, each block
// padded to 3 x 4 for 128-bit loads), so each unordered pair of the support
// is read once.  The CTA stages U_i in shared memory; a precomputed slot map
// gives, for every block it reads, the support slot of the block's column.
// Same-coloured vertices share no tet, and this kernel reads only g, H and U,
// so writing x in place is race-free for both schedules.
#include <vector>

#include "cc_internal.cuh"
#include "dmath.cuh"

namespace ccg {

namespace {

constexpr double kPivotRel = 1e-12;

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }



template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Loads the 3x3 block p of the padded upper rows.
template <typename HT>
__device__ __forceinline__ void load_block(const HT* __restrict__ bsr, int64_t p, HT* H);

template <>
__device__ __forceinline__ void load_block<float>(const float* __restrict__ bsr, int64_t p, float* H) {
  const float4* b = reinterpret_cast<const float4*>(bsr + p * 12);
  const float4 r0 = __ldg(b), r1 = __ldg(b + 1), r2 = __ldg(b + 2);
  H[0] = r0.x; H[1] = r0.y; H[2] = r0.z;
  H[3] = r1.x; H[4] = r1.y; H[5] = r1.z;
  H[6] = r2.x; H[7] = r2.y; H[8] = r2.z;
}

template <>
__device__ __forceinline__ void load_block<double>(const double* __restrict__ bsr, int64_t p, double* H) {
  const double2* b = reinterpret_cast<const double2*>(bsr + p * 12);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const double2 u = __ldg(b + 2 * r), v = __ldg(b + 2 * r + 1);
    H[3 * r] = u.x; H[3 * r + 1] = u.y; H[3 * r + 2] = v.x;
  }
}


// The coupling CTA's shared memory: U_i (padded rows), the support rows'
// starts, lengths, ids and slot-map offsets, the slot map, and the 18
// reduction partials of every thread (stride threads + 1).
template <typename HT>
__host__ __device__ inline size_t cta_smem_bytes(int sup_max, int64_t smap_max, int code_bytes, int nthreads) {
  return align16((size_t)sup_max * 12 * sizeof(HT)) + 4 * align16((size_t)(sup_max + 1) * 4) +
         align16((size_t)(smap_max + kSlotMapSlack) * code_bytes) + (size_t)18 * (nthreads + 1) * sizeof(HT);
}

template <typename SlotT>
struct SlotCodes;
template <>
struct SlotCodes<uint8_t> {
  static constexpr unsigned kNone = 0xFF, kSelf = 0xFE, kDiag = 0xFD;
};
template <>
struct SlotCodes<uint16_t> {
  static constexpr unsigned kNone = 0xFFFF, kSelf = 0xFFFE, kDiag = 0xFFFD;
};

// Stages U_i in shared memory, rotated for corotated bases (Sec. 3.1):
// U_i^rot[j] = R_j U_i[j] (rot: [n][9] row-major rotations, or nullptr).
// Slot a's entry (row r, column d) goes to Us[kSlot a + kRow r + d]: (9, 3)
// packs the blocks, (12, 4) pads each row to four values for vector loads
// (the pads are zeroed).
template <typename HT, int kSlot = 9, int kRow = 3>
__device__ __forceinline__ void stage_basis(HT* Us, const HT* __restrict__ U, const HT* __restrict__ rot,
                                            const int32_t* __restrict__ sup_idx, int s0, int m, int t, int nt) {
  if (!rot) {
    if constexpr (kSlot == 9) {
      for (int k = t; k < 9 * m; k += nt) Us[k] = U[(int64_t)s0 * 9 + k];
    } else {
      static_assert(kSlot == 12 && kRow == 4, "padded slots are three rows of four");
      // row q of the copy (slot q / 3, row q % 3) is the three values at 3 q
      // past the support's first block, stored as one padded row at 4 q
      const HT* src = U + (int64_t)s0 * 9;
      for (int q = t; q < 3 * m; q += nt) {
        const HT u0 = __ldg(src + 3 * q), u1 = __ldg(src + 3 * q + 1), u2 = __ldg(src + 3 * q + 2);
        if constexpr (sizeof(HT) == 4) {
          reinterpret_cast<float4*>(Us)[q] = make_float4(u0, u1, u2, 0.f);
        } else {
          reinterpret_cast<double2*>(Us)[2 * q] = make_double2(u0, u1);
          reinterpret_cast<double2*>(Us)[2 * q + 1] = make_double2(u2, 0.0);
        }
      }
    }
    return;
  }
  for (int a = t; a < m; a += nt) {
    const HT* R = rot + 9 * (int64_t)sup_idx[s0 + a];
    const HT* Ua = U + (int64_t)(s0 + a) * 9;
    HT r[9], u[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      r[q] = R[q];
      u[q] = Ua[q];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
      for (int d = 0; d < 3; ++d)
        Us[kSlot * a + kRow * i + d] = r[3 * i] * u[d] + r[3 * i + 1] * u[3 + d] + r[3 * i + 2] * u[6 + d];
      if (kRow == 4) Us[kSlot * a + kRow * i + 3] = HT(0);
    }
  }
}

// Loads the padded 3 x 4 slot at p (three 16-byte rows) into a packed 3 x 3.
template <typename HT>
__device__ __forceinline__ void load_slot(const HT* p, HT* u);
template <>
__device__ __forceinline__ void load_slot<float>(const float* p, float* u) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float4 v = q[r];
    u[3 * r] = v.x; u[3 * r + 1] = v.y; u[3 * r + 2] = v.z;
  }
}
template <>
__device__ __forceinline__ void load_slot<double>(const double* p, double* u) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const double2 a = q[2 * r], b = q[2 * r + 1];
    u[3 * r] = a.x; u[3 * r + 1] = a.y; u[3 * r + 2] = b.x;
  }
}

// What the condensation of a colour's vertices reads and writes.
template <typename HT>
struct CondenseArgs {
  const int32_t* verts;
  int64_t count;
  const HT* cpl;  // [count][32]: Ht (6), A (9), b (3), H_ii (9) per vertex
  const int32_t* sup_ptr;
  const int32_t* up_ptr;
  const HT* bsr;
  const double* g64;
  const float* g_hi;
  const float* g_lo;
  int64_t n;
  double* x;
  float4* x_hi;
  float4* x_lo;
  const int32_t* vert_mesh;
  const int32_t* active;
  unsigned long long* fallback;
  unsigned long long* err;
  int32_t* grp_cnt;  // arrivals per group of 32 list entries (fused kernel only)
};

// Condensation (Eq. 9-12) of list entry k.  3x3 inverses use the adjugate;
// the SPD guard is the Cholesky pivot test written with leading minors.  `AR`
// is the arithmetic type (double on both paths).  cpl is read through L2
// (__ldcg): in the fused kernel other CTAs wrote it during this launch.
template <typename AR, typename HT, bool kMixed, int kUpd>
__device__ __forceinline__ void condense_vertex(const CondenseArgs<HT>& c, int64_t k, AR rel) {
  using Ar = Arith<AR>;
  using V = typename Ar::V;
  const int i = c.verts[k];
  if (c.active[c.vert_mesh[i]] == 0) return;  // this mesh of the batch has stopped
  auto ld = [](HT v) -> V {
    if constexpr (sizeof(HT) == 4) return Ar::mkf((float)v);
    else return Ar::mk((double)v);
  };
  const HT* cp = c.cpl + k * 32;
  V H[9], gi[3];
  if (kUpd == CC_UPDATE_CD) {
    HT Hb[9];
    load_block(c.bsr, c.up_ptr[i], Hb);
#pragma unroll
    for (int q = 0; q < 9; ++q) H[q] = ld(Hb[q]);
  } else {
#pragma unroll
    for (int q = 0; q < 9; ++q) H[q] = ld(__ldcg(cp + 18 + q));
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if constexpr (!kMixed) gi[a] = Ar::mk(c.g64[3 * (int64_t)i + a]);
    else if constexpr (sizeof(V) == sizeof(double))
      gi[a] = (double)c.g_hi[3 * (int64_t)i + a] + (double)c.g_lo[3 * (int64_t)i + a];
    else gi[a] = V{c.g_hi[3 * (int64_t)i + a], c.g_lo[3 * (int64_t)i + a]};
  }
  V M[9], rhs[3];
  int fb = -1;
  bool done = false;
  if (kUpd != CC_UPDATE_CD) {
    const int m = c.sup_ptr[i + 1] - c.sup_ptr[i];
    if (m == 0) {
      fb = 0;
    } else {
      const V t0 = ld(__ldcg(cp + 0)), t1 = ld(__ldcg(cp + 1)), t2 = ld(__ldcg(cp + 2));
      const V t3 = ld(__ldcg(cp + 3)), t4 = ld(__ldcg(cp + 4)), t5 = ld(__ldcg(cp + 5));
      const V Ht[9] = {t0, t1, t2, t1, t3, t4, t2, t4, t5};
      V b[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) b[q] = ld(__ldcg(cp + 15 + q));
      if (kUpd == CC_UPDATE_JGS2) {
#pragma unroll
        for (int q = 0; q < 9; ++q) M[q] = Ar::add(H[q], Ht[q]);
#pragma unroll
        for (int q = 0; q < 3; ++q) rhs[q] = Ar::add(gi[q], b[q]);
        done = true;
      } else {
        V adj[6], det;
        if (sym3_adj<AR>(Ht, rel, adj, &det)) {
          V A[9];
#pragma unroll
          for (int q = 0; q < 9; ++q) A[q] = ld(__ldcg(cp + 6 + q));
          const V inv = Ar::div(Ar::mkf(1.0f), det);
          V Hi[9] = {adj[0], adj[1], adj[2], adj[1], adj[3], adj[4], adj[2], adj[4], adj[5]};
#pragma unroll
          for (int q = 0; q < 9; ++q) Hi[q] = Ar::mul(Hi[q], inv);
          // W = A Ht^{-1};  S = W A^T;  gt = g_i - W b
          V W[9];
#pragma unroll
          for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int q = 0; q < 3; ++q)
              W[3 * r + q] = Ar::fma(A[3 * r + 2], Hi[6 + q], Ar::fma(A[3 * r + 1], Hi[3 + q], Ar::mul(A[3 * r], Hi[q])));
#pragma unroll
          for (int r = 0; r < 3; ++r) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              const V Src = Ar::fma(W[3 * r + 2], A[3 * q + 2], Ar::fma(W[3 * r + 1], A[3 * q + 1], Ar::mul(W[3 * r], A[3 * q])));
              M[3 * r + q] = Ar::sub(H[3 * r + q], Src);
            }
            rhs[r] = Ar::sub(gi[r], Ar::fma(W[3 * r + 2], b[2], Ar::fma(W[3 * r + 1], b[1], Ar::mul(W[3 * r], b[0]))));
          }
          done = true;
        } else {
          fb = 1;
        }
      }
    }
  }
  V dx[3];
  bool ok = false;
  if (done) {
    V adj[6], det;
    if (sym3_adj<AR>(M, rel, adj, &det)) {
      const V inv = Ar::neg(Ar::div(Ar::mkf(1.0f), det));
      dx[0] = Ar::mul(inv, Ar::fma(adj[0], rhs[0], Ar::fma(adj[1], rhs[1], Ar::mul(adj[2], rhs[2]))));
      dx[1] = Ar::mul(inv, Ar::fma(adj[1], rhs[0], Ar::fma(adj[3], rhs[1], Ar::mul(adj[4], rhs[2]))));
      dx[2] = Ar::mul(inv, Ar::fma(adj[2], rhs[0], Ar::fma(adj[4], rhs[1], Ar::mul(adj[5], rhs[2]))));
      ok = true;
    } else {
      fb = kUpd == CC_UPDATE_JGS2 ? 1 : 2;
    }
  }
  if (!ok) {
    // coordinate descent step: one Newton step on vertex i
    V adj[6], det;
    if (sym3_adj<AR>(H, Ar::mkf(0.0f), adj, &det)) {
      const V inv = Ar::neg(Ar::div(Ar::mkf(1.0f), det));
      dx[0] = Ar::mul(inv, Ar::fma(adj[0], gi[0], Ar::fma(adj[1], gi[1], Ar::mul(adj[2], gi[2]))));
      dx[1] = Ar::mul(inv, Ar::fma(adj[1], gi[0], Ar::fma(adj[3], gi[1], Ar::mul(adj[4], gi[2]))));
      dx[2] = Ar::mul(inv, Ar::fma(adj[2], gi[0], Ar::fma(adj[4], gi[1], Ar::mul(adj[5], gi[2]))));
    } else {
      atomicOr(c.err, 1ull);
      return;
    }
  }
  if (fb >= 0) atomicAdd(&c.fallback[fb], 1ull);
  double d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) d[a] = Ar::to_double(dx[a]);
  if (!(isfinite(d[0]) && isfinite(d[1]) && isfinite(d[2]))) {
    atomicOr(c.err, 1ull);
    return;
  }
  double xn[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    xn[a] = c.x[a * c.n + i] + d[a];
    c.x[a * c.n + i] = xn[a];
  }
  if (kMixed) {
    df a0 = df_from_double(xn[0]), a1 = df_from_double(xn[1]), a2 = df_from_double(xn[2]);
    c.x_hi[i] = make_float4(a0.hi, a1.hi, a2.hi, 0.f);
    c.x_lo[i] = make_float4(a0.lo, a1.lo, a2.lo, 0.f);
  }
}

// Batched condensation, one list entry per thread: a warp condenses 32
// vertices at once, so the float64 3x3 algebra runs at full SIMD width
// instead of on one lane per vertex.
template <typename AR, typename HT, bool kMixed, int kUpd>
__global__ void k_condense(CondenseArgs<HT> c, AR rel) {
  pdl_entry();
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= c.count) return;
  condense_vertex<AR, HT, kMixed, kUpd>(c, k, rel);
}

// Tail of the fused coupling kernel: after its CTA has written the products
// of list entry blockIdx.x, the last CTA to finish in each group of 32
// entries condenses the whole group, one vertex per lane of its first warp
// (the float64 condensation at full warp width, no separate launch).  Every
// thread that wrote cpl fences before the CTA's arrival is counted; the
// counter is reset by the group's last CTA for the next launch.  Which CTA
// condenses does not change any result.
template <typename AR, typename HT, bool kMixed, int kUpd>
__device__ __forceinline__ void condense_group_tail(const CondenseArgs<HT>& c, AR rel) {
  __shared__ int last;
  __threadfence();
  __syncthreads();
  const int64_t grp = blockIdx.x >> 5;
  if (threadIdx.x == 0) {
    const int need = (int)min((int64_t)32, c.count - grp * 32);
    last = atomicAdd(c.grp_cnt + grp, 1) == need - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x >= 32) return;
  __threadfence();
  if (threadIdx.x == 0) c.grp_cnt[grp] = 0;
  const int64_t k = grp * 32 + threadIdx.x;
  if (k < c.count) condense_vertex<AR, HT, kMixed, kUpd>(c, k, rel);
}

// Coupling products, one CTA per free vertex i of the list.  Groups of
// 2^row_lanes_log2 threads take the block rows of the support S and of i
// itself; a group's threads take the row's upper blocks (H_jl, l >= j)
// round-robin.  The vertex's slot map (one code per block, staged in shared
// memory) gives each block's role.  Because H is symmetric,
//   Ht = sum_j (U_j^T Z_j + Z_j^T U_j),  Z_j = 1/2 H_jj U_j + sum_{l > j} H_jl U_l,
// so a thread accumulates its share of Z_j (27 FMA per block) and folds it
// with U_j once at the row's end; a block (j, i) of a support row gives A's
// term H_ij U_j = H_ji^T U_j; row i gives H_ii and the terms H_il U_l with
// l > i.  The CTA writes 27 values per vertex: Ht (6, symmetric), A (9),
// b (3), H_ii (9, stored directly by the thread that reads it).
// kFuse: the CTA then takes part in the group condensation (condense_group_tail).
template <typename HT, typename SlotT, bool kMixed, int kUpd, int kThreads, bool kFuse = false>
__global__ void __launch_bounds__(kThreads) k_couple(
    const int32_t* __restrict__ verts, int64_t count, const int32_t* __restrict__ sup_ptr,
    const int32_t* __restrict__ sup_idx, const HT* __restrict__ U, const int32_t* __restrict__ up_ptr,
    const int64_t* __restrict__ smap_ptr, const SlotT* __restrict__ smap, const HT* __restrict__ bsr,
    const double* __restrict__ g64, const float* __restrict__ g_hi, int sup_max, int64_t smap_max,
    const HT* __restrict__ rot, int row_lanes_log2, HT* __restrict__ cpl, CondenseArgs<HT> ca) {
  pdl_entry();
  using Codes = SlotCodes<SlotT>;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char* ptr = smem;
  HT* Us = reinterpret_cast<HT*>(ptr);  // [m][3][4]
  ptr += align16((size_t)sup_max * 12 * sizeof(HT));
  int* rstart = reinterpret_cast<int*>(ptr);
  ptr += align16((size_t)(sup_max + 1) * 4);
  int* rlen = reinterpret_cast<int*>(ptr);
  ptr += align16((size_t)(sup_max + 1) * 4);
  int* rid = reinterpret_cast<int*>(ptr);
  ptr += align16((size_t)(sup_max + 1) * 4);
  int* roff = reinterpret_cast<int*>(ptr);
  ptr += align16((size_t)(sup_max + 1) * 4);
  SlotT* code_words = reinterpret_cast<SlotT*>(ptr);
  ptr += align16((size_t)(smap_max + kSlotMapSlack) * sizeof(SlotT));
  HT* red = reinterpret_cast<HT*>(ptr);  // [18][kThreads + 1]

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i = verts[blockIdx.x];
  const int s0 = sup_ptr[i];
  const int m = sup_ptr[i + 1] - s0;
  const int64_t c0 = smap_ptr[i];
  const int ncodes = (int)(smap_ptr[i + 1] - c0);

  stage_basis<HT, 12, 4>(Us, U, rot, sup_idx, s0, m, tid, kThreads);
  // the slot map in 4-byte words from the word holding its first code (the
  // map is allocated with slack past its end); its codes start sh in
  constexpr int kPerWord = 4 / (int)sizeof(SlotT);
  const int64_t w0 = c0 / kPerWord;
  const int sh = (int)(c0 - w0 * kPerWord);
  const int nwords = (sh + ncodes + kPerWord - 1) / kPerWord;
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(smap) + w0;
    uint32_t* dst = reinterpret_cast<uint32_t*>(code_words);
    for (int k = tid; k < nwords; k += kThreads) dst[k] = __ldg(src + k);
  }
  const SlotT* codes = code_words + sh;
  for (int s = tid; s <= m; s += kThreads) {
    const int j = s < m ? sup_idx[s0 + s] : i;
    const int a = up_ptr[j];
    rstart[s] = a;
    rlen[s] = up_ptr[j + 1] - a;
    rid[s] = j;
  }
  __syncthreads();
  // exclusive prefix of the row lengths (offsets into the slot map), warp 0
  if (warp == 0) {
    int carry = 0;
    for (int base = 0; base <= m; base += 32) {
      const int s = base + lane;
      const int v = s <= m ? rlen[s] : 0;
      int incl = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      if (s <= m) roff[s] = carry + incl - v;
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
  }
  __syncthreads();

  HT h00 = 0, h01 = 0, h02 = 0, h11 = 0, h12 = 0, h22 = 0;
  HT A[9], b[3] = {0, 0, 0};
  mat3_zero(A);
  const int nl = 1 << row_lanes_log2, rl = tid & (nl - 1);
  for (int r = tid >> row_lanes_log2; r <= m; r += kThreads >> row_lanes_log2) {
    const int P = rstart[r], L = rlen[r], off = roff[r];
    if (r < m) {
      HT Uj[9], Z[9];
      load_slot(Us + 12 * r, Uj);
      mat3_zero(Z);
      bool any = false;
      for (int q = rl; q < L; q += nl) {
        const unsigned code = codes[off + q];
        if (code == Codes::kNone) continue;
        HT H[9];
        load_block(bsr, (int64_t)P + q, H);
        if (code == Codes::kSelf) {
          if (kUpd == CC_UPDATE_CC) mat3_tmul_acc(H, Uj, A);
        } else if (code == Codes::kDiag) {
#pragma unroll
          for (int c = 0; c < 9; ++c) H[c] *= HT(0.5);
          mat3_mul_acc(H, Uj, Z);
          any = true;
        } else {
          HT Ul[9];
          load_slot(Us + 12 * (int)code, Ul);
          mat3_mul_acc(H, Ul, Z);
          any = true;
        }
      }
      if (any) {
        HT M[9];
        mat3_zero(M);
        mat3_tmul_acc(Uj, Z, M);
        h00 += 2 * M[0]; h11 += 2 * M[4]; h22 += 2 * M[8];
        h01 += M[1] + M[3]; h02 += M[2] + M[6]; h12 += M[5] + M[7];
      }
      if (rl == 0) {
        const int j = rid[r];
        HT gj[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) gj[a] = kMixed ? (HT)g_hi[3 * (int64_t)j + a] : (HT)g64[3 * (int64_t)j + a];
#pragma unroll
        for (int c = 0; c < 3; ++c) b[c] += Uj[c] * gj[0] + Uj[3 + c] * gj[1] + Uj[6 + c] * gj[2];
      }
    } else {
      for (int q = rl; q < L; q += nl) {
        const unsigned code = codes[off + q];
        if (code == Codes::kNone) continue;
        HT H[9];
        load_block(bsr, (int64_t)P + q, H);
        if (code == Codes::kDiag) {
#pragma unroll
          for (int c = 0; c < 9; ++c) cpl[(int64_t)blockIdx.x * 32 + 18 + c] = H[c];
        } else if (kUpd == CC_UPDATE_CC) {
          HT Ul[9];
          load_slot(Us + 12 * (int)code, Ul);
          mat3_mul_acc(H, Ul, A);
        }
      }
    }
  }

  // CTA reduction of 18 values in a fixed order: every thread stores its
  // partials, thread v sums value v over the CTA's threads in four
  // interleaved chains (the padded stride puts the 18 readers in distinct
  // banks)
  const HT vals[18] = {h00, h01, h02, h11, h12, h22, A[0], A[1], A[2], A[3], A[4], A[5], A[6], A[7], A[8],
                       b[0], b[1], b[2]};
#pragma unroll
  for (int v = 0; v < 18; ++v) red[v * (kThreads + 1) + tid] = vals[v];
  __syncthreads();
  if (tid < 18) {
    const HT* src = red + tid * (kThreads + 1);
    HT t0 = 0, t1 = 0, t2 = 0, t3 = 0;
#pragma unroll 4
    for (int t = 0; t < kThreads; t += 4) {
      t0 += src[t];
      t1 += src[t + 1];
      t2 += src[t + 2];
      t3 += src[t + 3];
    }
    cpl[(int64_t)blockIdx.x * 32 + tid] = (t0 + t1) + (t2 + t3);
  }
  if constexpr (kFuse) condense_group_tail<double, HT, kMixed, kUpd>(ca, 1e-12);
}

// The same coupling products with one warp per vertex (kWarps vertices per
// CTA, no CTA-wide barrier).  The warp stages U_i and its rows' starts in its
// own slice of shared memory, then splits the support's flattened list of
// upper blocks (rows of S in support order, then row i) evenly over its
// lanes: lane L takes blocks [L c, (L+1) c) with c = ceil(total / 32), walking
// the row boundaries as it goes, so every lane issues about the same number
// of independent block loads.  b = U^T g_C takes the rows round-robin.  The
// 27 sums are reduced by a fixed shuffle tree.
template <typename HT, typename SlotT, bool kMixed, int kUpd, int kWarps>
__global__ void __launch_bounds__(32 * kWarps) k_couple_warp(
    const int32_t* __restrict__ verts, int64_t count, const int32_t* __restrict__ sup_ptr,
    const int32_t* __restrict__ sup_idx, const HT* __restrict__ U, const int32_t* __restrict__ up_ptr,
    const int64_t* __restrict__ smap_ptr, const SlotT* __restrict__ smap, const HT* __restrict__ bsr,
    const double* __restrict__ g64, const float* __restrict__ g_hi, int sup_max, const HT* __restrict__ rot,
    HT* __restrict__ cpl) {
  pdl_entry();
  using Codes = SlotCodes<SlotT>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t k = (int64_t)blockIdx.x * kWarps + warp;
  if (k >= count) return;  // whole warp leaves together
  const size_t per_warp = align16((size_t)sup_max * 9 * sizeof(HT)) + 2 * align16((size_t)(sup_max + 2) * 4);
  unsigned char* ptr = smem + (size_t)warp * per_warp;
  HT* Us = reinterpret_cast<HT*>(ptr);
  ptr += align16((size_t)sup_max * 9 * sizeof(HT));
  int* rstart = reinterpret_cast<int*>(ptr);  // [m + 1] first upper block of each row
  ptr += align16((size_t)(sup_max + 2) * 4);
  int* roff = reinterpret_cast<int*>(ptr);    // [m + 2] offset of each row in the flattened list

  const int i = verts[k];
  const int s0 = sup_ptr[i];
  const int m = sup_ptr[i + 1] - s0;
  const int64_t c0 = smap_ptr[i];
  stage_basis<HT>(Us, U, rot, sup_idx, s0, m, lane, 32);
  // row starts and the exclusive prefix of the row lengths (rows 0..m-1 = S, row m = i)
  int carry = 0;
  for (int base = 0; base <= m; base += 32) {
    const int r = base + lane;
    int len = 0;
    if (r <= m) {
      const int j = r < m ? sup_idx[s0 + r] : i;
      const int a = up_ptr[j];
      rstart[r] = a;
      len = up_ptr[j + 1] - a;
    }
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (r <= m) roff[r] = carry + incl - len;
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) roff[m + 1] = carry;
  __syncwarp();
  const int total = carry;

  HT h00 = 0, h01 = 0, h02 = 0, h11 = 0, h12 = 0, h22 = 0;
  HT A[9], Hii[9], b[3] = {0, 0, 0};
  mat3_zero(A);
  mat3_zero(Hii);
  const int chunk = (total + 31) >> 5;
  int q = lane * chunk;
  const int qend = min(total, q + chunk);
  if (q < qend) {
    // row containing flattened block q: the last r with roff[r] <= q
    int lo = 0, hi = m;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (roff[mid] <= q) lo = mid;
      else hi = mid - 1;
    }
    int r = lo;
    int rend = roff[r + 1];
    for (; q < qend; ++q) {
      while (q >= rend) {
        ++r;
        rend = roff[r + 1];
      }
      const unsigned code = smap[c0 + q];
      if (code == Codes::kNone) continue;
      HT H[9];
      load_block(bsr, (int64_t)rstart[r] + (q - roff[r]), H);
      if (r < m) {
        const HT* Uj = Us + 9 * r;
        if (code == Codes::kSelf) {
          if (kUpd == CC_UPDATE_CC) mat3_tmul_acc(H, Uj, A);
        } else {
          const bool dg = code == Codes::kDiag;
          const HT w = dg ? HT(0.5) : HT(1);
          HT T[9], M[9];
          mat3_zero(T);
          mat3_mul_acc(H, Us + 9 * (dg ? r : (int)code), T);
          mat3_zero(M);
          mat3_tmul_acc(Uj, T, M);
          h00 += 2 * w * M[0]; h11 += 2 * w * M[4]; h22 += 2 * w * M[8];
          h01 += w * (M[1] + M[3]); h02 += w * (M[2] + M[6]); h12 += w * (M[5] + M[7]);
        }
      } else {
        if (code == Codes::kDiag) {
#pragma unroll
          for (int c = 0; c < 9; ++c) Hii[c] = H[c];
        } else if (kUpd == CC_UPDATE_CC) {
          mat3_mul_acc(H, Us + 9 * code, A);
        }
      }
    }
  }
  for (int r = lane; r < m; r += 32) {
    const int j = sup_idx[s0 + r];
    const HT* Uj = Us + 9 * r;
    HT gj[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) gj[a] = kMixed ? (HT)g_hi[3 * (int64_t)j + a] : (HT)g64[3 * (int64_t)j + a];
#pragma unroll
    for (int c = 0; c < 3; ++c) b[c] += Uj[c] * gj[0] + Uj[3 + c] * gj[1] + Uj[6 + c] * gj[2];
  }
  HT vals27[27] = {h00, h01, h02, h11, h12, h22, A[0], A[1], A[2], A[3], A[4], A[5], A[6], A[7], A[8],
                   b[0], b[1], b[2], Hii[0], Hii[1], Hii[2], Hii[3], Hii[4], Hii[5], Hii[6], Hii[7], Hii[8]};
  HT mine = 0;
#pragma unroll
  for (int v = 0; v < 27; ++v) {
    const HT t = warp_sum(vals27[v]);
    if (lane == v) mine = t;
  }
  if (lane < 27) cpl[k * 32 + lane] = mine;
}

template <typename HT>
__host__ __device__ inline size_t warp_smem_bytes(int sup_max, int warps) {
  return (size_t)warps * (align16((size_t)sup_max * 9 * sizeof(HT)) + 2 * align16((size_t)(sup_max + 2) * 4));
}

template <typename HT, bool kMixed, int kUpd, int kThreads>
void launch_couple(Mesh& m, const int32_t* verts, int64_t count, const HT* U, const HT* bsr, const double* g64,
                   const float* g_hi, HT* cpl, const HT* rot, const CondenseArgs<HT>& ca, bool fuse,
                   cudaStream_t s) {
  const int supm = m.sup_max > 0 ? m.sup_max : 1;
  const int64_t smx = m.smap_max > 0 ? m.smap_max : 1;
  const int lanes = m.tune_couple_row_lanes;
  CCG_CHECK(lanes == 1 || lanes == 2 || lanes == 4 || lanes == 8, CC_ERR_STATE, "bad coupling row lanes");
  const int lanes_log2 = lanes == 1 ? 0 : lanes == 2 ? 1 : lanes == 4 ? 2 : 3;
  const size_t smem = cta_smem_bytes<HT>(supm, smx, m.smap_wide ? 2 : 1, kThreads);
  CCG_CHECK(smem <= 220 * 1024, CC_ERR_INVALID_ARG, "support too large for the coupling kernel");
  auto go = [&](auto kern, const auto* smap) {
    set_smem_limit(reinterpret_cast<const void*>(kern), smem);
    pdl_launch(kern, (unsigned)count, kThreads, smem, s, verts, count, (const int32_t*)m.d_sup_ptr.p,
               (const int32_t*)m.d_sup_idx.p, U, (const int32_t*)m.d_up_ptr.p, (const int64_t*)m.d_smap_ptr.p,
               smap, bsr, g64, g_hi, supm, smx, rot, lanes_log2, cpl, ca);
  };
  if (m.smap_wide) {
    if (fuse) go(k_couple<HT, uint16_t, kMixed, kUpd, kThreads, true>, (const uint16_t*)m.d_smap16.p);
    else go(k_couple<HT, uint16_t, kMixed, kUpd, kThreads, false>, (const uint16_t*)m.d_smap16.p);
  } else {
    if (fuse) go(k_couple<HT, uint8_t, kMixed, kUpd, kThreads, true>, (const uint8_t*)m.d_smap8.p);
    else go(k_couple<HT, uint8_t, kMixed, kUpd, kThreads, false>, (const uint8_t*)m.d_smap8.p);
  }
  CCG_CUDA(cudaGetLastError());
}

template <typename HT, bool kMixed, int kUpd>
void launch_couple_warp(Mesh& m, const int32_t* verts, int64_t count, const HT* U, const HT* bsr, const double* g64,
                        const float* g_hi, HT* cpl, const HT* rot, cudaStream_t s) {
  constexpr int kWarps = 4;
  const int supm = m.sup_max > 0 ? m.sup_max : 1;
  const size_t smem = warp_smem_bytes<HT>(supm, kWarps);
  CCG_CHECK(smem <= 220 * 1024, CC_ERR_INVALID_ARG, "support too large for the coupling kernel");
  const unsigned grid = (unsigned)((count + kWarps - 1) / kWarps);
  if (m.smap_wide) {
    auto kern = k_couple_warp<HT, uint16_t, kMixed, kUpd, kWarps>;
    set_smem_limit(reinterpret_cast<const void*>(kern), smem);
    pdl_launch(kern, grid, 32 * kWarps, smem, s, verts, count, (const int32_t*)m.d_sup_ptr.p,
               (const int32_t*)m.d_sup_idx.p, U, (const int32_t*)m.d_up_ptr.p, (const int64_t*)m.d_smap_ptr.p,
               (const uint16_t*)m.d_smap16.p, bsr, g64, g_hi, supm, rot, cpl);
  } else {
    auto kern = k_couple_warp<HT, uint8_t, kMixed, kUpd, kWarps>;
    set_smem_limit(reinterpret_cast<const void*>(kern), smem);
    pdl_launch(kern, grid, 32 * kWarps, smem, s, verts, count, (const int32_t*)m.d_sup_ptr.p,
               (const int32_t*)m.d_sup_idx.p, U, (const int32_t*)m.d_up_ptr.p, (const int64_t*)m.d_smap_ptr.p,
               (const uint8_t*)m.d_smap8.p, bsr, g64, g_hi, supm, rot, cpl);
  }
  CCG_CUDA(cudaGetLastError());
}

template <typename HT, bool kMixed, int kUpd>
void launch_one(Mesh& m, const int32_t* verts, int64_t count, const HT* U, const HT* bsr, const double* g64,
                const float* g_hi, const float* g_lo, HT* cpl, double* x, SweepCounters c, cudaStream_t s) {
  const CondenseArgs<HT> ca{verts, count, cpl, (const int32_t*)m.d_sup_ptr.p, (const int32_t*)m.d_up_ptr.p, bsr,
                            g64, g_hi, g_lo, m.n, x, kMixed ? m.mx.x_hi.p : nullptr, kMixed ? m.mx.x_lo.p : nullptr,
                            (const int32_t*)m.d_vert_mesh.p, (const int32_t*)m.d_mesh_active.p, c.fallback, c.error,
                            m.d_grp_cnt.p};
  // the coupling CTAs condense their vertices themselves (last of every 32),
  // except with the one-warp coupling kernel or when switched off
  const bool fuse = fused_local_solve(m, (cc_update)kUpd);
  CCG_CHECK(!fuse || (int64_t)m.d_grp_cnt.count >= (count + 31) / 32, CC_ERR_STATE, "group counters missing");
  const CondenseArgs<HT>& cf = ca;
  if (kUpd != CC_UPDATE_CD) {
    const HT* rot = nullptr;
    if (m.rot_active) {
      if constexpr (kMixed) rot = reinterpret_cast<const HT*>(m.mx.rot.p);
      else rot = reinterpret_cast<const HT*>(m.f64.rot.p);
    }
    switch (m.tune_couple_threads) {
      case 32: launch_couple_warp<HT, kMixed, kUpd>(m, verts, count, U, bsr, g64, g_hi, cpl, rot, s); break;
      case 64: launch_couple<HT, kMixed, kUpd, 64>(m, verts, count, U, bsr, g64, g_hi, cpl, rot, cf, fuse, s); break;
      case 256: launch_couple<HT, kMixed, kUpd, 256>(m, verts, count, U, bsr, g64, g_hi, cpl, rot, cf, fuse, s); break;
      default: launch_couple<HT, kMixed, kUpd, 128>(m, verts, count, U, bsr, g64, g_hi, cpl, rot, cf, fuse, s);
    }
  }
  if (fuse) return;
  // float64 condensation of the coupling products (the 3x3 Schur solves of
  // Eq. 11-12 stay in float64 in both precisions), one vertex per thread in
  // 32-thread blocks: a colour holds a few thousand vertices, so small blocks
  // spread the long per-vertex chains over every SM
  constexpr int kCondenseThreads = 32;
  const unsigned grid = (unsigned)((count + kCondenseThreads - 1) / kCondenseThreads);
  pdl_launch(k_condense<double, HT, kMixed, kUpd>, grid, kCondenseThreads, 0, s, ca, 1e-12);
  CCG_CUDA(cudaGetLastError());
}

}  // namespace

namespace {

// Per-vertex rotations of corotated bases (Sec. 3.1), one thread per vertex:
// F_j = A_j C_j^{-1} with A_j = sum over the 1-ring (ascending) of
// (x_l - x_j)(X_l - X_j)^T and C_j = sum of (X_l - X_j)(X_l - X_j)^T (the
// neighbourhood's least-squares deformation gradient, exact for homogeneous
// deformations); R_j = orthogonal polar factor of F_j by Newton's iteration
// Y <- (g Y + (g Y)^{-T}) / 2 with Higham's scaling g = sqrt(|Y^{-1}|_F / |Y|_F),
// stopped when the update is below 64 units of roundoff of T (at most 40
// steps); R_j = I when det F_j <= 0.  The sums are float64; the iteration
// runs in T (float64 for the plain path, float32 for the mixed one).
template <typename T>
__device__ __forceinline__ T inv3(const T* a, T* o) {  // o = a^{-1}, returns det a
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

template <typename T>
__global__ void k_rotations(int64_t n, const int32_t* __restrict__ nbr_ptr, const int32_t* __restrict__ nbr_idx,
                            const double* __restrict__ x, const double* __restrict__ X, T* __restrict__ R) {
  pdl_entry();
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  double A[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, C[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const double xj[3] = {x[j], x[n + j], x[2 * n + j]}, Xj[3] = {X[j], X[n + j], X[2 * n + j]};
  const int p0 = nbr_ptr[j], p1 = nbr_ptr[j + 1];
  for (int p = p0; p < p1; ++p) {
    const int l = nbr_idx[p];
    const double dx[3] = {x[l] - xj[0], x[n + l] - xj[1], x[2 * n + l] - xj[2]};
    const double dX[3] = {X[l] - Xj[0], X[n + l] - Xj[1], X[2 * n + l] - Xj[2]};
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        A[3 * r + c] = fma(dx[r], dX[c], A[3 * r + c]);
        C[3 * r + c] = fma(dX[r], dX[c], C[3 * r + c]);
      }
  }
  T out[9] = {T(1), T(0), T(0), T(0), T(1), T(0), T(0), T(0), T(1)};
  double Ci[9];
  if (p1 > p0 && inv3(C, Ci) > 0.0) {
    T Y[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) Y[3 * r + c] = (T)(A[3 * r] * Ci[c] + A[3 * r + 1] * Ci[3 + c] + A[3 * r + 2] * Ci[6 + c]);
    T Yi[9];
    if (inv3(Y, Yi) > T(0)) {
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
            const T v = T(0.5) * (g * Y[3 * r + c] + Yi[3 * c + r] / g);  // (g Y + (g Y)^{-T}) / 2
            dn += (v - Y[3 * r + c]) * (v - Y[3 * r + c]);
            yn += v * v;
            Y[3 * r + c] = v;
          }
        if (dn <= tol * tol * yn) break;
        inv3(Y, Yi);
      }
#pragma unroll
      for (int q = 0; q < 9; ++q) out[q] = Y[q];
    }
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) R[9 * j + q] = out[q];
}

}  // namespace

void launch_rotations(Mesh& m, const double* x, bool mixed, cudaStream_t s) {
  if (!m.d_Xrest.p) {
    std::vector<double> soa(3 * m.n);
    for (int64_t j = 0; j < m.n; ++j)
      for (int a = 0; a < 3; ++a) soa[a * m.n + j] = m.X[3 * j + a];
    m.d_Xrest.upload(soa, s);
  }
  const unsigned grid = (unsigned)((m.n + 127) / 128);
  if (mixed) {
    if (!m.mx.rot.p) m.mx.rot.alloc(9 * m.n);
    pdl_launch(k_rotations<float>, grid, 128, 0, s, m.n, (const int32_t*)m.d_nbr_ptr.p, (const int32_t*)m.d_nbr_idx.p,
               x, (const double*)m.d_Xrest.p, m.mx.rot.p);
  } else {
    if (!m.f64.rot.p) m.f64.rot.alloc(9 * m.n);
    pdl_launch(k_rotations<double>, grid, 128, 0, s, m.n, (const int32_t*)m.d_nbr_ptr.p,
               (const int32_t*)m.d_nbr_idx.p, x, (const double*)m.d_Xrest.p, m.f64.rot.p);
  }
}

void launch_local_solve_f64(Mesh& m, cc_update upd, const int32_t* verts, int64_t count, double* x,
                            SweepCounters c, cudaStream_t s) {
  if (count <= 0) return;
  double* cpl = m.f64.cpl.p;
  switch (upd) {
    case CC_UPDATE_CC:
      launch_one<double, false, CC_UPDATE_CC>(m, verts, count, m.f64.U.p, m.f64.bsr.p, m.f64.g.p, nullptr, nullptr, cpl, x, c, s);
      break;
    case CC_UPDATE_CD:
      launch_one<double, false, CC_UPDATE_CD>(m, verts, count, m.f64.U.p, m.f64.bsr.p, m.f64.g.p, nullptr, nullptr, cpl, x, c, s);
      break;
    default:
      launch_one<double, false, CC_UPDATE_JGS2>(m, verts, count, m.f64.U.p, m.f64.bsr.p, m.f64.g.p, nullptr, nullptr, cpl, x, c, s);
  }
}

void launch_local_solve_mixed(Mesh& m, cc_update upd, const int32_t* verts, int64_t count, double* x,
                              SweepCounters c, cudaStream_t s) {
  if (count <= 0) return;
  float* cpl = m.mx.cpl.p;
  switch (upd) {
    case CC_UPDATE_CC:
      launch_one<float, true, CC_UPDATE_CC>(m, verts, count, m.mx.U.p, m.mx.bsr.p, nullptr, m.mx.g_hi.p, m.mx.g_lo.p, cpl, x, c, s);
      break;
    case CC_UPDATE_CD:
      launch_one<float, true, CC_UPDATE_CD>(m, verts, count, m.mx.U.p, m.mx.bsr.p, nullptr, m.mx.g_hi.p, m.mx.g_lo.p, cpl, x, c, s);
      break;
    default:
      launch_one<float, true, CC_UPDATE_JGS2>(m, verts, count, m.mx.U.p, m.mx.bsr.p, nullptr, m.mx.g_hi.p, m.mx.g_lo.p, cpl, x, c, s);
  }
}

}  // namespace ccg
