// BF16 tensor-core GEMM for the learned-subspace MLP on sm_103a:
//   C[M x N] = A[M x K] . B[N x K]^T      (A, B row-major, K contiguous)
// Tiles of A (128 x 64) and B (BN x 64) are loaded by TMA with 128-byte
// swizzle into 1024-byte aligned shared memory; one thread issues
// tcgen05.mma (kind::f16, BF16 inputs, FP32 accumulator in tensor memory),
// four K=16 steps per 64-wide tile, and commits to an mbarrier; a two-stage
// ring overlaps the next tile's TMA with the current MMAs.  The epilogue
// moves the accumulator out of tensor memory with tcgen05.ld (warp w owns
// rows 32w..32w+31) and applies one of the fused epilogues below.
// Every mbarrier wait is bounded (about one second of %globaltimer): on
// expiry the kernel records an error, releases its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "cc_internal.cuh"
#include "mlp.cuh"

namespace ccg {
namespace {

constexpr int kBM = 128, kBK = 64, kStages = 2;
constexpr uint64_t kWaitLimitNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Returns false when the phase did not complete within about one second.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = smem_u32(bar);
  const uint64_t t0 = global_ns();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > kWaitLimitNs) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major tile, rows of 128 bytes, 128-byte
// swizzle, 8-row groups 1024 bytes apart (stride byte offset), version 1.
__device__ __forceinline__ uint64_t smem_desc_sw128(const void* base) {
  const uint64_t addr = smem_u32(base);
  uint64_t d = 0;
  d |= (addr >> 4) & 0x3FFFull;            // start address
  d |= (uint64_t)(16 >> 4) << 16;          // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset
  d |= 1ull << 46;                         // descriptor version
  d |= 2ull << 61;                         // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t instr_desc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

template <int BN, int EPI>
__global__ void __launch_bounds__(128) k_gemm_tn(const __grid_constant__ CUtensorMap mapA,
                                                 const __grid_constant__ CUtensorMap mapB, int M, int N, int K,
                                                 int kt_per_split, GemmEpilogue ep, int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte alignment of the tile ring (128-byte swizzle atoms)
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int kABytes = kBM * kBK * 2, kBBytes = BN * kBK * 2;
  uint8_t* tileA[kStages];
  uint8_t* tileB[kStages];
#pragma unroll
  for (int s = 0; s < kStages; ++s) {
    tileA[s] = smem + s * (kABytes + kBBytes);
    tileB[s] = tileA[s] + kABytes;
  }
  __shared__ __align__(8) uint64_t bar_full[kStages];
  __shared__ __align__(8) uint64_t bar_done[kStages];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int failed;
  constexpr uint32_t kCols = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
  // this split's K tiles: [kt0, kt0 + ktiles)
  const int kt_all = (K + kBK - 1) / kBK;
  const int kt0 = blockIdx.z * kt_per_split;
  const int ktiles = max(0, min(kt_all - kt0, kt_per_split));

  if (threadIdx.x == 0) {
    failed = 0;
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&bar_full[s], 1);
      mbar_init(&bar_done[s], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;
  constexpr uint32_t idesc = instr_desc_bf16(BN);

  if (threadIdx.x == 0) {
    // prologue: fill the ring
    for (int s = 0; s < kStages && s < ktiles; ++s) {
      mbar_expect_tx(&bar_full[s], kABytes + kBBytes);
      tma_load_2d(tileA[s], &mapA, &bar_full[s], (kt0 + s) * kBK, m0);
      tma_load_2d(tileB[s], &mapB, &bar_full[s], (kt0 + s) * kBK, n0);
    }
    for (int kt = 0; kt < ktiles; ++kt) {
      const int s = kt % kStages;
      const uint32_t ph = (kt / kStages) & 1;
      if (!mbar_wait(&bar_full[s], ph)) {
        failed = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t ad = smem_desc_sw128(tileA[s]), bd = smem_desc_sw128(tileB[s]);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk)  // 16 BF16 = 32 bytes = 2 descriptor units per step
        mma_bf16(tmem, ad + 2 * kk, bd + 2 * kk, idesc, (kt > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&bar_done[s]);
      const int nk = kt + kStages;
      if (nk < ktiles) {
        // the stage is reused once its MMAs have read it
        if (!mbar_wait(&bar_done[s], ph)) {
          failed = 1;
          break;
        }
        mbar_expect_tx(&bar_full[s], kABytes + kBBytes);
        tma_load_2d(tileA[s], &mapA, &bar_full[s], (kt0 + nk) * kBK, m0);
        tma_load_2d(tileB[s], &mapB, &bar_full[s], (kt0 + nk) * kBK, n0);
      }
    }
  }
  __syncthreads();
  // all MMAs done: wait on the last tile's commit (covers every earlier MMA)
  bool ok = failed == 0;
  if (ok && ktiles > 0) {
    const int last = ktiles - 1;
    ok = mbar_wait(&bar_done[last % kStages], (last / kStages) & 1);
  }
  ok = __syncthreads_and(ok) != 0;  // the epilogue's tensor-memory loads are warp-collective
  if (!ok && threadIdx.x == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  if (ok) {
    const int row = m0 + warp * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    float* c32 = ep.c32;
    if (EPI == kEpiF32 && c32) c32 += (int64_t)blockIdx.z * ep.split_stride;
#pragma unroll 1
    for (int c = 0; c < BN; c += 16) {
      float v[16];
      tmem_ld16(lane_base + c, v);
      if (row >= M) continue;
      const int col0 = n0 + c;
      if (col0 >= N) continue;
      const bool full = col0 + 16 <= N;
      if (EPI == kEpiF32 || EPI == kEpiBiasF32) {
        if (EPI == kEpiBiasF32) {
#pragma unroll
          for (int k = 0; k < 16; ++k) v[k] += (col0 + k < N) ? ep.bias[col0 + k] : 0.0f;
        }
        float* dst = c32 + (int64_t)row * ep.ldc + col0;
        if (full && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
#pragma unroll
          for (int k = 0; k < 16; k += 4) *reinterpret_cast<float4*>(dst + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
        } else {
          for (int k = 0; k < 16 && col0 + k < N; ++k) dst[k] = v[k];
        }
        continue;
      }
      __nv_bfloat16 hb[16];
      if (EPI == kEpiBiasGelu) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const float z = v[k] + ((col0 + k < N) ? ep.bias[col0 + k] : 0.0f);
          v[k] = z;
          hb[k] = __float2bfloat16_rn(gelu(z));
        }
        if (ep.z32) {  // pre-activations are kept for training only
          float* zdst = ep.z32 + (int64_t)row * ep.ldz + col0;
          if (full && ((reinterpret_cast<uintptr_t>(zdst) & 15) == 0)) {
#pragma unroll
            for (int k = 0; k < 16; k += 4)
              *reinterpret_cast<float4*>(zdst + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
          } else {
            for (int k = 0; k < 16 && col0 + k < N; ++k) zdst[k] = v[k];
          }
        }
      } else {  // kEpiGeluGrad: dZ = C * gelu'(Z)
        const float* zsrc = ep.z32 + (int64_t)row * ep.ldz + col0;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const float z = (col0 + k < N) ? zsrc[k] : 0.0f;
          hb[k] = __float2bfloat16_rn(v[k] * gelu_grad(z));
        }
      }
      __nv_bfloat16* hdst = ep.h16 + (int64_t)row * ep.ldh + col0;
      if (full && ((reinterpret_cast<uintptr_t>(hdst) & 15) == 0)) {
        uint4 w[2];
        memcpy(w, hb, sizeof(w));
        reinterpret_cast<uint4*>(hdst)[0] = w[0];
        reinterpret_cast<uint4*>(hdst)[1] = w[1];
      } else {
        for (int k = 0; k < 16 && col0 + k < N; ++k) hdst[k] = hb[k];
      }
      if (ep.ht16) {
        // transposed copy: consecutive lanes write consecutive rows
        for (int k = 0; k < 16 && col0 + k < N; ++k) ep.ht16[(int64_t)(col0 + k) * ep.ldt + row] = hb[k];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
  }
}

// ---- host side ----------------------------------------------------------------
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    CCG_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    CCG_CHECK(p && q == cudaDriverEntryPointSuccess, CC_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// Tensor map of a row-major BF16 matrix [rows x cols] with leading dimension
// ld (elements, multiple of 8), box [box_rows x 64], 128-byte swizzle, zero
// fill outside the matrix.
CUtensorMap make_map(const void* ptr, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  CCG_CHECK((reinterpret_cast<uintptr_t>(ptr) & 15) == 0, CC_ERR_INVALID_ARG, "GEMM operand not 16-byte aligned");
  CCG_CHECK(ld % 8 == 0 && ld >= cols, CC_ERR_INVALID_ARG, "GEMM leading dimension must be a multiple of 8");
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1u, 1u};
  const CUresult r = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box,
                                 es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CCG_CHECK(r == CUDA_SUCCESS, CC_ERR_CUDA, "cuTensorMapEncodeTiled failed");
  return map;
}

template <int BN, int EPI>
void launch_bn(const CUtensorMap& a, const CUtensorMap& b, int M, int N, int K, int splits, const GemmEpilogue& ep,
               int* err, cudaStream_t s) {
  const size_t smem = (size_t)kStages * (kBM * kBK * 2 + BN * kBK * 2) + 1024;
  auto kern = k_gemm_tn<BN, EPI>;
  set_smem_limit(reinterpret_cast<const void*>(kern), smem);
  const int kt_all = (K + kBK - 1) / kBK;
  const int per = (kt_all + splits - 1) / splits;
  const int z = (kt_all + per - 1) / per;  // every split gets at least one K tile
  const dim3 grid((unsigned)((M + kBM - 1) / kBM), (unsigned)((N + BN - 1) / BN), (unsigned)z);
  kern<<<grid, 128, smem, s>>>(a, b, M, N, K, per, ep, err);
  CCG_CUDA(cudaGetLastError());
}

template <int EPI>
void launch_epi(const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N, int K, GemmShape sh,
                const GemmEpilogue& ep, int* err, cudaStream_t s) {
  const CUtensorMap ma = make_map(A, M, K, lda, kBM);
  switch (sh.bn) {
    case 64: launch_bn<64, EPI>(ma, make_map(B, N, K, ldb, 64), M, N, K, sh.splits, ep, err, s); break;
    case 128: launch_bn<128, EPI>(ma, make_map(B, N, K, ldb, 128), M, N, K, sh.splits, ep, err, s); break;
    case 192: launch_bn<192, EPI>(ma, make_map(B, N, K, ldb, 192), M, N, K, sh.splits, ep, err, s); break;
    default: launch_bn<256, EPI>(ma, make_map(B, N, K, ldb, 256), M, N, K, sh.splits, ep, err, s); break;
  }
}

}  // namespace

GemmShape gemm_pick_shape(int M, int N, int K, bool allow_split) {
  constexpr int kSlots = 2 * 152;  // about two resident CTAs per SM
  GemmShape sh;
  const int mt = (M + kBM - 1) / kBM;
  const int cands[4] = {256, 192, 128, 64};
  sh.bn = 64;
  for (int bn : cands) {
    if (N % bn != 0 && bn != 64) continue;
    if ((int64_t)mt * ((N + bn - 1) / bn) >= kSlots || allow_split) {
      sh.bn = bn;
      break;
    }
  }
  if (allow_split) {
    const int tiles = mt * ((N + sh.bn - 1) / sh.bn);
    const int kt = (K + kBK - 1) / kBK;
    const int want = (kSlots + tiles - 1) / tiles;
    sh.splits = std::max(1, std::min(want, kt / 4));
  }
  return sh;
}

void gemm_tn(const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N, int K, int epi,
             const GemmEpilogue& ep, int* err, cudaStream_t s, GemmShape sh) {
  CCG_CHECK(M > 0 && N > 0 && K > 0, CC_ERR_INVALID_ARG, "GEMM sizes must be positive");
  CCG_CHECK(sh.bn == 64 || sh.bn == 128 || sh.bn == 192 || sh.bn == 256, CC_ERR_INVALID_ARG, "bad GEMM N tile");
  CCG_CHECK(sh.splits >= 1 && (sh.splits == 1 || epi == kEpiF32), CC_ERR_INVALID_ARG,
            "split K needs the float32 epilogue");
  // every buffer an epilogue writes or reads must be present
  const bool f32 = epi == kEpiF32 || epi == kEpiBiasF32;
  CCG_CHECK(!f32 || (ep.c32 && ep.ldc >= N), CC_ERR_INVALID_ARG, "GEMM epilogue: missing float32 output");
  CCG_CHECK(!(epi == kEpiBiasF32 || epi == kEpiBiasGelu) || ep.bias, CC_ERR_INVALID_ARG, "GEMM epilogue: missing bias");
  CCG_CHECK(f32 || (ep.h16 && ep.ldh >= N), CC_ERR_INVALID_ARG, "GEMM epilogue: missing BF16 output");
  CCG_CHECK(epi != kEpiGeluGrad || (ep.z32 && ep.ldz >= N), CC_ERR_INVALID_ARG,
            "GEMM epilogue: missing pre-activations");
  CCG_CHECK(!ep.z32 || ep.ldz >= N, CC_ERR_INVALID_ARG, "GEMM epilogue: bad pre-activation stride");
  CCG_CHECK(!ep.ht16 || ep.ldt >= M, CC_ERR_INVALID_ARG, "GEMM epilogue: transposed copy too narrow");
  switch (epi) {
    case kEpiF32: launch_epi<kEpiF32>(A, lda, B, ldb, M, N, K, sh, ep, err, s); break;
    case kEpiBiasF32: launch_epi<kEpiBiasF32>(A, lda, B, ldb, M, N, K, sh, ep, err, s); break;
    case kEpiBiasGelu: launch_epi<kEpiBiasGelu>(A, lda, B, ldb, M, N, K, sh, ep, err, s); break;
    default: launch_epi<kEpiGeluGrad>(A, lda, B, ldb, M, N, K, sh, ep, err, s); break;
  }
}

}  // namespace ccg
