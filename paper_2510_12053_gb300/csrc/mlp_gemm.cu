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

// Accumulator fragment for stores along rows, 32 lanes x 16 columns by two
// 16x256b.x2 loads: in each 16-lane half, thread t holds lanes t/4 (v[0..1],
// v[4..5]) and t/4 + 8 (v[2..3], v[6..7]) at columns 2 (t % 4) + {0, 1}
// (v[0..3]) and 8 + 2 (t % 4) + {0, 1} (v[4..7]), so four consecutive
// threads hold 32 contiguous bytes of a row; v[0..7] lanes 0..15, v[8..15]
// lanes 16..31; one wait for both loads.
__device__ __forceinline__ void tmem_ld_rows32(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile("tcgen05.ld.sync.aligned.16x256b.x2.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.ld.sync.aligned.16x256b.x2.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                 "=r"(r[15])
               : "r"(taddr + (16u << 16)));
  // the wait names the registers (in-out), so nothing reads them before it
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15])
               :
               : "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

}  // namespace

// Hardware approximations (flush to zero): reciprocal and 2^x.
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float exp2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// erfc(u) / 2 for u >= 0 by Abramowitz and Stegun, Handbook of Mathematical
// Functions (1964), formula 7.1.26 (Hastings' rational approximation):
//   erf(u) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-u^2),
//   t = 1 / (1 + p u), |error| <= 1.5e-7,
// with the a_k halved (exact in binary), and exp(-u^2) = 2^(-u^2 log2 e).
// Branch-free: one reciprocal, one exponential, five FMAs.  Its error is ~1e-4
// of a BF16 rounding step, where the activations it feeds are stored.  The
// operations are the non-contracting _rn forms, one per step, so the
// two-wide version below (fp32x2 instructions) gives the same bits.
constexpr float kAsP = 0.3275911f, kAsA5 = 0.5307027145f, kAsA4 = -0.7265760135f, kAsA3 = 0.7107068705f,
                kAsA2 = -0.142248368f, kAsA1 = 0.127414796f, kNegLog2e = -1.4426950408889634f,
                kRsqrt2 = 0.70710678118654752f;

struct HalfErfc {
  float h;  // erfc(u) / 2
  float e;  // exp(-u^2)
};

__device__ __forceinline__ HalfErfc half_erfc_as7126(float u) {
  const float t = rcp_approx(__fmaf_rn(kAsP, u, 1.0f));
  float q = __fmaf_rn(t, kAsA5, kAsA4);
  q = __fmaf_rn(t, q, kAsA3);
  q = __fmaf_rn(t, q, kAsA2);
  q = __fmaf_rn(t, q, kAsA1);
  const float e = exp2_approx(__fmul_rn(u, __fmul_rn(u, kNegLog2e)));
  return {__fmul_rn(__fmul_rn(q, t), e), e};
}

// erf(x) = sign(x) (1 - erfc(|x|))
__device__ __forceinline__ float erf_as7126(float x) {
  return copysignf(fmaf(-2.0f, half_erfc_as7126(fabsf(x)).h, 1.0f), x);
}

namespace {

// GELU, erf form: z Phi(z), Phi(z) = (1 + erf(z / sqrt 2)) / 2, i.e.
// 1 - h for z >= 0 and h below, h = erfc(|z| / sqrt 2) / 2; written
// branch-free as z / 2 + |z| (1/2 - h).  Its derivative Phi(z) + z phi(z),
// phi(z) = exp(-z^2 / 2) / sqrt(2 pi).
__device__ __forceinline__ float gelu(float z) {
  const float az = fabsf(z);
  const float h = half_erfc_as7126(__fmul_rn(az, kRsqrt2)).h;
  return __fmaf_rn(az, __fadd_rn(0.5f, -h), __fmul_rn(0.5f, z));
}

// gelu of two values with fp32x2 instructions (the MUFU steps stay scalar):
// the same operations as gelu(), so the same bits
__device__ __forceinline__ float2 gelu2(float2 z) {
  const float2 az = make_float2(fabsf(z.x), fabsf(z.y));
  const float2 u = __fmul2_rn(az, make_float2(kRsqrt2, kRsqrt2));
  const float2 d = __ffma2_rn(make_float2(kAsP, kAsP), u, make_float2(1.0f, 1.0f));
  const float2 t = make_float2(rcp_approx(d.x), rcp_approx(d.y));
  float2 q = __ffma2_rn(t, make_float2(kAsA5, kAsA5), make_float2(kAsA4, kAsA4));
  q = __ffma2_rn(t, q, make_float2(kAsA3, kAsA3));
  q = __ffma2_rn(t, q, make_float2(kAsA2, kAsA2));
  q = __ffma2_rn(t, q, make_float2(kAsA1, kAsA1));
  const float2 w = __fmul2_rn(u, __fmul2_rn(u, make_float2(kNegLog2e, kNegLog2e)));
  const float2 e = make_float2(exp2_approx(w.x), exp2_approx(w.y));
  const float2 h = __fmul2_rn(__fmul2_rn(q, t), e);
  return __ffma2_rn(az, __fadd2_rn(make_float2(0.5f, 0.5f), make_float2(-h.x, -h.y)),
                    __fmul2_rn(make_float2(0.5f, 0.5f), z));
}

__device__ __forceinline__ float gelu_grad(float z) {
  const HalfErfc r = half_erfc_as7126(fabsf(z) * kRsqrt2);
  return (z >= 0.0f ? 1.0f - r.h : r.h) + z * 0.39894228040143268f * r.e;
}

__global__ void k_erf_check(const float* __restrict__ x, int n, float* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) {
    out[3 * k] = erf_as7126(x[k]);
    out[3 * k + 1] = gelu(x[k]);
    out[3 * k + 2] = gelu_grad(x[k]);
  }
}

__device__ __forceinline__ bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

__device__ __forceinline__ void load16(const float* src, float (&d)[16]) {
#pragma unroll
  for (int k = 0; k < 16; k += 4) {
    const float4 q = *reinterpret_cast<const float4*>(src + k);
    d[k] = q.x; d[k + 1] = q.y; d[k + 2] = q.z; d[k + 3] = q.w;
  }
}

__device__ __forceinline__ void store16(float* dst, const float (&v)[16]) {
#pragma unroll
  for (int k = 0; k < 16; k += 4) *reinterpret_cast<float4*>(dst + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
}

// 16 float32 values -> 16 BF16 (round to nearest even), two per conversion
__device__ __forceinline__ void store16_bf16(__nv_bfloat16* dst, const float (&g)[16]) {
  uint32_t w[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const __nv_bfloat162 p2 = __floats2bfloat162_rn(g[2 * k], g[2 * k + 1]);
    w[k] = *reinterpret_cast<const uint32_t*>(&p2);
  }
  reinterpret_cast<uint4*>(dst)[0] = make_uint4(w[0], w[1], w[2], w[3]);
  reinterpret_cast<uint4*>(dst)[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

// Epilogue of 16 accumulator columns [col0, col0 + 16) of one row.  Full,
// aligned chunks take vector loads and stores with no per-column checks.
template <int EPI>
__device__ __forceinline__ void epilogue_chunk(float (&v)[16], int row, int col0, int N, const GemmEpilogue& ep,
                                               float* c32) {
  const bool full = col0 + 16 <= N;
  if (EPI == kEpiF32 || EPI == kEpiBiasF32) {
    float* dst = c32 + (int64_t)row * ep.ldc + col0;
    if (full && aligned16(dst) && (EPI == kEpiF32 || aligned16(ep.bias + col0))) {
      if (EPI == kEpiBiasF32) {
        float b[16];
        load16(ep.bias + col0, b);
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] += b[k];
      }
      store16(dst, v);
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k)
        if (col0 + k < N) dst[k] = v[k] + (EPI == kEpiBiasF32 ? ep.bias[col0 + k] : 0.0f);
    }
    return;
  }
  float g[16];
  __nv_bfloat16* hdst = ep.h16 + (int64_t)row * ep.ldh + col0;
  if (EPI == kEpiBiasGelu) {
    float* zdst = ep.z32 ? ep.z32 + (int64_t)row * ep.ldz + col0 : nullptr;
    if (full && aligned16(ep.bias + col0) && aligned16(hdst) && (!zdst || aligned16(zdst))) {
      float b[16];
      load16(ep.bias + col0, b);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        v[k] += b[k];
        g[k] = gelu(v[k]);
      }
      if (zdst) store16(zdst, v);  // pre-activations are kept for training only
      store16_bf16(hdst, g);
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        if (col0 + k < N) {
          const float z = v[k] + ep.bias[col0 + k];
          g[k] = gelu(z);
          if (zdst) zdst[k] = z;
          hdst[k] = __float2bfloat16_rn(g[k]);
        } else {
          g[k] = 0.0f;
        }
      }
    }
  } else {  // kEpiGeluGrad: dZ = C * gelu'(Z)
    const float* zsrc = ep.z32 + (int64_t)row * ep.ldz + col0;
    if (full && aligned16(zsrc) && aligned16(hdst)) {
      float z[16];
      load16(zsrc, z);
#pragma unroll
      for (int k = 0; k < 16; ++k) g[k] = v[k] * gelu_grad(z[k]);
      store16_bf16(hdst, g);
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        if (col0 + k < N) {
          g[k] = v[k] * gelu_grad(zsrc[k]);
          hdst[k] = __float2bfloat16_rn(g[k]);
        } else {
          g[k] = 0.0f;
        }
      }
    }
  }
  if (ep.ht16) {
    // transposed copy: consecutive lanes write consecutive rows
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (col0 + k < N) ep.ht16[(int64_t)(col0 + k) * ep.ldt + row] = __float2bfloat16_rn(g[k]);
  }
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
      if (row >= M || n0 + c >= N) continue;
      epilogue_chunk<EPI>(v, row, n0 + c, N, ep, c32);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
  }
}

// ---- persistent, warp-specialised version --------------------------------------
// One CTA per SM loops over output tiles (and K splits).  Warp 0 (one thread)
// is the TMA producer of a kWsStages-deep ring of A/B tiles; warp 1 (one
// thread) issues the tcgen05 MMAs into one of two accumulators in tensor
// memory (2 x 256 columns = the SM's 512); warps 2..17 are the epilogue, four
// per tensor-memory lane quarter (warp w reads lanes 32 (w % 4) ..), each
// owning a quarter of the tile's columns.  While the epilogue drains
// accumulator a, the MMAs of the next tile fill accumulator a ^ 1.
//   full[s]      producer -> MMA: stage s loaded (TMA transaction bytes)
//   empty[s]     MMA -> producer: stage s read (tcgen05.commit)
//   acc_full[a]  MMA -> epilogue: accumulator a complete (tcgen05.commit)
//   acc_empty[a] epilogue -> MMA: accumulator a drained (one arrival per warp)
// Every wait is bounded; a role that times out raises the CTA's failure flag,
// the others stop at their next wait, in-flight copies and MMAs are waited
// for (bounded) and tensor memory is freed before the CTA returns.
constexpr int kWsEpiWarps = 16;
constexpr int kWsThreads = 32 * (2 + kWsEpiWarps);
constexpr int kWsAccCols = 256;

__host__ __device__ constexpr int ws_stages(int bn) {
  return (200 * 1024) / (kBM * kBK * 2 + bn * kBK * 2) > 8 ? 8 : (200 * 1024) / (kBM * kBK * 2 + bn * kBK * 2);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <int BN, int EPI>
__global__ void __launch_bounds__(kWsThreads, 1) k_gemm_ws(const __grid_constant__ CUtensorMap mapA,
                                                           const __grid_constant__ CUtensorMap mapB, int M, int N,
                                                           int K, int kt_per_split, int splits, GemmEpilogue ep,
                                                           int* __restrict__ err) {
  constexpr int S = ws_stages(BN);
  constexpr int kABytes = kBM * kBK * 2, kBBytes = BN * kBK * 2;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full[S], empty[S], acc_full[2], acc_empty[2], mma_done;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int failed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = (M + kBM - 1) / kBM, nt = (N + BN - 1) / BN;
  const int kt_all = (K + kBK - 1) / kBK;
  const int tiles = mt * nt * splits;

  if (threadIdx.x == 0) {
    failed = 0;
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], kWsEpiWarps);
    }
    mbar_init(&mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(2 * kWsAccCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0 && lane == 0) {
    // ---- producer ----
    int it = 0;
    for (int t = blockIdx.x; t < tiles && !failed; t += gridDim.x) {
      const int z = t % splits, tn = (t / splits) % nt, tm = t / (splits * nt);
      const int kt0 = z * kt_per_split, nk = min(kt_all - kt0, kt_per_split);
      for (int kk = 0; kk < nk; ++kk, ++it) {
        const int s = it % S;
        const uint32_t ph = (uint32_t)(it / S) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u)) {
          failed = 1;
          break;
        }
        uint8_t* a = smem + s * (kABytes + kBBytes);
        mbar_expect_tx(&full[s], kABytes + kBBytes);
        tma_load_2d(a, &mapA, &full[s], (kt0 + kk) * kBK, tm * kBM);
        tma_load_2d(a + kABytes, &mapB, &full[s], (kt0 + kk) * kBK, tn * BN);
      }
    }
    // copies still in flight complete before the CTA can exit: the last load
    // of every stage is consumed by the MMA thread or waited for here
    if (failed) {
      for (int q = max(0, it - S); q < it; ++q) mbar_wait(&full[q % S], (uint32_t)(q / S) & 1u);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    constexpr uint32_t idesc = instr_desc_bf16(BN);
    int it = 0, tc = 0;
    for (int t = blockIdx.x; t < tiles && !failed; t += gridDim.x, ++tc) {
      const int z = t % splits;
      const int kt0 = z * kt_per_split, nk = min(kt_all - kt0, kt_per_split);
      const int a = tc & 1;
      const uint32_t aph = (uint32_t)(tc >> 1) & 1u;
      if (!mbar_wait(&acc_empty[a], aph ^ 1u)) {
        failed = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t acc = tmem + (uint32_t)(a * kWsAccCols);
      bool ok = true;
      for (int kk = 0; kk < nk; ++kk, ++it) {
        const int s = it % S;
        const uint32_t ph = (uint32_t)(it / S) & 1u;
        if (!mbar_wait(&full[s], ph)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint8_t* sa = smem + s * (kABytes + kBBytes);
        const uint64_t ad = smem_desc_sw128(sa), bd = smem_desc_sw128(sa + kABytes);
#pragma unroll
        for (int k4 = 0; k4 < kBK / 16; ++k4)
          mma_bf16(acc, ad + 2 * k4, bd + 2 * k4, idesc, (kk > 0 || k4 > 0) ? 1u : 0u);
        mma_commit(&empty[s]);
      }
      if (!ok) {
        failed = 1;
        break;
      }
      mma_commit(&acc_full[a]);
    }
    // every MMA issued by this thread has completed before tensor memory is freed
    mma_commit(&mma_done);
    mbar_wait(&mma_done, 0u);
  } else if (warp >= 2) {
    // ---- epilogue ----
    const int ew = warp - 2, quarter = warp & 3, cg = ew >> 2;
    constexpr int kColsPerWarp = BN / 4;
    int tc = 0;
    for (int t = blockIdx.x; t < tiles && !failed; t += gridDim.x, ++tc) {
      const int z = t % splits, tn = (t / splits) % nt, tm = t / (splits * nt);
      const int a = tc & 1;
      const uint32_t aph = (uint32_t)(tc >> 1) & 1u;
      const bool ok = mbar_wait(&acc_full[a], aph);
      if (!__all_sync(0xffffffffu, ok)) {
        failed = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int row = tm * kBM + 32 * quarter + lane;
      const uint32_t base = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(a * kWsAccCols);
      float* c32 = ep.c32;
      if (EPI == kEpiF32 && c32) c32 += (int64_t)z * ep.split_stride;
#pragma unroll 1
      for (int c = cg * kColsPerWarp; c < (cg + 1) * kColsPerWarp; c += 16) {
        float v[16];
        tmem_ld16(base + (uint32_t)c, v);
        const int col0 = tn * BN + c;
        if (row < M && col0 < N) epilogue_chunk<EPI>(v, row, col0, N, ep, c32);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[a]);
    }
  }
  __syncthreads();
  if (failed && threadIdx.x == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kWsAccCols)
                 : "memory");
  }
}

// ---- fused network inference ----------------------------------------------------
// Every layer of the network for 128-row tiles in one persistent kernel: the
// activations of a tile never leave shared memory.  CTAs run in clusters of
// two on a pair of SMs, each taking 128 rows of a 256-row super-tile through
// the same sequence of jobs: each CTA fetches half the rows of every weight
// tile and multicasts it into the same ring stage of both CTAs, so the pair
// reads each weight tile from L2 once; a stage is released when both CTAs'
// MMAs have read it (each MMA thread's commit arrives on both CTAs' empty
// barrier).  A tile's hidden
// activations (128 rows x up to 256 BF16) sit in its 64 KB buffer in the same
// 128-byte-swizzled K-major layout TMA would give them, so the next layer's
// tcgen05.mma reads them directly as its A operand; the input rows and every
// weight tile stream through a ring of 32 KB stages by TMA.  Two tiles are in
// flight per CTA (slots 0 and 1, each with its own activation buffer and
// 256-column accumulator in tensor memory): while the epilogue warps drain one
// slot's accumulator (bias, GELU, BF16 into the slot's buffer; bias and
// float32 to global memory for the output layer), the MMAs of the other
// slot's next layer run.  A job is one (tile, layer, N chunk); hidden layers
// are one chunk (N <= 256), the output layer is split into chunks of at most
// 256 columns.  Per slot, jobs run in order: MMA(j) -> epilogue(j) ->
// MMA(j + 1), so a hidden layer's epilogue overwrites the activations the
// layer's MMAs have finished reading.  The arithmetic of every output element
// (K order of the MMAs, bias, GELU, BF16 rounding) is that of the per-layer
// kernels, so both paths give the same bits.
//   full[s] / empty[s]        producers <-> MMA, ring stage s (empty counts
//                             both CTAs' MMA commits)
//   acc_full[a] / acc_empty[a]  MMA <-> epilogue, slot a
// Every wait is bounded as in the kernels above.
constexpr int kFusedRing = 3;
constexpr int kFusedStage = 32768;
constexpr int kFusedHBytes = 65536;
constexpr size_t kFusedSmem = 2 * (size_t)kFusedHBytes + (size_t)kFusedRing * kFusedStage + 1024;

struct FusedMaps {
  CUtensorMap x;
  CUtensorMap w[kFusedMaxLayers];
};

// Walks one CTA's jobs in the order all three roles (and both CTAs of the
// cluster) share.  The cluster's 256-row super-tiles t = cluster + k clusters
// alternate between the slots (k even: slot 0), each slot's jobs are its
// tiles' (layer, chunk) lists in turn, and the slots run half a tile's jobs
// apart: net.shift jobs of slot 0 first, then one job of each slot in turn.
// So consecutive epilogue jobs alternate between the output layer's stores
// and a hidden layer's arithmetic, and one slot's MMAs run while the other
// slot's epilogue does.  kWarp: the caller is a whole warp whose job runs
// warp-collective instructions, so the failure flag is read once for the
// warp.
template <bool kWarp, typename F>
__device__ __forceinline__ void fused_jobs(const FusedNet& net, volatile int* failed, F&& job) {
  const int tiles = (net.M + 2 * kBM - 1) / (2 * kBM);
  const int clusters = (int)gridDim.x >> 1, cid = (int)blockIdx.x >> 1;
  const int mine = cid < tiles ? (tiles - cid + clusters - 1) / clusters : 0;
  const int J = net.njobs;
  const int n[2] = {(mine + 1) / 2 * J, mine / 2 * J};
  int next[2] = {0, 0};
  auto run = [&](int sl) -> bool {
    const int stop = kWarp ? __shfl_sync(0xffffffffu, *failed, 0) : *failed;
    if (stop) return false;
    const int i = next[sl]++;
    const int q = i % J;
    if (!job(cid + (2 * (i / J) + sl) * clusters, sl, net.job_layer[q], net.job_chunk[q])) {
      *failed = 1;
      return false;
    }
    return true;
  };
  while (next[0] < n[0] && next[0] < net.shift)
    if (!run(0)) return;
  while (next[0] < n[0] || next[1] < n[1]) {
    if (next[1] < n[1] && !run(1)) return;
    if (next[0] < n[0] && !run(0)) return;
  }
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// TMA tile load delivered to the same shared-memory offset of every CTA in
// mask, each CTA's mbarrier at the same offset receiving the bytes it got.
__device__ __forceinline__ void tma_load_2d_mc(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                               uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar)), "h"(mask)
      : "memory");
}

// Shared-memory address of the same variable in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}

__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar) : "memory");
}

// mbar_wait for barriers that other CTAs of the cluster arrive on.
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = smem_u32(bar);
  const uint64_t t0 = global_ns();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > kWaitLimitNs) return false;
  }
}

// Pair MMA (cta_group::2): D [256 x N] over the two CTAs' tensor memories;
// A's rows 0..127 come from this CTA's shared memory and rows 128..255 from
// the peer's at the same offset, B's rows 0..N/2-1 from this CTA and the rest
// from the peer.
__device__ __forceinline__ void mma_bf16_pair(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                              uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit_pair(uint64_t* bar, uint16_t mask) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
               ::"r"(smem_u32(bar)), "h"(mask)
               : "memory");
}

// Arrives (once) on the mbarrier at this offset in every CTA of mask when this
// thread's earlier tcgen05 operations have completed.
__device__ __forceinline__ void mma_commit_mc(uint64_t* bar, uint16_t mask) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
               ::"r"(smem_u32(bar)), "h"(mask)
               : "memory");
}

// kPair = false: each CTA runs M = 128 MMAs on its own rows, the weight tiles
// shared by multicast (3 stages of 32 KB).  kPair = true: the pair runs
// M = 256 MMAs (cta_group::2, issued by CTA 0) over both CTAs' rows, each
// CTA holding only its half of every weight tile (6 stages of 16 KB); CTA
// 1's idle MMA thread forwards its stage arrivals to CTA 0 (pfull), and CTA
// 1's epilogue warps arrive on CTA 0's acc_empty.
template <bool kPair>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kWsThreads, 1) k_mlp_fused(const __grid_constant__ FusedMaps maps,
                                                             const __grid_constant__ FusedNet net,
                                                             int* __restrict__ err) {
  constexpr int kRing = kPair ? 6 : kFusedRing;
  constexpr int kStage = kPair ? kFusedStage / 2 : kFusedStage;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // the ring first: every operand read from it stays inside the allocation
  uint8_t* ring = smem;                              // [kRing][kStage] (96 KB)
  uint8_t* hbuf = smem + kFusedRing * kFusedStage;   // [2][64 KB]
  __shared__ __align__(8) uint64_t full[kRing], pfull[kRing], empty[kRing], acc_full[2], acc_empty[2], mma_done;
  __shared__ uint32_t tmem_base_sh;
  __shared__ volatile int failed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    failed = 0;
    for (int s = 0; s < kRing; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&pfull[s], 1);
      mbar_init(&empty[s], kPair ? 1 : 2);  // the MMAs that read the stage
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], kPair ? 2 * kWsEpiWarps : kWsEpiWarps);
    }
    mbar_init(&mma_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // the peer's barriers are initialised before anything multicasts or
  // arrives on them, and both CTAs are resident for the pair allocation
  cluster_sync_all();
  if (warp == 0) {
    // with cta_group::2, warp 0 of both CTAs allocates collectively (the
    // same columns in both tensor memories)
    if constexpr (kPair) {
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;"
                   ::"r"(smem_u32(&tmem_base_sh)), "r"(2 * kWsAccCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                   ::"r"(smem_u32(&tmem_base_sh)), "r"(2 * kWsAccCols)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;
  const int rank = (int)cluster_rank();
  const int row0 = rank * kBM;  // this CTA's rows within a 256-row super-tile

  if (warp == 0 && lane == 0) {
    // ---- producer: per job, (input tile, weight tile) per K tile of layer 0,
    // a weight tile per K tile of the later layers.  Input rows are this
    // CTA's own; of each N x 64 weight tile this CTA fetches rows
    // [rank N / 2, (rank + 1) N / 2): multicast to both CTAs (kPair false) or
    // into its own stage only, as its half of B (kPair true) ----
    int it = 0;
    auto stage = [&](bool weight, const CUtensorMap* map, int c0, int c1, int N) -> bool {
      const int s = it % kRing;
      const uint32_t ph = (uint32_t)(it / kRing) & 1u;
      if (!mbar_wait(&empty[s], ph ^ 1u)) return false;
      uint8_t* dst = ring + s * kStage;
      if (weight && kPair) {
        mbar_expect_tx(&full[s], (uint32_t)(N / 2) * kBK * 2);
        tma_load_2d(dst, map, &full[s], c0, c1 + rank * (N / 2));
      } else if (weight) {
        mbar_expect_tx(&full[s], (uint32_t)N * kBK * 2);  // both halves land here
        tma_load_2d_mc(dst + rank * (N / 2) * kBK * 2, map, &full[s], c0, c1 + rank * (N / 2), (uint16_t)3);
      } else {
        mbar_expect_tx(&full[s], kBM * kBK * 2);
        tma_load_2d(dst, map, &full[s], c0, c1);
      }
      ++it;
      return true;
    };
    fused_jobs<false>(net, &failed, [&](int tile, int, int l, int c) -> bool {
      const int kt = (net.dims[l] + kBK - 1) / kBK, N = net.chunk[l];
      for (int k = 0; k < kt; ++k) {
        if (l == 0 && !stage(false, &maps.x, k * kBK, tile * 2 * kBM + row0, kBM)) return false;
        if (!stage(true, &maps.w[l], k * kBK, c * N, N)) return false;
      }
      return true;
    });
    if (failed) {
      for (int q = max(0, it - kRing); q < it; ++q) mbar_wait(&full[q % kRing], (uint32_t)(q / kRing) & 1u);
    }
  } else if (warp == 1 && lane == 0 && kPair && rank != 0) {
    // ---- CTA 1 of a pair: tells CTA 0's MMA thread when each of its stages
    // has landed ----
    int it = 0;
    const uint32_t lead_pfull = cluster_addr(&pfull[0], 0);
    fused_jobs<false>(net, &failed, [&](int, int, int l, int) -> bool {
      const int n = ((net.dims[l] + kBK - 1) / kBK) * (l == 0 ? 2 : 1);
      for (int q = 0; q < n; ++q, ++it) {
        const int s = it % kRing;
        if (!mbar_wait(&full[s], (uint32_t)(it / kRing) & 1u)) return false;
        mbar_arrive_remote(lead_pfull + (uint32_t)(s * sizeof(uint64_t)));
      }
      return true;
    });
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer (CTA 0 of a pair, or every CTA without pairs) ----
    int it = 0;
    int jc[2] = {0, 0};
    auto take = [&](int& s) -> bool {
      s = it % kRing;
      const uint32_t ph = (uint32_t)(it / kRing) & 1u;
      bool ok = mbar_wait(&full[s], ph);
      if (kPair && ok) ok = mbar_wait_cluster(&pfull[s], ph);
      ++it;
      return ok;
    };
    fused_jobs<false>(net, &failed, [&](int, int sl, int l, int) -> bool {
      const uint32_t eph = ((uint32_t)jc[sl] & 1u) ^ 1u;
      if (!(kPair ? mbar_wait_cluster(&acc_empty[sl], eph) : mbar_wait(&acc_empty[sl], eph))) return false;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t acc = tmem + (uint32_t)(sl * kWsAccCols);
      // M = 256 over the pair (kPair) or 128
      const uint32_t idesc = (instr_desc_bf16(net.chunk[l]) & ~(31u << 24)) | ((uint32_t)((kPair ? 256 : 128) >> 4) << 24);
      const int kt = (net.dims[l] + kBK - 1) / kBK;
      for (int k = 0; k < kt; ++k) {
        int sx = -1, sw = -1;
        if (l == 0 && !take(sx)) return false;
        if (!take(sw)) return false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint64_t ad = smem_desc_sw128(l == 0 ? ring + sx * kStage : hbuf + sl * kFusedHBytes + k * kBM * kBK * 2);
        const uint64_t bd = smem_desc_sw128(ring + sw * kStage);
#pragma unroll
        for (int k4 = 0; k4 < kBK / 16; ++k4) {
          if constexpr (kPair) mma_bf16_pair(acc, ad + 2 * k4, bd + 2 * k4, idesc, (k > 0 || k4 > 0) ? 1u : 0u);
          else mma_bf16(acc, ad + 2 * k4, bd + 2 * k4, idesc, (k > 0 || k4 > 0) ? 1u : 0u);
        }
        if constexpr (kPair) {
          if (sx >= 0) mma_commit_pair(&empty[sx], (uint16_t)3);
          mma_commit_pair(&empty[sw], (uint16_t)3);
        } else {
          if (sx >= 0) mma_commit_mc(&empty[sx], (uint16_t)3);
          mma_commit_mc(&empty[sw], (uint16_t)3);
        }
      }
      if constexpr (kPair) mma_commit_pair(&acc_full[sl], (uint16_t)3);
      else mma_commit(&acc_full[sl]);
      ++jc[sl];
      return true;
    });
    if constexpr (kPair) mma_commit_pair(&mma_done, (uint16_t)1);
    else mma_commit(&mma_done);
    mbar_wait(&mma_done, 0u);
  } else if (warp >= 2) {
    // ---- epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. and a
    // quarter of the job's columns ----
    const int ew = warp - 2, quarter = warp & 3, cg = ew >> 2;
    const int rt = 32 * quarter + lane;  // row within the tile
    int jc[2] = {0, 0};
    fused_jobs<true>(net, &failed, [&](int tile, int sl, int l, int c) -> bool {
      const bool hidden = l + 1 < net.L;
      const bool ok = mbar_wait(&acc_full[sl], (uint32_t)jc[sl] & 1u);
      if (!__all_sync(0xffffffffu, ok)) return false;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int N = net.chunk[l], n0 = c * N, cpw = N / 4;
      const uint32_t base = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(sl * kWsAccCols);
      const float* bias = net.bias[l] + n0;
      const uint32_t hrow = smem_u32(hbuf + sl * kFusedHBytes) + (uint32_t)rt * 128u;
      if (!hidden) {
        // output layer: sector-complete float32 stores (8 rows x 32 bytes per
        // warp store), from the 16-lane accumulator fragment; each piece's
        // bias values (columns cc + 8 rp + 2 (lane % 4) + {0, 1}) are loaded
        // before its accumulator read
#pragma unroll 1
        for (int cc = cg * cpw; cc < (cg + 1) * cpw; cc += 16) {
          float ob[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) ob[k] = bias[cc + 8 * (k >> 1) + 2 * (lane & 3) + (k & 1)];
          float v[16];
          tmem_ld_rows32(base + (uint32_t)cc, v);
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int half = 0; half < 2; ++half) {
              const int r = tile * 2 * kBM + row0 + 32 * quarter + 16 * h + 8 * half + (lane >> 2);
              if (r >= net.M) continue;
#pragma unroll
              for (int rp = 0; rp < 2; ++rp) {
                float* dst = net.y + (int64_t)r * net.ldy + n0 + cc + 8 * rp + 2 * (lane & 3);
                const float y0 = v[8 * h + 4 * rp + 2 * half] + ob[2 * rp];
                const float y1 = v[8 * h + 4 * rp + 2 * half + 1] + ob[2 * rp + 1];
                if ((reinterpret_cast<uintptr_t>(dst) & 7) == 0) {
                  *reinterpret_cast<float2*>(dst) = make_float2(y0, y1);
                } else {
                  dst[0] = y0;
                  dst[1] = y1;
                }
              }
            }
        }
      }
#pragma unroll 1
      for (int cc = cg * cpw; hidden && cc < (cg + 1) * cpw; cc += 16) {
        // bias first, so its load overlaps the accumulator read
        float b[16];
        if (aligned16(bias + cc)) {
          load16(bias + cc, b);
        } else {
#pragma unroll
          for (int k = 0; k < 16; ++k) b[k] = bias[cc + k];
        }
        float v[16];
        tmem_ld16(base + (uint32_t)cc, v);
        {
          uint32_t w[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const float2 g = gelu2(__fadd2_rn(make_float2(v[2 * k], v[2 * k + 1]), make_float2(b[2 * k], b[2 * k + 1])));
            const __nv_bfloat162 p2 = __floats2bfloat162_rn(g.x, g.y);
            w[k] = *reinterpret_cast<const uint32_t*>(&p2);
          }
          // columns cc .. cc + 15 = 16-byte chunks j, j + 1 of swizzle atom cc / 64
          const int col = n0 + cc;
          const uint32_t atom = hrow + (uint32_t)(col >> 6) * (uint32_t)(kBM * kBK * 2);
          const uint32_t j = (uint32_t)(col & 63) >> 3, sw = (uint32_t)rt & 7u;
          st_shared_v4(atom + ((j ^ sw) << 4), w[0], w[1], w[2], w[3]);
          st_shared_v4(atom + (((j + 1) ^ sw) << 4), w[4], w[5], w[6], w[7]);
        }
      }
      // activations written by these threads become the async proxy's MMA operand
      // (all state spaces: with pairs the reader is the other CTA's MMA)
      if (hidden) asm volatile("fence.proxy.async;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        if (kPair && rank != 0) mbar_arrive_remote(cluster_addr(&acc_empty[sl], 0));
        else mbar_arrive(&acc_empty[sl]);
      }
      ++jc[sl];
      return true;
    });
  }
  __syncthreads();
  if (failed && threadIdx.x == 0) atomicExch(err, 1);
  // neither CTA leaves while the peer may still multicast into its ring or
  // commit to its barriers
  cluster_sync_all();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) {
    if constexpr (kPair)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kWsAccCols)
                   : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kWsAccCols)
                   : "memory");
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

int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  CCG_CUDA(cudaGetDevice(&dev));
  int& v = cached[dev & 63];
  if (!v) CCG_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
  return v;
}

template <int BN, int EPI>
void launch_bn(const CUtensorMap& a, const CUtensorMap& b, int M, int N, int K, const GemmShape& sh,
               const GemmEpilogue& ep, int* err, cudaStream_t s) {
  const int kt_all = (K + kBK - 1) / kBK;
  const int per = (kt_all + sh.splits - 1) / sh.splits;
  const int z = (kt_all + per - 1) / per;  // every split gets at least one K tile
  if (sh.persistent) {
    const size_t smem = (size_t)ws_stages(BN) * (kBM * kBK * 2 + BN * kBK * 2) + 1024;
    auto kern = k_gemm_ws<BN, EPI>;
    set_smem_limit(reinterpret_cast<const void*>(kern), smem);
    const int64_t tiles = (int64_t)((M + kBM - 1) / kBM) * ((N + BN - 1) / BN) * z;
    const unsigned grid = (unsigned)std::min<int64_t>(tiles, num_sms());
    kern<<<grid, kWsThreads, smem, s>>>(a, b, M, N, K, per, z, ep, err);
  } else {
    const size_t smem = (size_t)kStages * (kBM * kBK * 2 + BN * kBK * 2) + 1024;
    auto kern = k_gemm_tn<BN, EPI>;
    set_smem_limit(reinterpret_cast<const void*>(kern), smem);
    const dim3 grid((unsigned)((M + kBM - 1) / kBM), (unsigned)((N + BN - 1) / BN), (unsigned)z);
    kern<<<grid, 128, smem, s>>>(a, b, M, N, K, per, ep, err);
  }
  CCG_CUDA(cudaGetLastError());
}

template <int EPI>
void launch_epi(const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N, int K, GemmShape sh,
                const GemmEpilogue& ep, int* err, cudaStream_t s) {
  const CUtensorMap ma = make_map(A, M, K, lda, kBM);
  switch (sh.bn) {
    case 64: launch_bn<64, EPI>(ma, make_map(B, N, K, ldb, 64), M, N, K, sh, ep, err, s); break;
    case 128: launch_bn<128, EPI>(ma, make_map(B, N, K, ldb, 128), M, N, K, sh, ep, err, s); break;
    case 192: launch_bn<192, EPI>(ma, make_map(B, N, K, ldb, 192), M, N, K, sh, ep, err, s); break;
    default: launch_bn<256, EPI>(ma, make_map(B, N, K, ldb, 256), M, N, K, sh, ep, err, s); break;
  }
}

}  // namespace

void gelu_check(const float* x, int n, float* out, cudaStream_t s) {
  k_erf_check<<<(n + 255) / 256, 256, 0, s>>>(x, n, out);
  CCG_CUDA(cudaGetLastError());
}

bool mlp_fused_supported(const std::vector<int>& dims) {
  const int L = (int)dims.size() - 1;
  if (L < 1 || L > kFusedMaxLayers || dims[0] < 1) return false;
  for (int l = 1; l < L; ++l)
    if (dims[l] % 64 != 0 || dims[l] > 256) return false;
  // one job per hidden layer, output chunks of at least 64 columns
  return dims[L] % 64 == 0 && (L - 1) + dims[L] / 64 <= kFusedMaxJobs;
}

void mlp_forward_fused(const void* X, int64_t ldx, int M, const std::vector<int>& dims,
                       const std::vector<const __nv_bfloat16*>& w, const std::vector<int>& ldk,
                       const std::vector<const float*>& bias, float* Y, int64_t ldy, int* err, cudaStream_t s,
                       bool pair) {
  CCG_CHECK(mlp_fused_supported(dims), CC_ERR_INVALID_ARG, "network shape not covered by the fused kernel");
  const int L = (int)dims.size() - 1;
  CCG_CHECK(M > 0 && (int)w.size() == L && (int)ldk.size() == L && (int)bias.size() == L && Y && ldy >= dims[L],
            CC_ERR_INVALID_ARG, "fused network forward: bad arguments");
  FusedMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  FusedNet net;
  net.L = L;
  net.M = M;
  net.y = Y;
  net.ldy = ldy;
  maps.x = make_map(X, M, dims[0], ldx, kBM);
  for (int l = 0; l <= L; ++l) net.dims[l] = dims[l];
  for (int l = 0; l < L; ++l) {
    int chunk = dims[l + 1];
    if (l + 1 == L)  // the widest multiple of 64 up to 256 that divides the output width
      for (chunk = 256; dims[L] % chunk != 0; chunk -= 64) {}
    net.chunk[l] = chunk;
    for (int c = 0; c < dims[l + 1] / chunk; ++c) {
      CCG_CHECK(net.njobs < kFusedMaxJobs, CC_ERR_INVALID_ARG, "network shape not covered by the fused kernel");
      net.job_layer[net.njobs] = l;
      net.job_chunk[net.njobs] = c;
      ++net.njobs;
    }
    net.bias[l] = bias[l];
    maps.w[l] = make_map(w[l], dims[l + 1], dims[l], ldk[l], chunk / 2);  // each CTA of a pair fetches half
  }
  net.shift = net.njobs / 2;
  const void* kern = pair ? reinterpret_cast<const void*>(k_mlp_fused<true>) : reinterpret_cast<const void*>(k_mlp_fused<false>);
  set_smem_limit(kern, kFusedSmem);
  // clusters of two CTAs (one per SM), one 256-row super-tile pair at a time
  const int tiles = (M + 2 * kBM - 1) / (2 * kBM);
  const unsigned grid = 2u * (unsigned)std::max(1, std::min(tiles, num_sms() / 2));
  if (pair) k_mlp_fused<true><<<grid, kWsThreads, kFusedSmem, s>>>(maps, net, err);
  else k_mlp_fused<false><<<grid, kWsThreads, kFusedSmem, s>>>(maps, net, err);
  CCG_CUDA(cudaGetLastError());
}

GemmShape gemm_pick_shape(int M, int N, int K, bool allow_split) {
  // the persistent kernel keeps one CTA per SM; aim for at least one tile per SM
  const int slots = num_sms();
  GemmShape sh;
  const int mt = (M + kBM - 1) / kBM;
  const int cands[4] = {256, 192, 128, 64};
  sh.bn = 64;
  for (int bn : cands) {
    if (N % bn != 0 && bn != 64) continue;
    if ((int64_t)mt * ((N + bn - 1) / bn) >= slots || allow_split) {
      sh.bn = bn;
      break;
    }
  }
  if (allow_split) {
    const int tiles = mt * ((N + sh.bn - 1) / sh.bn);
    const int kt = (K + kBK - 1) / kBK;
    const int want = (slots + tiles - 1) / tiles;
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
