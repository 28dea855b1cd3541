// Internal declarations of the learned-subspace MLP (BF16 tensor-core GEMMs).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace ccg {

enum : int {
  kEpiF32 = 0,       // C (float32); with split K, one slice per split
  kEpiBiasF32 = 1,   // C + bias (float32)
  kEpiBiasGelu = 2,  // Z = C + bias (float32), H = gelu(Z) (bf16, optionally also transposed)
  kEpiGeluGrad = 3   // dZ = C * gelu'(Z) (bf16, optionally also transposed)
};

struct GemmEpilogue {
  float* c32 = nullptr;
  int64_t ldc = 0;
  int64_t split_stride = 0;      // elements between the float32 slices of a split-K product
  const float* bias = nullptr;
  float* z32 = nullptr;          // pre-activation (written by kEpiBiasGelu, read by kEpiGeluGrad)
  int64_t ldz = 0;
  __nv_bfloat16* h16 = nullptr;  // activation or gradient, row-major
  int64_t ldh = 0;
  __nv_bfloat16* ht16 = nullptr; // the same, transposed (column-major copy), or nullptr
  int64_t ldt = 0;
};

struct GemmShape {
  int bn = 64;             // N tile (64, 128, 192 or 256)
  int splits = 1;          // K splits (kEpiF32 only)
  bool persistent = true;  // persistent warp-specialised kernel; false: one tile per CTA
};

// C[M x N] = A[M x K] . B[N x K]^T, A and B row-major BF16 with leading
// dimensions lda, ldb (multiples of 8), through the tcgen05 kernel.  With
// shape.splits > 1 (kEpiF32 only) split z of the K tiles writes its partial
// product to ep.c32 + z * ep.split_stride.
void gemm_tn(const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N, int K, int epi,
             const GemmEpilogue& ep, int* err, cudaStream_t s, GemmShape shape);
// Launch shape for an M x N x K product: the widest N tile that still gives
// at least one tile per SM, and (when allow_split) enough K splits to fill the
// GPU with at least four K tiles per split.
GemmShape gemm_pick_shape(int M, int N, int K, bool allow_split);
// out[3k .. 3k+2] = (erf, GELU, GELU') of x[k] with the epilogues' arithmetic
void gelu_check(const float* x, int n, float* out, cudaStream_t s);

}  // namespace ccg
