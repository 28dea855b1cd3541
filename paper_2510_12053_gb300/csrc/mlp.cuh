// Internal declarations of the learned-subspace MLP (BF16 tensor-core GEMMs).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace ccg {

enum : int {
  kEpiF32 = 0,       // C (float32)
  kEpiBiasF32 = 1,   // C + bias (float32)
  kEpiBiasGelu = 2,  // Z = C + bias (bf16), H = gelu(Z) (bf16, optionally also transposed)
  kEpiGeluGrad = 3   // dZ = C * gelu'(Z) (bf16, optionally also transposed)
};

struct GemmEpilogue {
  float* c32 = nullptr;
  int64_t ldc = 0;
  const float* bias = nullptr;
  __nv_bfloat16* z16 = nullptr;  // pre-activation (written by kEpiBiasGelu, read by kEpiGeluGrad)
  int64_t ldz = 0;
  __nv_bfloat16* h16 = nullptr;  // activation or gradient, row-major
  int64_t ldh = 0;
  __nv_bfloat16* ht16 = nullptr; // the same, transposed (column-major copy), or nullptr
  int64_t ldt = 0;
};

// C[M x N] = A[M x K] . B[N x K]^T, A and B row-major BF16 with leading
// dimensions lda, ldb (multiples of 8), through the tcgen05 kernel.
void gemm_tn(const void* A, int64_t lda, const void* B, int64_t ldb, int M, int N, int K, int epi,
             const GemmEpilogue& ep, int* err, cudaStream_t s);
int gemm_pick_bn(int N);

}  // namespace ccg
