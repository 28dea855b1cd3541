// Internal declarations of the learned-subspace MLP (BF16 tensor-core GEMMs).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

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
// The whole network's inference in one kernel (activations kept on chip).
constexpr int kFusedMaxLayers = 6;
constexpr int kFusedMaxJobs = 32;           // (layer, N chunk) passes per tile
struct FusedNet {
  int L = 0, M = 0;
  int dims[kFusedMaxLayers + 1] = {};       // d_in, hidden..., d_out
  int chunk[kFusedMaxLayers] = {};          // N columns per accumulator pass
  int njobs = 0, shift = 0;                 // passes per tile; slot 1 runs `shift` passes behind slot 0
  int job_layer[kFusedMaxJobs] = {};
  int job_chunk[kFusedMaxJobs] = {};
  const float* bias[kFusedMaxLayers] = {};
  float* y = nullptr;
  int64_t ldy = 0;
};
// True when the fused kernel covers the shape: at most kFusedMaxLayers layers,
// hidden widths multiples of 64 up to 256, an output width that is a multiple
// of 64 (any input width), at most kFusedMaxJobs passes per tile.
bool mlp_fused_supported(const std::vector<int>& dims);
// Y[M x d_out] (float32, leading dim ldy) = the network applied to the rows of
// X (BF16, leading dim ldx, a multiple of 8): per hidden layer GELU(W h + b)
// rounded to BF16, the output layer W h + b; w[l] is the BF16 [d_{l+1} x ldk[l]]
// weight, bias[l] the float32 bias.  Bitwise the same as the per-layer GEMMs.
// pair: M = 256 MMAs over SM pairs (cta_group::2), each SM holding half of
// every weight tile; otherwise M = 128 per SM with the weight tiles
// multicast to both SMs of a pair.
void mlp_forward_fused(const void* X, int64_t ldx, int M, const std::vector<int>& dims,
                       const std::vector<const __nv_bfloat16*>& w, const std::vector<int>& ldk,
                       const std::vector<const float*>& bias, float* Y, int64_t ldy, int* err, cudaStream_t s,
                       bool pair);
// out[3k .. 3k+2] = (erf, GELU, GELU') of x[k] with the epilogues' arithmetic
void gelu_check(const float* x, int n, float* out, cudaStream_t s);

}  // namespace ccg
