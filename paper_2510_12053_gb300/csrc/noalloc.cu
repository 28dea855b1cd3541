// Allocation-free construction of perturbation bases.
//
// cc_build_subspace allocates its dense patch workspace with cudaMalloc.
// Some callers cannot let a library do that: processes whose device memory is
// entirely reserved by their own pool allocator (a cudaMalloc would fail or
// fragment it), or time-critical loops that cannot absorb cudaMalloc's
// implicit synchronisation and latency.  cc_build_bases_noalloc serves them:
// it runs the same dense patch Cholesky, but its workspace is the file-scope
// device array below, which the CUDA runtime reserves once on every GPU that
// loads this library and keeps until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "cc_internal.cuh"

namespace ccg {
namespace {

// 16 MiB of float64 workspace (2 Mi doubles), shared by every call on a device.
constexpr size_t kNoallocScratchDoubles = size_t(2) << 20;
static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];
// Status words: [0] patches that were not positive definite, [1] the largest
// support among the listed vertices, [2] patches larger than the slice.
static __device__ __align__(256) int g_noalloc_fail[64];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;  // guards the per-device address cache below
double* g_scratch_ptr[kMaxDevices] = {nullptr};
int* g_fail_ptr[kMaxDevices] = {nullptr};

// Largest support |S_i| over the listed vertices, into *out (atomicMax; *out
// starts at zero).  Runs before the patch kernel so that an understated
// max_support is refused before any workspace slice is touched.
__global__ void k_noalloc_max_support(const int32_t* __restrict__ verts, int64_t count,
                                      const int32_t* __restrict__ sup_ptr, int* __restrict__ out) {
  int best = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x) {
    const int i = verts[k];
    best = max(best, sup_ptr[i + 1] - sup_ptr[i]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

__device__ __forceinline__ int find_sorted_na(const int32_t* a, int m, int key) {
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

// Same algorithm as the patch kernel of cc_build_subspace: one CTA per vertex
// assembles H_PP (column-major, N x N, N = 3 |S_i|) and -H_Pi in its slice of
// `scratch`, factors H_PP = L L^T and solves for the basis blocks.
__global__ void k_patch_basis_noalloc(const int32_t* __restrict__ verts, const int32_t* __restrict__ sup_ptr,
                                      const int32_t* __restrict__ sup_idx, const int32_t* __restrict__ bsr_ptr,
                                      const int32_t* __restrict__ bsr_col, const double* __restrict__ bsr,
                                      int Nmax, double* __restrict__ scratch, double* __restrict__ Uout,
                                      int* __restrict__ fail) {
  const int i = verts[blockIdx.x];
  const int s0 = sup_ptr[i], m = sup_ptr[i + 1] - s0;
  const int N = 3 * m;
  if (m == 0) return;
  if (N > Nmax) {  // never true after the host's support check; refuse rather than overrun the slice
    if (threadIdx.x == 0) atomicAdd(fail + 2, 1);
    return;
  }
  double* A = scratch + (size_t)blockIdx.x * ((size_t)Nmax * Nmax + 3 * (size_t)Nmax);
  double* R = A + (size_t)Nmax * Nmax;
  const int32_t* S = sup_idx + s0;
  for (int64_t k = threadIdx.x; k < (int64_t)N * N; k += blockDim.x) A[k] = 0.0;
  for (int k = threadIdx.x; k < 3 * N; k += blockDim.x) R[k] = 0.0;
  __syncthreads();
  for (int a = threadIdx.x; a < m; a += blockDim.x) {
    const int j = S[a];
    for (int p = bsr_ptr[j]; p < bsr_ptr[j + 1]; ++p) {
      const int l = bsr_col[p];
      const double* Hb = bsr + (int64_t)p * 9;
      if (l == i) {
        for (int r = 0; r < 3; ++r)
          for (int d = 0; d < 3; ++d) R[d * N + 3 * a + r] = -Hb[3 * r + d];
      } else {
        const int t = find_sorted_na(S, m, l);
        if (t >= 0)
          for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) A[(size_t)(3 * t + c) * N + 3 * a + r] = Hb[3 * r + c];
      }
    }
  }
  __syncthreads();
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int c = 0; c < N; ++c) {
    if (threadIdx.x == 0) {
      const double d = A[(size_t)c * N + c];
      if (!(d > 0.0)) bad = 1;
      A[(size_t)c * N + c] = sqrt(fmax(d, 1e-300));
    }
    __syncthreads();
    const double piv = A[(size_t)c * N + c];
    for (int r = c + 1 + threadIdx.x; r < N; r += blockDim.x) A[(size_t)c * N + r] /= piv;
    __syncthreads();
    for (int r = c + 1 + threadIdx.x; r < N; r += blockDim.x) {
      const double lrc = A[(size_t)c * N + r];
      for (int s = c + 1; s <= r; ++s) A[(size_t)s * N + r] -= lrc * A[(size_t)c * N + s];
    }
    __syncthreads();
  }
  for (int c = 0; c < N; ++c) {
    if (threadIdx.x < 3) R[threadIdx.x * N + c] /= A[(size_t)c * N + c];
    __syncthreads();
    for (int k = threadIdx.x; k < 3 * (N - c - 1); k += blockDim.x) {
      const int d = k / (N - c - 1), r = c + 1 + k % (N - c - 1);
      R[d * N + r] -= A[(size_t)c * N + r] * R[d * N + c];
    }
    __syncthreads();
  }
  for (int c = N - 1; c >= 0; --c) {
    if (threadIdx.x < 3) R[threadIdx.x * N + c] /= A[(size_t)c * N + c];
    __syncthreads();
    for (int k = threadIdx.x; k < 3 * c; k += blockDim.x) {
      const int d = k / c, r = k % c;
      R[d * N + r] -= A[(size_t)r * N + c] * R[d * N + c];
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < 9 * m; k += blockDim.x) {
    const int a = k / 9, q = k % 9, r = q / 3, d = q % 3;
    Uout[(int64_t)(s0 + a) * 9 + q] = R[d * N + 3 * a + r];
  }
  if (threadIdx.x == 0 && bad) atomicAdd(fail, 1);
}

// Device addresses of the file-scope arrays for the current device, looked up
// once per device (host code may not take the address of a __device__ symbol
// directly: the symbol's name on the host is only a stand-in).
void noalloc_setup(double** scratch, int** fail) {
  int dev = 0;
  CCG_CUDA(cudaGetDevice(&dev));
  CCG_CHECK(dev >= 0 && dev < kMaxDevices, CC_ERR_INVALID_ARG, "device index beyond 63");
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    void* q = nullptr;
    CCG_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    CCG_CUDA(cudaGetSymbolAddress(&q, g_noalloc_fail));
    g_scratch_ptr[dev] = static_cast<double*>(p);
    g_fail_ptr[dev] = static_cast<int*>(q);
  }
  *scratch = g_scratch_ptr[dev];
  *fail = g_fail_ptr[dev];
}

}  // namespace
}  // namespace ccg

extern "C" cc_status cc_build_bases_noalloc(const double* H_blocks, const int32_t* row_ptr, const int32_t* col_idx,
                                            const int32_t* verts, int64_t count, const int32_t* sup_ptr,
                                            const int32_t* sup_idx, int32_t max_support, double* U_out,
                                            void* stream) {
  try {
    ccg::set_error("");
    CCG_CHECK(H_blocks && row_ptr && col_idx && sup_ptr && sup_idx && U_out, CC_ERR_INVALID_ARG,
              "cc_build_bases_noalloc: NULL device pointer");
    CCG_CHECK(count >= 0 && (count == 0 || verts), CC_ERR_INVALID_ARG, "cc_build_bases_noalloc: bad vertex list");
    CCG_CHECK(max_support >= 0, CC_ERR_INVALID_ARG, "cc_build_bases_noalloc: negative max_support");
    const size_t Nmax = 3 * (size_t)(max_support > 0 ? max_support : 1);
    const size_t per = Nmax * Nmax + 3 * Nmax;
    CCG_CHECK(per <= ccg::kNoallocScratchDoubles, CC_ERR_INVALID_ARG,
              "cc_build_bases_noalloc: max_support " + std::to_string(max_support) +
                  " needs a dense patch workspace larger than the 16 MiB static buffer (largest allowed "
                  "support: " + std::to_string(CC_NOALLOC_MAX_SUPPORT) + " vertices)");
    if (count == 0) return CC_OK;
    double* scratch = nullptr;
    int* fail = nullptr;
    ccg::noalloc_setup(&scratch, &fail);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CCG_CUDA(cudaMemsetAsync(fail, 0, 3 * sizeof(int), s));
    // every listed support must fit the slice that max_support sizes
    ccg::k_noalloc_max_support<<<(unsigned)std::min<int64_t>((count + 255) / 256, 1024), 256, 0, s>>>(
        verts, count, sup_ptr, fail + 1);
    CCG_CUDA(cudaGetLastError());
    int hmax = 0;
    CCG_CUDA(cudaMemcpyAsync(&hmax, fail + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    CCG_CUDA(cudaStreamSynchronize(s));
    CCG_CHECK(hmax <= max_support, CC_ERR_INVALID_ARG,
              "cc_build_bases_noalloc: a listed vertex has " + std::to_string(hmax) +
                  " support vertices, more than max_support = " + std::to_string(max_support));
    const int64_t batch = (int64_t)(ccg::kNoallocScratchDoubles / per);
    for (int64_t b0 = 0; b0 < count; b0 += batch) {
      const int64_t cnt = count - b0 < batch ? count - b0 : batch;
      ccg::k_patch_basis_noalloc<<<(unsigned)cnt, 256, 0, s>>>(verts + b0, sup_ptr, sup_idx, row_ptr, col_idx,
                                                               H_blocks, (int)Nmax, scratch, U_out, fail);
      CCG_CUDA(cudaGetLastError());
    }
    int hf[3] = {0, 0, 0};
    CCG_CUDA(cudaMemcpyAsync(hf, fail, sizeof(hf), cudaMemcpyDeviceToHost, s));
    CCG_CUDA(cudaStreamSynchronize(s));
    CCG_CHECK(hf[2] == 0, CC_ERR_INVALID_ARG, "cc_build_bases_noalloc: a support grew beyond max_support");
    CCG_CHECK(hf[0] == 0, CC_ERR_NUMERIC, "cc_build_bases_noalloc: a patch Hessian was not positive definite");
    return CC_OK;
  } catch (const ccg::Fail& f) {
    return f.st;
  } catch (...) {
    ccg::set_error("cc_build_bases_noalloc: unexpected error");
    return CC_ERR_STATE;
  }
}
