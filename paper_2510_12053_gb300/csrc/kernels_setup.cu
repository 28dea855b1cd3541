// Setup kernels: greedy colouring of the 1-ring graph and the perturbation
// bases U_i = -H_PP^{-1} H_Pi (Eq. 5 on the patch P = S_i, Sec. 3.1).
#include <algorithm>
#include <vector>

#include "cc_internal.cuh"
#include "dmath.cuh"

namespace ccg {

namespace {

// One Jones-Plassmann round with index priority: an uncoloured vertex whose
// lower-id neighbours are all coloured takes the smallest colour none of them
// uses.  Higher-id neighbours cannot be coloured before it, so the result is
// exactly sequential greedy colouring in ascending id.
__global__ void k_color_round(int64_t n, const int32_t* __restrict__ nbr_ptr, const int32_t* __restrict__ nbr_idx,
                              int32_t* color, int32_t* changed) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= n) return;
  volatile int32_t* col = color;
  if (col[v] >= 0) return;
  const int p0 = nbr_ptr[v], p1 = nbr_ptr[v + 1];
  unsigned long long used = 0ull;
  bool big = false;
  for (int p = p0; p < p1; ++p) {
    const int u = nbr_idx[p];
    if (u >= v) break;  // neighbours are ascending
    const int cu = col[u];
    if (cu < 0) return;  // not ready this round
    if (cu < 64) used |= 1ull << cu;
    else big = true;
  }
  int c;
  if (!big) {
    c = __ffsll((long long)~used) - 1;
    if (c < 0) big = true;
  }
  if (big) {
    for (c = 0;; ++c) {
      bool taken = false;
      for (int p = p0; p < p1; ++p) {
        const int u = nbr_idx[p];
        if (u >= v) break;
        if (col[u] == c) { taken = true; break; }
      }
      if (!taken) break;
    }
  }
  col[v] = c;
  *changed = 1;
}

__device__ __forceinline__ int find_sorted(const int32_t* a, int m, int key) {
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

// Plain float64 patch solve (patches above 192 unknowns, and those the mixed
// kernel below declines): one CTA per free vertex of the batch.  A
// (column-major, N x N, N = 3m) and the right-hand sides R (column-major
// N x 3) live in the CTA's slice of scratch.  H is read from its upper 3x3 blocks (padded to 3 x 4): a block
// (j, l) of a support row j fills both (a, t) and (t, a); block (j, i) and
// blocks (i, l) of row i fill -H_Pi.  Writes
// U[(s0 + a) * 9 + 3 r + d] = z[3a + r][d] with H_PP z = -H_Pi.
__global__ void k_patch_basis(const int32_t* __restrict__ verts, const int32_t* __restrict__ sup_ptr,
                              const int32_t* __restrict__ sup_idx, const int32_t* __restrict__ up_ptr,
                              const int32_t* __restrict__ up_col, const double* __restrict__ bsr, int Nmax,
                              double* __restrict__ scratch, double* __restrict__ Uout, int32_t* __restrict__ fail) {
  const int i = verts[blockIdx.x];
  const int s0 = sup_ptr[i], m = sup_ptr[i + 1] - s0;
  const int N = 3 * m;
  if (m == 0) return;
  double* A = scratch + (size_t)blockIdx.x * ((size_t)Nmax * Nmax + 3 * (size_t)Nmax);
  double* R = A + (size_t)Nmax * Nmax;
  const int32_t* S = sup_idx + s0;
  for (int64_t k = threadIdx.x; k < (int64_t)N * N; k += blockDim.x) A[k] = 0.0;
  for (int k = threadIdx.x; k < 3 * N; k += blockDim.x) R[k] = 0.0;
  __syncthreads();
  for (int a = threadIdx.x; a <= m; a += blockDim.x) {
    const int j = a < m ? S[a] : i;
    for (int p = up_ptr[j]; p < up_ptr[j + 1]; ++p) {
      const int l = up_col[p];
      const double* Hb = bsr + (int64_t)p * 12;  // H_jl, row r at Hb[4 r]
      if (a < m) {
        if (l == j) {
          for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) A[(size_t)(3 * a + c) * N + 3 * a + r] = Hb[4 * r + c];
        } else if (l == i) {
          for (int r = 0; r < 3; ++r)
            for (int d = 0; d < 3; ++d) R[d * N + 3 * a + r] = -Hb[4 * r + d];
        } else {
          const int t = find_sorted(S, m, l);
          if (t >= 0)
            for (int r = 0; r < 3; ++r)
              for (int c = 0; c < 3; ++c) {
                A[(size_t)(3 * t + c) * N + 3 * a + r] = Hb[4 * r + c];
                A[(size_t)(3 * a + r) * N + 3 * t + c] = Hb[4 * r + c];
              }
        }
      } else if (l != i) {
        // row i: H_il with l > i; the patch needs H_li = H_il^T
        const int t = find_sorted(S, m, l);
        if (t >= 0)
          for (int r = 0; r < 3; ++r)
            for (int d = 0; d < 3; ++d) R[d * N + 3 * t + r] = -Hb[4 * d + r];
      }
    }
  }
  __syncthreads();
  // right-looking Cholesky, lower triangle, column-major
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
  // forward substitution L y = R, then L^T z = y (3 columns)
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
  // a patch whose H_PP is not positive definite leaves its basis untouched
  if (!bad)
    for (int k = threadIdx.x; k < 9 * m; k += blockDim.x) {
      const int a = k / 9, q = k % 9, r = q / 3, d = q % 3;
      Uout[(int64_t)(s0 + a) * 9 + q] = R[d * N + 3 * a + r];
    }
  if (threadIdx.x == 0 && bad) atomicAdd(fail, 1);
}

}  // namespace

void run_coloring(Mesh& m) {
  cudaStream_t s = m.stream;
  DBuf<int32_t> changed;
  changed.alloc(1);
  m.d_color.alloc(m.n);
  CCG_CUDA(cudaMemsetAsync(m.d_color.p, 0xff, m.n * sizeof(int32_t), s));
  int32_t* h_changed = nullptr;
  CCG_CUDA(cudaMallocHost((void**)&h_changed, sizeof(int32_t)));
  const unsigned grid = (unsigned)((m.n + 255) / 256);
  int64_t rounds = 0;
  try {
    while (true) {
      CCG_CUDA(cudaMemsetAsync(changed.p, 0, sizeof(int32_t), s));
      k_color_round<<<grid, 256, 0, s>>>(m.n, m.d_nbr_ptr.p, m.d_nbr_idx.p, m.d_color.p, changed.p);
      CCG_CUDA(cudaGetLastError());
      CCG_CUDA(cudaMemcpyAsync(h_changed, changed.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      CCG_CUDA(cudaStreamSynchronize(s));
      if (*h_changed == 0) break;
      CCG_CHECK(++rounds <= m.n, CC_ERR_STATE, "colouring did not terminate");
    }
  } catch (...) {
    cudaFreeHost(h_changed);
    throw;
  }
  cudaFreeHost(h_changed);
  m.color.assign(m.n, -1);
  CCG_CUDA(cudaMemcpy(m.color.data(), m.d_color.p, m.n * sizeof(int32_t), cudaMemcpyDeviceToHost));
  int32_t C = 0;
  for (int64_t v = 0; v < m.n; ++v) {
    CCG_CHECK(m.color[v] >= 0, CC_ERR_STATE, "colouring left a vertex uncoloured");
    C = std::max(C, m.color[v] + 1);
  }
  m.num_colors = C;
  build_color_lists(m);
}

void set_coloring(Mesh& m, const int32_t* colors, int32_t C) {
  CCG_CHECK(C >= 1 && C <= 1024, CC_ERR_INVALID_ARG, "number of colours must be in [1, 1024]");
  for (int64_t v = 0; v < m.n; ++v) {
    CCG_CHECK(colors[v] >= 0 && colors[v] < C, CC_ERR_INVALID_ARG, "colour out of range");
    for (int64_t p = m.nbr_ptr[v]; p < m.nbr_ptr[v + 1]; ++p)
      CCG_CHECK(colors[m.nbr_idx[p]] != colors[v], CC_ERR_INVALID_ARG,
                "two vertices of one tet share a colour (vertex " + std::to_string(v) + ")");
  }
  m.color.assign(colors, colors + m.n);
  m.num_colors = C;
  m.d_color.upload(m.color, m.stream);
  build_color_lists(m);
}

void build_color_lists(Mesh& m) {
  cudaStream_t s = m.stream;
  const int32_t C = m.num_colors;
  // free vertices per colour (ascending) and tets whose free vertex of colour c moves
  m.cv_ptr.assign(C + 1, 0);
  std::vector<std::vector<int32_t>> cv(C), tl(C);
  for (int64_t v = 0; v < m.n; ++v)
    if (!m.pinned[v]) cv[m.color[v]].push_back((int32_t)v);
  for (int64_t t = 0; t < m.T; ++t)
    for (int c = 0; c < 4; ++c) {
      const int32_t v = m.tets[4 * t + c];
      if (!m.pinned[v]) tl[m.color[v]].push_back((int32_t)t);
    }
  std::vector<int32_t> cv_flat, tl_flat;
  m.tl_ptr.assign(C + 1, 0);
  for (int c = 0; c < C; ++c) {
    cv_flat.insert(cv_flat.end(), cv[c].begin(), cv[c].end());
    m.cv_ptr[c + 1] = (int32_t)cv_flat.size();
    std::sort(tl[c].begin(), tl[c].end());
    tl_flat.insert(tl_flat.end(), tl[c].begin(), tl[c].end());
    m.tl_ptr[c + 1] = (int32_t)tl_flat.size();
  }
  m.d_cv_idx.upload(cv_flat, s);
  m.d_tl.upload(tl_flat, s);
  CCG_CUDA(cudaStreamSynchronize(s));
}

// k-ring supports on the host: breadth-first over the 1-ring CSR, free
// vertices only, i excluded, ascending.  Uploads them and the slot maps.
namespace {
// Index of key in the ascending a[0..m), or -1.
__device__ __forceinline__ int find_in_sorted(const int32_t* __restrict__ a, int m, int key) {
  int lo = 0, hi = m - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int x = a[mid];
    if (x == key) return mid;
    if (x < key) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

// Slot maps, one warp per free vertex v: for every upper block of the rows
// of S_v (in support order) and then of v's own row, in row order, a code:
// the diagonal block, the block whose column is v itself, the support slot
// of the block's column, or none (column outside the support).  Lane r takes
// row r of a 32-row chunk; a warp scan of the row lengths places the rows.
template <typename SlotT>
__global__ void k_slot_maps(const int32_t* __restrict__ rows, int64_t nrows, const int32_t* __restrict__ sup_ptr,
                            const int32_t* __restrict__ sup_idx, const int32_t* __restrict__ up_ptr,
                            const int32_t* __restrict__ up_col, const int64_t* __restrict__ smap_ptr,
                            SlotT* __restrict__ codes) {
  constexpr unsigned kNone = sizeof(SlotT) == 1 ? 0xFFu : 0xFFFFu, kSelf = kNone - 1, kDiag = kNone - 2;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= nrows) return;  // whole warps leave together
  const int v = rows[w];
  const int s0 = sup_ptr[v], m = sup_ptr[v + 1] - s0;
  const int32_t* S = sup_idx + s0;
  int64_t base = smap_ptr[v];
  for (int r0 = 0; r0 <= m; r0 += 32) {
    const int r = r0 + lane;
    int len = 0, p0 = 0;
    if (r <= m) {
      const int j = r < m ? S[r] : v;
      p0 = up_ptr[j];
      len = up_ptr[j + 1] - p0;
    }
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    for (int q = 0; q < len; ++q) {
      const int l = up_col[p0 + q];
      unsigned code;
      if (q == 0) code = kDiag;
      else if (l == v) code = kSelf;
      else {
        const int t = find_in_sorted(S, m, l);
        code = t >= 0 ? (unsigned)t : kNone;
      }
      codes[base + (incl - len) + q] = (SlotT)code;
    }
    base += __shfl_sync(0xffffffffu, incl, 31);
  }
}
}  // namespace

// Slot maps of the current supports (cc_build_subspace / cc_set_subspace),
// built on the device from the uploaded supports and upper block pattern.
// The host only sums the row lengths per vertex for the offsets.
void build_slot_maps(Mesh& m) {
  const int64_t n = m.n;
  cudaStream_t s = m.stream;
  m.smap_wide = m.sup_max >= 250;
  std::vector<int64_t> len(n, 0);
  const int nt = host_threads(n);
  std::vector<int64_t> longest_t(nt, 0);
  parallel_ranges(n, nt, [&](int t, int64_t v0, int64_t v1) {
    for (int64_t v = v0; v < v1; ++v) {
      if (m.pinned[v]) continue;
      int64_t c = m.up_ptr[v + 1] - m.up_ptr[v];
      for (int64_t p = m.sup_ptr[v]; p < m.sup_ptr[v + 1]; ++p) {
        const int32_t j = m.sup_idx[p];
        c += m.up_ptr[j + 1] - m.up_ptr[j];
      }
      len[v] = c;
      longest_t[t] = std::max(longest_t[t], c);
    }
  });
  std::vector<int64_t> ptr(n + 1, 0);
  for (int64_t v = 0; v < n; ++v) ptr[v + 1] = ptr[v] + len[v];
  m.smap_max = *std::max_element(longest_t.begin(), longest_t.end());
  m.d_smap_ptr.upload(ptr, s);

  const int64_t total = std::max<int64_t>(ptr[n], 1);
  const unsigned grid = (unsigned)((m.n_free * 32 + 255) / 256);
  if (m.smap_wide) {
    m.d_smap16.alloc(total + kSlotMapSlack);
    m.d_smap8.release();
    CCG_CUDA(cudaMemsetAsync(m.d_smap16.p + total, 0, kSlotMapSlack * sizeof(uint16_t), s));
    if (m.n_free > 0)
      k_slot_maps<uint16_t><<<grid, 256, 0, s>>>(m.d_free_rows.p, m.n_free, m.d_sup_ptr.p, m.d_sup_idx.p,
                                                 m.d_up_ptr.p, m.d_up_col.p, m.d_smap_ptr.p, m.d_smap16.p);
  } else {
    m.d_smap8.alloc(total + kSlotMapSlack);
    m.d_smap16.release();
    CCG_CUDA(cudaMemsetAsync(m.d_smap8.p + total, 0, kSlotMapSlack, s));
    if (m.n_free > 0)
      k_slot_maps<uint8_t><<<grid, 256, 0, s>>>(m.d_free_rows.p, m.n_free, m.d_sup_ptr.p, m.d_sup_idx.p,
                                                m.d_up_ptr.p, m.d_up_col.p, m.d_smap_ptr.p, m.d_smap8.p);
  }
  CCG_CUDA(cudaGetLastError());
  CCG_CUDA(cudaStreamSynchronize(s));
}

void build_supports(Mesh& m, int32_t k) {
  cudaStream_t s = m.stream;
  const int64_t n = m.n;
  // vertex ranges in parallel (each with its own visit stamps); concatenated in order
  const int nt = host_threads(n);
  std::vector<std::vector<int32_t>> idx_t(nt);
  std::vector<int64_t> len(n, 0);
  std::vector<int32_t> supmax_t(nt, 0);
  parallel_ranges(n, nt, [&](int t, int64_t v0, int64_t v1) {
    std::vector<int32_t> stamp(n, -1), ring, frontier, next;
    std::vector<int32_t>& out = idx_t[t];
    for (int64_t v = v0; v < v1; ++v) {
      if (m.pinned[v]) continue;
      ring.clear();
      frontier.assign(1, (int32_t)v);
      stamp[v] = (int32_t)v;
      for (int hop = 0; hop < k; ++hop) {
        next.clear();
        for (int32_t a : frontier)
          for (int64_t p = m.nbr_ptr[a]; p < m.nbr_ptr[a + 1]; ++p) {
            const int32_t b = m.nbr_idx[p];
            if (stamp[b] != (int32_t)v) {
              stamp[b] = (int32_t)v;
              next.push_back(b);
              if (!m.pinned[b]) ring.push_back(b);
            }
          }
        frontier.swap(next);
      }
      std::sort(ring.begin(), ring.end());
      out.insert(out.end(), ring.begin(), ring.end());
      len[v] = (int64_t)ring.size();
      supmax_t[t] = std::max<int32_t>(supmax_t[t], (int32_t)ring.size());
    }
  });
  m.sup_ptr.assign(n + 1, 0);
  for (int64_t v = 0; v < n; ++v) m.sup_ptr[v + 1] = m.sup_ptr[v] + len[v];
  m.sup_idx.clear();
  m.sup_idx.reserve(m.sup_ptr[n]);
  for (int t = 0; t < nt; ++t) m.sup_idx.insert(m.sup_idx.end(), idx_t[t].begin(), idx_t[t].end());
  const int32_t supmax = *std::max_element(supmax_t.begin(), supmax_t.end());
  CCG_CHECK(m.sup_idx.size() < (size_t(1) << 31), CC_ERR_INVALID_ARG, "support arrays exceed 2^31 entries");
  CCG_CHECK(supmax < 32768, CC_ERR_INVALID_ARG, "support larger than 32767 vertices");
  m.sup_max = supmax;
  int hs = 32;
  while (hs < 2 * std::max(supmax, 1)) hs <<= 1;
  m.hash_size = hs;
  m.k_ring = k;
  std::vector<int32_t> sp32(n + 1);
  for (int64_t v = 0; v <= n; ++v) sp32[v] = (int32_t)m.sup_ptr[v];
  m.d_sup_ptr.upload(sp32, s);
  m.d_sup_idx.upload(m.sup_idx, s);
  build_slot_maps(m);  // on the device, from the uploaded supports
  const int64_t total = (int64_t)m.sup_idx.size();
  m.f64.U.alloc(9 * std::max<int64_t>(total, 1));
  m.mx.U.alloc(9 * std::max<int64_t>(total, 1));
}

// Hessian of E at x (device float64 [3][n]) in float64 into the float64
// block rows (dynamic meshes: M + h^2 K).  The float64 solver state must exist.
void hessian_f64_at(Mesh& m, const double* x) {
  cudaStream_t s = m.stream;
  const double w = m.h > 0.0 ? m.h * m.h : 1.0;
  launch_tet_grad_f64(m, x, m.d_all_tets.p, m.n_active_tets, w, s);
  launch_rows_f64(m, x, x, w, s);
  CCG_CUDA(cudaStreamSynchronize(s));
}

// Rest Hessian (the bases' configuration, Sec. 3.1).
void rest_hessian_f64(Mesh& m) {
  const int64_t n = m.n;
  DBuf<double> Xs;
  std::vector<double> soa(3 * n);
  for (int64_t j = 0; j < n; ++j)
    for (int a = 0; a < 3; ++a) soa[a * n + j] = m.X[3 * j + a];
  Xs.upload(soa, m.stream);
  hessian_f64_at(m, Xs.p);
}

// Restarted bases: Eq. 5 on the current supports with the Hessian at x,
// written over the current bases; patches whose H_PP is not positive
// definite keep their basis.  Returns how many kept theirs.
int64_t rebuild_bases_at(Mesh& m, const double* x) {
  hessian_f64_at(m, x);
  const int64_t kept = patch_solves(m, m.d_free_rows.p, m.n_free, false);
  bases_to_f32(m);
  CCG_CUDA(cudaStreamSynchronize(m.stream));
  return kept;
}

// Dense patch solves (Eq. 5 on P = S_i) for a device list of free vertices,
// written into the float64 bases.  Needs the rest Hessian in the block rows.
namespace {
// ---- patch solves in float32 with float64 iterative refinement --------------
// For patches of at most kPmMaxN = 192 unknowns (every 2-ring of a Kuhn grid):
// H_PP is assembled in float32 into shared memory (packed lower triangle,
// column-major) and factored by Cholesky there; U = -H_PP^{-1} H_Pi is then
// reached by iterative refinement -- z += L^{-T} L^{-1} (B - H_PP z), B = -H_Pi,
// with the residual in float64 from the float64 block rows -- until the
// correction is below 1e-12 of z or stops shrinking (it then sits at the
// rounding level of the float64 residual).  A patch whose float32
// factorization meets a non-positive pivot, or whose last correction is above
// 1e-11 of z, is queued for the float64 kernel (which also decides positive
// definiteness).
constexpr int kPmMaxN = 192;
constexpr int kPmMaxIt = 4;
constexpr int kPmThreads = 256;

__host__ __device__ constexpr size_t pm_smem_bytes() {
  return (size_t)kPmMaxN * (kPmMaxN + 1) / 2 * sizeof(float) + 3 * (3 * (size_t)kPmMaxN * sizeof(double)) +
         3 * (size_t)kPmMaxN * sizeof(float) + (size_t)kPmMaxN * (kPmMaxN + 1) / 2 + 64;
}

__device__ __forceinline__ int pm_idx(int N, int c, int r) {  // lower (r >= c), column c
  return c * N - (c * (c - 1)) / 2 + (r - c);
}

// y_a = sum_t H_{S[a] S[t]} z_t (float64, 3 columns) for row block a of the
// patch, from the upper block rows: blocks (j, l >= j) of row j = S[a], and
// blocks (l, j) of the rows of j's lower neighbours l (stored transposed).
__device__ void pm_apply_row(int a, int i, const int32_t* __restrict__ S, int m, int N,
                             const int32_t* __restrict__ up_ptr, const int32_t* __restrict__ up_col,
                             const int32_t* __restrict__ nbr_ptr, const int32_t* __restrict__ nbr_idx,
                             const double* __restrict__ bsr, const double* Z, double* y /*[3][3] rows x cols*/) {
  const int j = S[a];
  for (int q = 0; q < 9; ++q) y[q] = 0.0;
  for (int p = up_ptr[j]; p < up_ptr[j + 1]; ++p) {
    const int l = up_col[p];
    const int t = l == j ? a : (l == i ? -1 : find_sorted(S, m, l));
    if (t < 0) continue;
    const double* Hb = bsr + (int64_t)p * 12;  // H_jl, row r at Hb[4 r]
    for (int r = 0; r < 3; ++r)
      for (int d = 0; d < 3; ++d) {
        double acc = y[3 * r + d];
        for (int c = 0; c < 3; ++c) acc = fma(Hb[4 * r + c], Z[d * N + 3 * t + c], acc);
        y[3 * r + d] = acc;
      }
  }
  for (int e = nbr_ptr[j]; e < nbr_ptr[j + 1]; ++e) {
    const int l = nbr_idx[e];
    if (l >= j) break;
    if (l == i) continue;
    const int t = find_sorted(S, m, l);
    if (t < 0) continue;
    const int q0 = up_ptr[l] + 1, q1 = up_ptr[l + 1];
    const int pos = find_sorted(up_col + q0, q1 - q0, j);
    if (pos < 0) continue;
    const double* Hb = bsr + (int64_t)(q0 + pos) * 12;  // H_lj; H_jl = H_lj^T
    for (int r = 0; r < 3; ++r)
      for (int d = 0; d < 3; ++d) {
        double acc = y[3 * r + d];
        for (int c = 0; c < 3; ++c) acc = fma(Hb[4 * c + r], Z[d * N + 3 * t + c], acc);
        y[3 * r + d] = acc;
      }
  }
}

__global__ void __launch_bounds__(kPmThreads) k_patch_basis_mixed(
    const int32_t* __restrict__ verts, const int32_t* __restrict__ sup_ptr, const int32_t* __restrict__ sup_idx,
    const int32_t* __restrict__ up_ptr, const int32_t* __restrict__ up_col, const int32_t* __restrict__ nbr_ptr,
    const int32_t* __restrict__ nbr_idx, const double* __restrict__ bsr, double* __restrict__ Uout,
    int32_t* __restrict__ redo, int32_t* __restrict__ n_redo) {
  extern __shared__ __align__(16) unsigned char pm_smem[];
  float* L = reinterpret_cast<float*>(pm_smem);
  double* B = reinterpret_cast<double*>(pm_smem + (size_t)kPmMaxN * (kPmMaxN + 1) / 2 * sizeof(float));
  double* Z = B + 3 * kPmMaxN;
  double* R = Z + 3 * kPmMaxN;
  float* D = reinterpret_cast<float*>(R + 3 * kPmMaxN);
  uint8_t* colof = reinterpret_cast<uint8_t*>(D + 3 * kPmMaxN);  // packed index -> its column
  __shared__ int cstart[kPmMaxN + 1];                              // packed start of each column
  __shared__ int bad;
  __shared__ double dmax, zmax;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i = verts[blockIdx.x];
  const int s0 = sup_ptr[i], m = sup_ptr[i + 1] - s0;
  const int N = 3 * m;
  if (m == 0) return;  // the whole CTA leaves
  const int32_t* S = sup_idx + s0;
  const int nL = N * (N + 1) / 2;
  for (int k = tid; k < nL; k += kPmThreads) L[k] = 0.0f;
  for (int k = tid; k < 3 * N; k += kPmThreads) {
    B[k] = 0.0;
    Z[k] = 0.0;
  }
  if (tid == 0) bad = 0;
  for (int c = tid; c <= N; c += kPmThreads) cstart[c] = c * N - (c * (c - 1)) / 2;
  for (int c = tid; c < N; c += kPmThreads) {
    const int e0 = c * N - (c * (c - 1)) / 2;
    for (int e = e0; e < e0 + N - c; ++e) colof[e] = (uint8_t)c;
  }
  __syncthreads();
  // assembly: lower triangle of H_PP (float32) and B = -H_Pi (float64)
  for (int a = tid; a <= m; a += kPmThreads) {
    const int j = a < m ? S[a] : i;
    for (int p = up_ptr[j]; p < up_ptr[j + 1]; ++p) {
      const int l = up_col[p];
      const double* Hb = bsr + (int64_t)p * 12;  // H_jl, row r at Hb[4 r]
      if (a < m) {
        if (l == j) {
          for (int r = 0; r < 3; ++r)
            for (int c = 0; c <= r; ++c) L[pm_idx(N, 3 * a + c, 3 * a + r)] = (float)Hb[4 * r + c];
        } else if (l == i) {
          for (int r = 0; r < 3; ++r)
            for (int d = 0; d < 3; ++d) B[d * N + 3 * a + r] = -Hb[4 * r + d];
        } else {
          const int t = find_sorted(S, m, l);  // l > j, so t > a: the block sits below the diagonal
          if (t >= 0)
            for (int r = 0; r < 3; ++r)
              for (int c = 0; c < 3; ++c) L[pm_idx(N, 3 * a + r, 3 * t + c)] = (float)Hb[4 * r + c];
        }
      } else if (l != i) {
        const int t = find_sorted(S, m, l);  // row i: H_li = H_il^T
        if (t >= 0)
          for (int r = 0; r < 3; ++r)
            for (int d = 0; d < 3; ++d) B[d * N + 3 * t + r] = -Hb[4 * d + r];
      }
    }
  }
  __syncthreads();
  // right-looking Cholesky in shared memory, two barriers per column: every
  // thread takes the pivot from the (final) diagonal entry itself; the
  // factor's diagonal is kept aside in dg and written back at the end
  __shared__ float dg[kPmMaxN];
  for (int c = 0; c < N; ++c) {
    const float d = L[pm_idx(N, c, c)];
    const float piv = sqrtf(fmaxf(d, 1e-30f));
    if (tid == 0) {
      if (!(d > 0.0f)) bad = 1;
      dg[c] = piv;
    }
    for (int r = c + 1 + tid; r < N; r += kPmThreads) L[pm_idx(N, c, r)] /= piv;
    __syncthreads();
    // trailing update L(s, r) -= L(r, c) L(s, c), s > c, r >= s: the trailing
    // columns are contiguous in the packed layout, so the threads stride over
    // their elements evenly
    const float* Lc = L + cstart[c] - c;  // Lc[r] = L(r, c)
    for (int e = cstart[c + 1] + tid; e < nL; e += kPmThreads) {
      const int sc = colof[e];
      const int r = sc + (e - cstart[sc]);
      L[e] -= Lc[r] * Lc[sc];
    }
    __syncthreads();
  }
  for (int c = tid; c < N; c += kPmThreads) L[pm_idx(N, c, c)] = dg[c];
  __syncthreads();
  bool ok = bad == 0;
  // iterative refinement: R = B - H_PP Z (float64), D = (L L^T)^{-1} R (float32), Z += D
  bool settled = false;
  double prev = 1e300, ratio = 1e300;
  for (int it = 0; ok && it < kPmMaxIt && !settled; ++it) {
    for (int a = tid; a < m; a += kPmThreads) {
      double y[9];
      pm_apply_row(a, i, S, m, N, up_ptr, up_col, nbr_ptr, nbr_idx, bsr, Z, y);
      for (int r = 0; r < 3; ++r)
        for (int d = 0; d < 3; ++d) {
          R[d * N + 3 * a + r] = B[d * N + 3 * a + r] - y[3 * r + d];
          D[d * N + 3 * a + r] = (float)R[d * N + 3 * a + r];
        }
    }
    if (tid == 0) {
      dmax = 0.0;
      zmax = 0.0;
    }
    __syncthreads();
    // triangular solves, warp w < 3 for right-hand side w
    if (warp < 3) {
      float* y = D + warp * N;
      for (int c = 0; c < N; ++c) {
        if (lane == 0) y[c] /= L[pm_idx(N, c, c)];
        __syncwarp();
        const float yc = y[c];
        for (int r = c + 1 + lane; r < N; r += 32) y[r] -= L[pm_idx(N, c, r)] * yc;
        __syncwarp();
      }
      // L^T x = y as dot products down the columns of L (contiguous in the
      // packed layout): x_c = (y_c - sum_{r > c} L(r, c) x_r) / L(c, c)
      for (int c = N - 1; c >= 0; --c) {
        const float* Lc = L + cstart[c] - c;  // Lc[r] = L(r, c)
        float acc = 0.0f;
        for (int r = c + 1 + lane; r < N; r += 32) acc += Lc[r] * y[r];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) y[c] = (y[c] - acc) / Lc[c];
        __syncwarp();
      }
    }
    __syncthreads();
    double dl = 0.0, zl = 0.0;
    bool nonfinite = false;
    for (int k = tid; k < 3 * N; k += kPmThreads) {
      const double d = (double)D[k];
      Z[k] += d;
      nonfinite |= !isfinite(d) || !isfinite(Z[k]);  // fmax below would drop a NaN
      dl = fmax(dl, fabs(d));
      zl = fmax(zl, fabs(Z[k]));
    }
    if (nonfinite) bad = 1;  // float32 overflow in the triangular solves: the float64 kernel redoes the patch
    for (int o = 16; o > 0; o >>= 1) {
      dl = fmax(dl, __shfl_xor_sync(0xffffffffu, dl, o));
      zl = fmax(zl, __shfl_xor_sync(0xffffffffu, zl, o));
    }
    if (lane == 0) {
      atomicMax(reinterpret_cast<unsigned long long*>(&dmax), __double_as_longlong(dl));
      atomicMax(reinterpret_cast<unsigned long long*>(&zmax), __double_as_longlong(zl));
    }
    __syncthreads();
    const double dm = dmax, zm = zmax;
    ok = bad == 0;
    __syncthreads();
    if (!ok) break;
    settled = dm <= 1e-12 * zm;
    ratio = zm > 0.0 ? dm / zm : 0.0;
    if (dm > 0.5 * prev) break;  // corrections at the float64 rounding level of the residual
    prev = dm;
  }
  // accepted when the last correction is at most 1e-11 of z (the float64
  // solve's own rounding is about cond(H_PP) * 1e-16)
  if (!(ok && (settled || ratio <= 1e-11))) {
    if (tid == 0) redo[atomicAdd(n_redo, 1)] = i;
    return;
  }
  for (int k = tid; k < 9 * m; k += kPmThreads) {
    const int a = k / 9, q = k % 9, r = q / 3, d = q % 3;
    Uout[(int64_t)(s0 + a) * 9 + q] = Z[d * N + 3 * a + r];
  }
}
}  // namespace

int64_t patch_solves(Mesh& m, const int32_t* d_verts, int64_t count, bool throw_on_fail) {
  cudaStream_t s = m.stream;
  if (count <= 0) return 0;
  DBuf<int32_t> redo;
  m.last_patch_redo = count;
  if (3 * m.sup_max <= kPmMaxN) {
    // float32 factor + float64 refinement; the patches it hands back go to
    // the float64 kernel below
    redo.alloc(count + 1);
    CCG_CUDA(cudaMemsetAsync(redo.p + count, 0, sizeof(int32_t), s));
    const size_t smem = pm_smem_bytes();
    set_smem_limit(reinterpret_cast<const void*>(k_patch_basis_mixed), smem);
    k_patch_basis_mixed<<<(unsigned)count, kPmThreads, smem, s>>>(
        d_verts, m.d_sup_ptr.p, m.d_sup_idx.p, m.d_up_ptr.p, m.d_up_col.p, m.d_nbr_ptr.p, m.d_nbr_idx.p,
        m.f64.bsr.p, m.f64.U.p, redo.p, redo.p + count);
    CCG_CUDA(cudaGetLastError());
    int32_t nr = 0;
    CCG_CUDA(cudaMemcpyAsync(&nr, redo.p + count, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CCG_CUDA(cudaStreamSynchronize(s));
    m.last_patch_redo = nr;
    if (nr == 0) return 0;
    d_verts = redo.p;
    count = nr;
  }
  const int Nmax = 3 * std::max(m.sup_max, 1);
  const size_t per = (size_t)Nmax * Nmax + 3 * (size_t)Nmax;
  int64_t batch = std::max<int64_t>(1, (int64_t)((size_t(1) << 30) / (per * sizeof(double))));
  batch = std::min<int64_t>(batch, count);
  DBuf<double> scratch;
  scratch.alloc(per * std::max<int64_t>(batch, 1));
  DBuf<int32_t> fail;
  fail.alloc(1);
  CCG_CUDA(cudaMemsetAsync(fail.p, 0, sizeof(int32_t), s));
  for (int64_t b0 = 0; b0 < count; b0 += batch) {
    const int64_t cnt = std::min<int64_t>(batch, count - b0);
    k_patch_basis<<<(unsigned)cnt, 256, 0, s>>>(d_verts + b0, m.d_sup_ptr.p, m.d_sup_idx.p, m.d_up_ptr.p,
                                                 m.d_up_col.p, m.f64.bsr.p, Nmax, scratch.p, m.f64.U.p, fail.p);
    CCG_CUDA(cudaGetLastError());
  }
  int32_t nfail = 0;
  CCG_CUDA(cudaMemcpyAsync(&nfail, fail.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CCG_CUDA(cudaStreamSynchronize(s));
  CCG_CHECK(nfail == 0 || !throw_on_fail, CC_ERR_NUMERIC, "a patch Hessian was not positive definite");
  return nfail;
}

namespace {
__global__ void k_f64_to_f32(const double* __restrict__ a, int64_t count, float* __restrict__ b) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x)
    b[k] = (float)a[k];
}
}  // namespace

// float32 copy of the float64 bases (used by the mixed-precision sweep).
void bases_to_f32(Mesh& m) {
  const int64_t count = 9 * (int64_t)m.sup_idx.size();
  if (count == 0) return;
  const unsigned grid = (unsigned)std::min<int64_t>((count + 255) / 256, 152 * 16);
  k_f64_to_f32<<<grid, 256, 0, m.stream>>>(m.f64.U.p, count, m.mx.U.p);
  CCG_CUDA(cudaGetLastError());
}

namespace {

__device__ __forceinline__ uint64_t sig_mix(uint64_t tag, uint64_t idx, uint64_t v) {
  // SplitMix64's output function (Steele, Lea and Flood 2014) on a keyed word
  uint64_t z = v + 0x9E3779B97F4A7C15ull * (tag * 0x100000001B3ull + idx + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Signature of vertex i's patch, one warp per listed vertex: the support as
// offsets from i with each support vertex's tet count, i's 1-ring (offsets,
// rest positions relative to X_i as bit patterns, pinned flags) and the
// material of i's first tet, summed as keyed
// 64-bit mixes (order-free, so the warp's partial sums combine exactly).
// Equal signatures only propose that two patches are translated copies.
__global__ void k_patch_signature(const int32_t* __restrict__ verts, int64_t count, const int32_t* __restrict__ sup_ptr,
                                  const int32_t* __restrict__ sup_idx, const int32_t* __restrict__ nbr_ptr,
                                  const int32_t* __restrict__ nbr_idx, const double* __restrict__ Xr, int64_t n,
                                  const uint8_t* __restrict__ pinned, const int32_t* __restrict__ vt_ptr,
                                  const int32_t* __restrict__ vt_tet, const double2* __restrict__ mat,
                                  unsigned long long* __restrict__ sig) {
  const int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= count) return;
  const int i = verts[k];
  const int s0 = sup_ptr[i], m = sup_ptr[i + 1] - s0;
  const int e0 = nbr_ptr[i], ne = nbr_ptr[i + 1] - e0;
  uint64_t h = 0;
  for (int a = lane; a < m; a += 32) {
    // the support vertex's offset and tet count (a support vertex on the
    // mesh surface has a different block row than one inside)
    const int j = sup_idx[s0 + a];
    h += sig_mix(1, a, (uint64_t)(uint32_t)(j - i));
    h += sig_mix(9, a, (uint64_t)(vt_ptr[j + 1] - vt_ptr[j]));
  }
  for (int e = lane; e < ne; e += 32) {
    const int l = nbr_idx[e0 + e];
    h += sig_mix(2, e, (uint64_t)(uint32_t)(l - i));
#pragma unroll
    for (int c = 0; c < 3; ++c)
      h += sig_mix(3 + c, e, (uint64_t)__double_as_longlong(Xr[c * n + l] - Xr[c * n + i]));
    h += sig_mix(6, e, pinned[l]);
  }
  if (lane == 0) {
    h += sig_mix(7, (uint64_t)m, (uint64_t)ne);
    const double2 mt = mat[vt_tet[vt_ptr[i]]];
    h += sig_mix(8, 0, (uint64_t)__double_as_longlong(mt.x)) + sig_mix(8, 1, (uint64_t)__double_as_longlong(mt.y));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
  if (lane == 0) sig[k] = h;
}

// U_v = U_rep (block for block) for the pairs (v, rep) of equal support size;
// a pair whose sizes differ is flagged in bad[] and copies nothing.
__global__ void k_copy_bases(const int32_t* __restrict__ dst_v, const int32_t* __restrict__ src_v, int64_t count,
                             const int32_t* __restrict__ sup_ptr, double* __restrict__ U, int32_t* __restrict__ bad) {
  const int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= count) return;
  const int v = dst_v[k], r = src_v[k];
  const int m = sup_ptr[v + 1] - sup_ptr[v];
  if (m != sup_ptr[r + 1] - sup_ptr[r]) {
    if (lane == 0) bad[k] = 1;
    return;
  }
  const double* src = U + 9 * (int64_t)sup_ptr[r];
  double* dst = U + 9 * (int64_t)sup_ptr[v];
  for (int q = lane; q < 9 * m; q += 32) dst[q] = src[q];
}

}  // namespace

int64_t patch_solves_shared(Mesh& m, const int32_t* d_verts, int64_t count, bool throw_on_fail) {
  cudaStream_t s = m.stream;
  m.last_patch_shared = 0;
  m.last_patch_solved = count;
  if (count < 1024) return patch_solves(m, d_verts, count, throw_on_fail);
  if (!m.d_Xrest.p) {
    std::vector<double> soa(3 * m.n);
    for (int64_t j = 0; j < m.n; ++j)
      for (int a = 0; a < 3; ++a) soa[a * m.n + j] = m.X[3 * j + a];
    m.d_Xrest.upload(soa, s);
    CCG_CUDA(cudaStreamSynchronize(s));
  }
  DBuf<unsigned long long> sig;
  sig.alloc(count);
  k_patch_signature<<<(unsigned)((count * 32 + 255) / 256), 256, 0, s>>>(
      d_verts, count, m.d_sup_ptr.p, m.d_sup_idx.p, m.d_nbr_ptr.p, m.d_nbr_idx.p, m.d_Xrest.p, m.n, m.d_pinned.p,
      m.d_vt_ptr.p, m.d_vt_tet.p, m.d_mat64.p, sig.p);
  CCG_CUDA(cudaGetLastError());
  std::vector<unsigned long long> hs(count);
  std::vector<int32_t> hv(count);
  CCG_CUDA(cudaMemcpyAsync(hs.data(), sig.p, count * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  CCG_CUDA(cudaMemcpyAsync(hv.data(), d_verts, count * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CCG_CUDA(cudaStreamSynchronize(s));
  // the first listed vertex of every signature solves; the others copy it
  std::vector<int64_t> order(count);
  for (int64_t k = 0; k < count; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return hs[a] < hs[b]; });
  std::vector<int32_t> reps, mem_v, mem_r, mem_ri;
  for (int64_t q = 0; q < count;) {
    int64_t e = q;
    while (e < count && hs[order[e]] == hs[order[q]]) ++e;
    const int32_t r = hv[order[q]];
    for (int64_t t = q + 1; t < e; ++t) {
      mem_v.push_back(hv[order[t]]);
      mem_r.push_back(r);
      mem_ri.push_back((int32_t)reps.size());
    }
    reps.push_back(r);
    q = e;
  }
  if ((int64_t)mem_v.size() * 4 < count) return patch_solves(m, d_verts, count, throw_on_fail);  // little to share
  DBuf<int32_t> d_reps, d_mv, d_mr, d_bad;
  d_reps.upload(reps, s);
  int64_t fails = patch_solves(m, d_reps.p, (int64_t)reps.size(), throw_on_fail);
  const int64_t nm = (int64_t)mem_v.size();
  d_mv.upload(mem_v, s);
  d_mr.upload(mem_r, s);
  d_bad.alloc(nm);
  CCG_CUDA(cudaMemsetAsync(d_bad.p, 0, nm * sizeof(int32_t), s));
  k_copy_bases<<<(unsigned)((nm * 32 + 255) / 256), 256, 0, s>>>(d_mv.p, d_mr.p, nm, m.d_sup_ptr.p, m.f64.U.p,
                                                                 d_bad.p);
  CCG_CUDA(cudaGetLastError());
  // every copied basis must solve its own patch's Eq. 5 as well as it solves
  // the patch it was computed on: a translated copy (bitwise equal H_PP,
  // H_Pi) reproduces its source's residual, while a patch that differs even
  // in the last digits of its geometry leaves a residual of that size
  const int64_t nr = (int64_t)reps.size();
  DBuf<double> rho, rho_r;
  rho.alloc(nm);
  rho_r.alloc(nr);
  basis_residuals(m, d_mv.p, nm, rho.p, s);
  basis_residuals(m, d_reps.p, nr, rho_r.p, s);
  std::vector<double> hr(nm), hrr(nr);
  std::vector<int32_t> hb(nm);
  CCG_CUDA(cudaMemcpyAsync(hr.data(), rho.p, nm * sizeof(double), cudaMemcpyDeviceToHost, s));
  CCG_CUDA(cudaMemcpyAsync(hrr.data(), rho_r.p, nr * sizeof(double), cudaMemcpyDeviceToHost, s));
  CCG_CUDA(cudaMemcpyAsync(hb.data(), d_bad.p, nm * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CCG_CUDA(cudaStreamSynchronize(s));
  std::vector<int32_t> own;
  for (int64_t k = 0; k < nm; ++k)
    if (hb[k] || !(hr[k] <= std::max(1e-10, 4.0 * hrr[mem_ri[k]]))) own.push_back(mem_v[k]);
  if (!own.empty()) {
    DBuf<int32_t> d_own;
    d_own.upload(own, s);
    fails += patch_solves(m, d_own.p, (int64_t)own.size(), throw_on_fail);
  }
  m.last_patch_shared = nm - (int64_t)own.size();
  m.last_patch_solved = (int64_t)reps.size() + (int64_t)own.size();
  return fails;
}

void run_subspace_build(Mesh& m, int32_t k) {
  build_supports(m, k);
  rest_hessian_f64(m);
  patch_solves_shared(m, m.d_free_rows.p, m.n_free, true);
  bases_to_f32(m);
  CCG_CUDA(cudaStreamSynchronize(m.stream));
}

}  // namespace ccg
