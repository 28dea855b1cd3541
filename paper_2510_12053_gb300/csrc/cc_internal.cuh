// Internal declarations of the GB300 Coordinate Condensation library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <functional>
#include <new>
#include <utility>
#include <string>
#include <vector>

#include "../../include/cc.h"

namespace ccg {

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);

struct Fail {
  cc_status st;
};

#define CCG_CUDA(call)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      ::ccg::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));               \
      throw ::ccg::Fail{e_ == cudaErrorMemoryAllocation ? CC_ERR_OOM : CC_ERR_CUDA};      \
    }                                                                                      \
  } while (0)

#define CCG_CHECK(cond, status, msg)      \
  do {                                    \
    if (!(cond)) {                        \
      ::ccg::set_error(msg);              \
      throw ::ccg::Fail{status};          \
    }                                     \
  } while (0)

// ---------------------------------------------------------------------------
// Device buffers owned by a mesh
// ---------------------------------------------------------------------------
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t count = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), count(o.count) {
    o.p = nullptr;
    o.count = 0;
  }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p;
      count = o.count;
      o.p = nullptr;
      o.count = 0;
    }
    return *this;
  }
  ~DBuf() { release(); }
  void alloc(size_t c) {
    release();
    if (c == 0) c = 1;
    CCG_CUDA(cudaMalloc((void**)&p, c * sizeof(T)));
    count = c;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    count = 0;
  }
  void upload(const T* h, size_t c, cudaStream_t s) {
    alloc(c);
    if (c) CCG_CUDA(cudaMemcpyAsync(p, h, c * sizeof(T), cudaMemcpyHostToDevice, s));
  }
  template <typename V>
  void upload(const std::vector<V>& v, cudaStream_t s) {
    upload(reinterpret_cast<const T*>(v.data()), v.size() * sizeof(V) / sizeof(T), s);
  }
};

// Per-tet Hessian store: a tet's ten upper 3x3 blocks, corner pairs (a, b)
// with a <= b in the order (0,0) (0,1) (0,2) (0,3) (1,1) (1,2) (1,3) (2,2)
// (2,3) (3,3).  The four diagonal blocks are symmetric and keep their upper
// triangles (6 values: (0,0) (0,1) (0,2) (1,1) (1,2) (2,2)), the six others
// all 9 values row-major: 78 values, kTetStore per tet.
constexpr int kTetStore = 80;
// Codes allocated past the end of a slot map (zeroed): the coupling kernel
// copies a vertex's map in 4-byte words from the word holding its first code,
// which reads up to 3 codes past the map's end.
constexpr int kSlotMapSlack = 8;
constexpr bool tet_pair_is_diag(int pair) { return pair == 0 || pair == 4 || pair == 7 || pair == 9; }
// first value of a pair's block in the tet's record
constexpr int tet_pair_offset(int pair) {
  int o = 0;
  for (int p = 0; p < pair; ++p) o += tet_pair_is_diag(p) ? 6 : 9;
  return o;
}
static_assert(tet_pair_offset(5) == 39 && tet_pair_offset(10) == 78, "per-tet store layout");

// Per-precision solver state: per-(vertex, incident-tet) contributions, the
// assembled gradient and 3x3-block Hessian, and the basis blocks.
struct StateF64 {
  DBuf<double> gcon;  // [4T][3]   gradient of tet at each (vertex, slot)
  DBuf<double> hten;  // [T][kTetStore]  the tet's 10 upper 3x3 Hessian blocks (corner pairs a <= b)
  DBuf<double> g;     // [n][3]
  DBuf<double> bsr;   // [nnz_up][12] upper Hessian blocks, rows padded to 4
  DBuf<double> U;     // [sup_total][9]
  DBuf<double> cpl;   // [n_free][32] coupling products of the vertices being solved
  DBuf<double> rot;   // [n][9] per-vertex rotations of corotated bases
};

struct StateMixed {
  DBuf<float2> gcon;  // [4T][3]   float-float (hi, lo)
  DBuf<float> hten;   // [T][kTetStore]
  DBuf<float> g_hi;   // [n][3]
  DBuf<float> g_lo;   // [n][3]
  DBuf<float> bsr;    // [nnz_up][12]
  DBuf<float> U;      // [sup_total][9]
  DBuf<float> cpl;    // [n_free][32]
  DBuf<float> rot;    // [n][9] per-vertex rotations of corotated bases
  DBuf<float4> x_hi;  // [n] position mirror, float-float split
  DBuf<float4> x_lo;
  DBuf<float4> xt_hi; // inertial target mirror
  DBuf<float4> xt_lo;
};

// Optional per-kernel-class event timing (cc_profile_*).  Intervals recorded
// while a graph is being captured become event nodes of that graph; their
// times are added up after every replay.
struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<int> mark_cls, mark_begin, mark_end, mark_launches;
  int64_t total_launches = 0;
  bool capturing = false;
  std::vector<cudaEvent_t> gpool;
  std::vector<int> gmark_cls, gmark_begin, gmark_end, gmark_launches;
  int64_t graph_launches = 0;    // kernel launches per replay of the current graph
  double acc_ms[CC_PROFILE_CLASSES] = {0, 0, 0, 0, 0};
  int64_t acc_launches[CC_PROFILE_CLASSES] = {0, 0, 0, 0, 0};
};

// Raises a kernel's dynamic shared-memory limit once per (kernel, device):
// the attribute call costs host time and is not repeated on every launch.
void set_smem_limit(const void* kernel, size_t bytes);

struct Mesh {
  Prof prof;
  // launch configurations chosen by cc_autotune (defaults before tuning)
  int tune_couple_threads = 64;   // threads per vertex in the coupling kernel (32: one warp)
  int tune_couple_row_lanes = 4;  // threads per block row in the coupling kernel (1, 2, 4, 8)
  int tune_gather_wpb = 4;        // warps (rows) per block in the row gather
  bool fused_condense = false;    // the coupling kernel's last CTA of every 32 vertices condenses them
  bool rows_build = false;        // mixed stable Neo-Hookean rows formed from the positions (k_row_build)
  int64_t n = 0, T = 0, n_free = 0, nnzb = 0;
  int32_t max_valence = 0;
  double E = 0, nu = 0, rho = 0, mu = 0, lam_hat = 0, h = 0;
  int model = CC_MODEL_SNH;   // energy density (per mesh; batches share it)
  double grav[3] = {0, 0, 0};
  cudaStream_t stream = nullptr;

  // host copies (setup, export)
  std::vector<double> X;       // [n][3]
  std::vector<int32_t> tets;   // [T][4] positively oriented
  std::vector<uint8_t> pinned; // [n]
  std::vector<int64_t> vt_ptr;
  std::vector<int32_t> vt_tet, vt_corner;
  std::vector<int64_t> nbr_ptr;
  std::vector<int32_t> nbr_idx;
  std::vector<int64_t> up_ptr;   // upper 3x3-block pattern (diagonal first)
  std::vector<int32_t> up_col;
  int64_t nnz_up = 0;
  int32_t max_up = 0;          // longest upper block row
  int32_t max_rs = 0;          // most staged sources of one free row
  int64_t last_patch_redo = 0; // patches the last mixed patch solve handed to the float64 kernel
  int64_t last_patch_shared = 0; // bases the last build copied from an identical patch (no solve of their own)
  int64_t last_patch_solved = 0; // patches the last build solved
  std::vector<double> mass;
  std::vector<double> tet_mu, tet_lh, tet_rho;   // per-tet material (a batch mixes materials);
                                                 // tet_lh = lam + mu (stable Neo-Hookean) or lam (FCR)
  std::vector<double> tet_E, tet_nu;             // the same as given (Young's modulus, Poisson ratio)
  // batches: mesh b owns vertices [mesh_vptr[b], mesh_vptr[b+1]) and tets [mesh_tptr[b], mesh_tptr[b+1])
  std::vector<int64_t> mesh_vptr, mesh_tptr;
  std::vector<int32_t> mesh_fptr;                // free rows of mesh b: [mesh_fptr[b], mesh_fptr[b+1])
  DBuf<int32_t> d_vert_mesh;                     // [n] mesh of every vertex
  DBuf<int32_t> d_mesh_fptr;                     // [B+1]
  DBuf<int32_t> d_mesh_active;                   // [B] 1 while the mesh is still being solved
  DBuf<int32_t> d_mesh_ones;                     // [B] all ones (resets d_mesh_active)
  DBuf<double> d_mesh_gsq;                       // [B] squared free gradient norm per mesh
  DBuf<int64_t> d_mesh_vptr, d_mesh_tptr;        // [B+1] vertex and tet ranges (per-mesh energy)
  DBuf<double> d_mesh_energy;                    // [B] per-mesh energy (batched line search)
  DBuf<double> d_mesh_alpha;                     // [B] per-mesh line search step
  std::vector<int32_t> color;
  int32_t num_colors = 0;
  std::vector<int64_t> sup_ptr;
  std::vector<int32_t> sup_idx;
  int32_t k_ring = 0;
  int32_t sup_max = 0;
  int32_t hash_size = 0;       // unused (kept for layout stability)
  int64_t smap_max = 0;        // longest per-vertex slot map
  bool smap_wide = false;      // slot maps in uint16 (supports of 250+ vertices)

  // device rest data
  DBuf<int4> d_tets;
  DBuf<int4> d_tslot;        // [T] global (vertex, slot) entry of each corner
  DBuf<double> d_Bm;         // [T][9] D_m^{-1}, row-major (row c = shape vector of corner c+1)
  DBuf<float2> d_Bm_df;      // [T][9] float-float copy
  DBuf<float> d_Bm32;        // [T][9]
  DBuf<float> d_Bm32p;       // [T][3][4] rows padded to four (row build)
  DBuf<double> d_vol;        // [T]
  DBuf<double2> d_mat64;     // [T] (mu, lam_hat) of the tet's material
  DBuf<float4> d_matdf;      // [T] (mu hi, mu lo, lam_hat hi, lam_hat lo)
  DBuf<double> d_volw;       // [T] vol * elastic weight (h^2 or 1), float64
  DBuf<float> d_volw32;      // [T] same, float32
  DBuf<float2> d_volw_df;    // [T] same, float-float
  DBuf<double> d_mass;       // [n]
  DBuf<float> d_mass32;      // [n]
  DBuf<float2> d_mass_df;    // [n]
  DBuf<uint8_t> d_pinned;    // [n]
  DBuf<int32_t> d_vt_ptr;    // [n+1]
  DBuf<int32_t> d_nbr_ptr;   // [n+1]
  DBuf<int32_t> d_nbr_idx;
  DBuf<int32_t> d_vt_tet;    // [4T]
  DBuf<uint8_t> d_vt_corner; // [4T]
  DBuf<int32_t> d_up_ptr;    // [n+1] upper block rows
  DBuf<int32_t> d_up_col;    // [nnz_up]
  DBuf<int32_t> d_rs_ptr;    // [nnz_up+1] sources of each upper block (free rows)
  DBuf<int32_t> d_rs_src;    // per-tet store offset of each source, bit 31 = transpose
  DBuf<uint16_t> d_rs_loc;   // the same sources as row-local codes k * 4 + w (row build)
  DBuf<int32_t> d_free_rows; // free vertices, ascending
  DBuf<int4> d_row_hdr;      // [2 n_free] row gather records: (j, p0, nup, rb), (rcount, e0, val, 0)
  DBuf<int32_t> d_color;     // [n]
  std::vector<int32_t> cv_ptr;  // [C+1] free vertices per colour
  DBuf<int32_t> d_cv_idx;
  std::vector<int32_t> tl_ptr;  // [C+1] tets with a free vertex of colour c
  DBuf<int32_t> d_tl;
  DBuf<int32_t> d_all_tets;     // tets with at least one free vertex
  int64_t n_active_tets = 0;
  DBuf<int32_t> d_sup_ptr;   // [n+1]
  DBuf<int32_t> d_sup_idx;
  // Slot maps of the coupling kernel: for free vertex i, one code per upper
  // block of each support row and of row i (in support order, row i last):
  // the block column's slot in S_i, or kSlotNone / kSlotSelf (column i) /
  // kSlotDiag (the row's diagonal block).
  DBuf<int64_t> d_smap_ptr;  // [n+1]
  DBuf<uint8_t> d_smap8;
  DBuf<uint16_t> d_smap16;
  DBuf<int4> d_vt_ids;       // [4T] vertex ids of the tet at each (vertex, slot) entry
  DBuf<double> d_Xrest;      // [3][n] rest positions (uploaded on first use)
  bool rot_active = false;   // the current sweep uses corotated bases

  StateF64 f64;
  StateMixed mx;

  // scratch
  DBuf<double> d_red;        // reduction partials
  DBuf<double> d_scalars;    // [8]
  DBuf<unsigned long long> d_counters; // [4] fallback counters + [4] error flags
  DBuf<int32_t> d_grp_cnt;   // arrivals per 32-vertex group of the fused coupling + condensation (self-resetting)
  DBuf<double> d_xtilde;     // [3][n] dynamic target (solve_step)
  DBuf<double> d_xold;       // [3][n]
  DBuf<double> d_xls0;       // [3][n] line search: x before the sweep
  DBuf<double> d_xls1;       // [3][n] line search: x after the sweep
  double* h_pinned_scalars = nullptr; // pinned host [8]
  cudaGraphExec_t graph_exec = nullptr;
  std::string graph_key;
};

// ---------------------------------------------------------------------------
// Programmatic dependent launch (opt-in, see pdl_enabled).  A kernel started
// by pdl_launch may be scheduled while its predecessor in the stream is still
// finishing: its
// launch and CTA dispatch overlap the predecessor's tail.  Every such kernel
// begins with pdl_entry(): it lets its own successor be scheduled once all of
// its CTAs have started, then waits until the predecessor has completed and
// its writes are visible, before touching global memory (for an ordinary
// launch the wait returns at once).  Because each kernel waits for the
// previous one, completion is transitive along the stream.
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_entry() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
#endif

bool pdl_enabled();  // true when CC_GB300_PDL is set in the environment (default: ordinary launches)

// The mixed path of the stable Neo-Hookean material forms its float32 block
// rows from the positions (k_row_build) instead of a per-tet Hessian store;
// the float64 path and Fixed Corotational keep the store (FCR's blocks need
// the polar rotation, too costly to form four times per tet).
// The coupling kernel condenses its vertices itself (one launch per colour
// for the local solves) unless switched off or with the one-warp coupling kernel.
inline bool fused_local_solve(const Mesh& m, cc_update upd) {
  return upd != CC_UPDATE_CD && m.fused_condense && m.tune_couple_threads != 32;
}

inline bool rows_from_positions(const Mesh& m) {
  return m.rows_build && m.model == CC_MODEL_SNH && m.max_valence <= 64;
}

template <typename... KArgs, typename... Args>
void pdl_launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  CCG_CUDA(cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...));
}

// ---------------------------------------------------------------------------
// Host-side helpers implemented in mesh_build.cpp (topology, plain C++)
// ---------------------------------------------------------------------------
void build_topology(Mesh& m);
// Slot maps for the current supports (after cc_build_subspace / cc_set_subspace;
// kernels_setup.cu, built on the device: d_sup_ptr / d_sup_idx must be uploaded).
void build_slot_maps(Mesh& m);
// host worker threads for setup passes, and a parallel loop over vertex ranges
int host_threads(int64_t items);
void parallel_ranges(int64_t n, int nt, const std::function<void(int, int64_t, int64_t)>& f);

// ---------------------------------------------------------------------------
// Kernel launchers (kernels_*.cu)
// ---------------------------------------------------------------------------
struct SweepCounters {
  unsigned long long* fallback;  // [3] empty, reduced, schur
  unsigned long long* error;     // [1] non-finite update seen
};

// phase A: per-tet gradient contributions of a tet list -> (vertex, slot) entries
void launch_tet_grad_f64(Mesh& m, const double* x, const int32_t* list, int64_t count, double weight,
                         cudaStream_t s);
void launch_tet_grad_mixed(Mesh& m, const int32_t* list, int64_t count, double weight, cudaStream_t s);
// phase B: gradient and upper Hessian block rows of every free vertex
void launch_rows_f64(Mesh& m, const double* x, const double* xt, double weight, cudaStream_t s);
void launch_rows_mixed(Mesh& m, double weight, cudaStream_t s);
// local solves for a list of free vertices
void launch_local_solve_f64(Mesh& m, cc_update upd, const int32_t* verts, int64_t count,
                            double* x, SweepCounters c, cudaStream_t s);
void launch_local_solve_mixed(Mesh& m, cc_update upd, const int32_t* verts, int64_t count,
                              double* x, SweepCounters c, cudaStream_t s);
// per-vertex rotations of the corotated bases at x (float64 or float32 result)
void launch_rotations(Mesh& m, const double* x, bool mixed, cudaStream_t s);
// reductions
void launch_energy(Mesh& m, const double* x, const double* xt, double* out_scalar,
                   cudaStream_t s);
void launch_gnorm_f64(Mesh& m, double* grad_out, double* out_scalar, cudaStream_t s);
void launch_gnorm_mixed(Mesh& m, double* grad_out, double* out_scalar, cudaStream_t s);
void launch_gnorm_mesh(Mesh& m, bool mixed, cudaStream_t s);  // per-mesh squared norms -> d_mesh_gsq
// per-mesh energies of a batch -> out[B]; per-mesh line points x = x0 + alpha_b (x1 - x0)
void launch_energy_mesh(Mesh& m, const double* x, const double* xt, double* out, cudaStream_t s);
void launch_line_point_mesh(Mesh& m, const double* x0, const double* x1, const double* alpha, double* x,
                            cudaStream_t s);
// mirrors and small vector ops
void launch_split_df(const double* x, int64_t n, float4* hi, float4* lo, cudaStream_t s);
void launch_inertial_target(const double* x, const double* v, int64_t n, double h,
                            const double* grav, double* xt, cudaStream_t s);
void launch_velocity(const double* x, const double* xold, int64_t n, double h, double* v,
                     cudaStream_t s);
// x = x0 + alpha (x1 - x0), all 3n entries (line search trial point)
void launch_line_point(const double* x0, const double* x1, int64_t n, double alpha, double* x, cudaStream_t s);
// colouring and subspace build
void run_coloring(Mesh& m);
// a caller's colouring (validated: colours in [0, C), no two vertices of a
// tet alike), then the per-colour vertex and tet lists
void set_coloring(Mesh& m, const int32_t* colors, int32_t C);
void build_color_lists(Mesh& m);
void run_subspace_build(Mesh& m, int32_t k);
void build_supports(Mesh& m, int32_t k);
void rest_hessian_f64(Mesh& m);
void hessian_f64_at(Mesh& m, const double* x);
// U_i = -H_PP^{-1} H_Pi for the listed vertices from the float64 block rows:
// float32 factor + float64 refinement where the patch fits (<= 192 unknowns),
// float64 Cholesky otherwise; returns the patches that were not positive
// definite (their bases untouched), or throws when throw_on_fail.
int64_t patch_solves(Mesh& m, const int32_t* d_verts, int64_t count, bool throw_on_fail);
int64_t rebuild_bases_at(Mesh& m, const double* x);
// Eq. 5 residuals of the float64 bases of a device vertex list (mlp.cu)
void basis_residuals(Mesh& m, const int32_t* d_rows, int64_t count, double* rho, cudaStream_t s);
// Patch solves of a vertex list that share one solve between vertices with
// identical patches (translated copies on regular grids); every shared basis
// is checked against its own Eq. 5 and re-solved on its own if it fails.
int64_t patch_solves_shared(Mesh& m, const int32_t* d_verts, int64_t count, bool throw_on_fail);
void bases_to_f32(Mesh& m);
// solver state of one precision (allocated once, on first use)
void ensure_state(Mesh& m, cc_precision p);
// forgets the captured sweep graph (its nodes hold buffer pointers)
void drop_graph(Mesh& m);
void clear_error();
bool error_empty();

// Body of a C entry point: runs the statements, maps exceptions to status codes.
#define CC_API_BODY(name, ...)                                              \
  try {                                                                      \
    ::ccg::clear_error();                                                    \
    __VA_ARGS__;                                                             \
    return CC_OK;                                                            \
  } catch (const ::ccg::Fail& f) {                                           \
    if (::ccg::error_empty()) ::ccg::set_error(name);                        \
    return f.st;                                                             \
  } catch (const std::bad_alloc&) {                                          \
    ::ccg::set_error(std::string(name) + ": host out of memory");            \
    return CC_ERR_OOM;                                                       \
  } catch (...) {                                                            \
    ::ccg::set_error(std::string(name) + ": unexpected error");              \
    return CC_ERR_STATE;                                                     \
  }

}  // namespace ccg
