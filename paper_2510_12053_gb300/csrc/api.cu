// C ABI entry points (include/cc.h): argument checks, state management and
// the order of kernel launches for sweeps and solves.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <system_error>
#include <thread>
#include <vector>

#include "cc_internal.cuh"
#include "mlp.cuh"

namespace ccg {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }

bool pdl_enabled() {
  // opt-in: measured no gain on the sweep (32^3 cube: 861 us per sweep with it, 816 without)
  static const bool on = std::getenv("CC_GB300_PDL") != nullptr;
  return on;
}
bool error_empty() { return g_last_error.empty(); }

void set_smem_limit(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> done;
  if (bytes <= 48 * 1024) return;
  int dev = 0;
  CCG_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  size_t& have = done[{dev, kernel}];
  if (have >= bytes) return;
  CCG_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  have = bytes;
}

void drop_graph(Mesh& m) {
  if (m.graph_exec) cudaGraphExecDestroy(m.graph_exec);
  m.graph_exec = nullptr;
  m.graph_key.clear();
  for (cudaEvent_t e : m.prof.gpool) cudaEventDestroy(e);
  m.prof.gpool.clear();
  m.prof.gmark_cls.clear();
  m.prof.gmark_begin.clear();
  m.prof.gmark_end.clear();
  m.prof.gmark_launches.clear();
  m.prof.graph_launches = 0;
}

void ensure_state(Mesh& m, cc_precision p) {
  cudaStream_t s = m.stream;
  const size_t ne = 4 * (size_t)m.T;
  if (!m.d_grp_cnt.p) {  // arrival counters of the fused local solves (they reset themselves)
    m.d_grp_cnt.alloc((size_t)(m.n_free + 31) / 32 + 1);
    CCG_CUDA(cudaMemsetAsync(m.d_grp_cnt.p, 0, m.d_grp_cnt.count * sizeof(int32_t), s));
  }
  if (p == CC_PREC_FP64) {
    if (!m.f64.gcon.p) {
      m.f64.gcon.alloc(3 * ne);
      m.f64.hten.alloc(kTetStore * (size_t)m.T);
      m.f64.g.alloc(3 * m.n);
      m.f64.bsr.alloc(12 * m.nnz_up);
      m.f64.cpl.alloc(32 * m.n_free);
      CCG_CUDA(cudaMemsetAsync(m.f64.g.p, 0, 3 * m.n * sizeof(double), s));
    }
  } else {
    if (!m.mx.gcon.p) {
      m.mx.gcon.alloc(3 * ne);
      m.mx.g_hi.alloc(3 * m.n);
      m.mx.g_lo.alloc(3 * m.n);
      m.mx.bsr.alloc(12 * m.nnz_up);
      m.mx.cpl.alloc(32 * m.n_free);
      m.mx.x_hi.alloc(m.n);
      m.mx.x_lo.alloc(m.n);
      m.mx.xt_hi.alloc(m.n);
      m.mx.xt_lo.alloc(m.n);
      CCG_CUDA(cudaMemsetAsync(m.mx.g_hi.p, 0, 3 * m.n * sizeof(float), s));
      CCG_CUDA(cudaMemsetAsync(m.mx.g_lo.p, 0, 3 * m.n * sizeof(float), s));
      CCG_CUDA(cudaMemsetAsync(m.mx.xt_hi.p, 0, m.n * sizeof(float4), s));
      CCG_CUDA(cudaMemsetAsync(m.mx.xt_lo.p, 0, m.n * sizeof(float4), s));
    }
    // the per-tet Hessian store exists only for the gather path
    if (!rows_from_positions(m) && !m.mx.hten.p) m.mx.hten.alloc(kTetStore * (size_t)m.T);
  }
}

namespace {

enum { P_TET = 0, P_GATHER = 1, P_SOLVE = 2, P_RED = 3, P_OTHER = 4 };

int prof_event(Mesh& m) {
  if (!m.prof.on) return -1;
  if (m.prof.capturing) {
    cudaEvent_t e;
    CCG_CUDA(cudaEventCreate(&e));
    m.prof.gpool.push_back(e);
    CCG_CUDA(cudaEventRecord(e, m.stream));
    return (int)m.prof.gpool.size() - 1;
  }
  if (m.prof.used == m.prof.pool.size()) {
    cudaEvent_t e;
    CCG_CUDA(cudaEventCreate(&e));
    m.prof.pool.push_back(e);
  }
  const int k = (int)m.prof.used++;
  CCG_CUDA(cudaEventRecord(m.prof.pool[k], m.stream));
  return k;
}

// Counts `launches` kernels of class `cls`; with timing on, records the
// closing event of an interval opened by prof_event.
void prof_close(Mesh& m, int cls, int begin, int launches) {
  if (m.prof.capturing) {
    m.prof.graph_launches += launches;
    if (!m.prof.on || begin < 0) return;
    const int end = prof_event(m);
    m.prof.gmark_cls.push_back(cls);
    m.prof.gmark_begin.push_back(begin);
    m.prof.gmark_end.push_back(end);
    m.prof.gmark_launches.push_back(launches);
    return;
  }
  m.prof.total_launches += launches;
  if (!m.prof.on || begin < 0) return;
  const int end = prof_event(m);
  m.prof.mark_cls.push_back(cls);
  m.prof.mark_begin.push_back(begin);
  m.prof.mark_end.push_back(end);
  m.prof.mark_launches.push_back(launches);
}

// After a completed graph replay: adds the replay's launches and, with timing
// on, the intervals between its captured event nodes.
void prof_after_replay(Mesh& m) {
  m.prof.total_launches += m.prof.graph_launches;
  if (!m.prof.on) return;
  for (size_t k = 0; k < m.prof.gmark_cls.size(); ++k) {
    float ms = 0.f;
    CCG_CUDA(cudaEventElapsedTime(&ms, m.prof.gpool[m.prof.gmark_begin[k]], m.prof.gpool[m.prof.gmark_end[k]]));
    m.prof.acc_ms[m.prof.gmark_cls[k]] += ms;
    m.prof.acc_launches[m.prof.gmark_cls[k]] += m.prof.gmark_launches[k];
  }
}


double elastic_weight(const Mesh& m) { return m.h > 0.0 ? m.h * m.h : 1.0; }

// Re-evaluates the per-tet derivatives for a tet list and re-gathers g, H.
void refresh(Mesh& m, cc_precision p, const double* x, const double* xt, const int32_t* list, int64_t count) {
  cudaStream_t s = m.stream;
  int e0 = prof_event(m);
  if (p == CC_PREC_FP64)
    launch_tet_grad_f64(m, x, list, count, elastic_weight(m), s);
  else
    launch_tet_grad_mixed(m, list, count, elastic_weight(m), s);
  prof_close(m, P_TET, e0, count > 0 ? 1 : 0);
  e0 = prof_event(m);
  if (p == CC_PREC_FP64)
    launch_rows_f64(m, x, xt, elastic_weight(m), s);
  else
    launch_rows_mixed(m, elastic_weight(m), s);
  prof_close(m, P_GATHER, e0, 1);
}

void refresh_all(Mesh& m, cc_precision p, const double* x, const double* xt) {
  refresh(m, p, x, xt, m.d_all_tets.p, m.n_active_tets);
}

SweepCounters counters(Mesh& m) { return SweepCounters{m.d_counters.p, m.d_counters.p + 4}; }

void solve_list(Mesh& m, const cc_sweep_opts& o, const int32_t* verts, int64_t count, double* x) {
  if (count <= 0) return;
  const int e0 = prof_event(m);
  if (o.precision == CC_PREC_FP64)
    launch_local_solve_f64(m, o.update, verts, count, x, counters(m), m.stream);
  else
    launch_local_solve_mixed(m, o.update, verts, count, x, counters(m), m.stream);
  prof_close(m, P_SOLVE, e0, o.update == CC_UPDATE_CD || fused_local_solve(m, o.update) ? 1 : 2);
}

// One sweep over colours [cb, ce).  `fresh` means g and H already hold the
// derivatives at x (no refresh needed before the first colour).
void sweep_body(Mesh& m, double* x, const double* xt, const cc_sweep_opts& o, int cb, int ce, bool fresh) {
  m.rot_active = o.corotated != 0 && o.update != CC_UPDATE_CD;
  if (m.rot_active) {
    // corotated bases: rotations of the configuration at the start of the sweep (Sec. 3.1)
    const int e0 = prof_event(m);
    launch_rotations(m, x, o.precision == CC_PREC_MIXED, m.stream);
    prof_close(m, P_SOLVE, e0, 1);
  }
  if (o.schedule == CC_SCHED_JACOBI) {
    if (!fresh) refresh_all(m, o.precision, x, xt);
    solve_list(m, o, m.d_free_rows.p, m.n_free, x);
    return;
  }
  for (int c = cb; c < ce; ++c) {
    if (c == cb) {
      if (!fresh) refresh_all(m, o.precision, x, xt);
    } else {
      refresh(m, o.precision, x, xt, m.d_tl.p + m.tl_ptr[c - 1], m.tl_ptr[c] - m.tl_ptr[c - 1]);
    }
    solve_list(m, o, m.d_cv_idx.p + m.cv_ptr[c], m.cv_ptr[c + 1] - m.cv_ptr[c], x);
  }
}

// Brings g and H up to date after a sweep over [cb, ce).
void post_refresh(Mesh& m, double* x, const double* xt, const cc_sweep_opts& o, int ce) {
  if (o.schedule == CC_SCHED_JACOBI)
    refresh_all(m, o.precision, x, xt);
  else
    refresh(m, o.precision, x, xt, m.d_tl.p + m.tl_ptr[ce - 1], m.tl_ptr[ce] - m.tl_ptr[ce - 1]);
}

void gnorm(Mesh& m, cc_precision p, double* grad_out, double* out) {
  const int e0 = prof_event(m);
  if (p == CC_PREC_FP64)
    launch_gnorm_f64(m, grad_out, out, m.stream);
  else
    launch_gnorm_mixed(m, grad_out, out, m.stream);
  prof_close(m, P_RED, e0, 2);
}

void split(Mesh& m, const double* x, float4* hi, float4* lo) {
  const int e0 = prof_event(m);
  launch_split_df(x, m.n, hi, lo, m.stream);
  prof_close(m, P_OTHER, e0, 1);
}

double read_scalar(Mesh& m, const double* dev) {
  CCG_CUDA(cudaMemcpyAsync(m.h_pinned_scalars, dev, sizeof(double), cudaMemcpyDeviceToHost, m.stream));
  CCG_CUDA(cudaStreamSynchronize(m.stream));
  return m.h_pinned_scalars[0];
}

void read_counters(Mesh& m, cc_sweep_stats* st, int64_t updates) {
  unsigned long long h[8];
  CCG_CUDA(cudaMemcpyAsync(h, m.d_counters.p, sizeof(h), cudaMemcpyDeviceToHost, m.stream));
  CCG_CUDA(cudaStreamSynchronize(m.stream));
  if (st) {
    st->updates = updates;
    st->fallback_empty = (int64_t)h[0];
    st->fallback_reduced = (int64_t)h[1];
    st->fallback_schur = (int64_t)h[2];
  }
  CCG_CHECK(h[4] == 0, CC_ERR_NUMERIC, "non-finite local update");
}

void check_sweep_opts(const Mesh& m, const cc_sweep_opts& o, int* cb, int* ce) {
  CCG_CHECK(o.update >= CC_UPDATE_CC && o.update <= CC_UPDATE_JGS2, CC_ERR_INVALID_ARG, "bad update kind");
  CCG_CHECK(o.schedule == CC_SCHED_COLORED || o.schedule == CC_SCHED_JACOBI, CC_ERR_INVALID_ARG, "bad schedule");
  CCG_CHECK(o.precision == CC_PREC_FP64 || o.precision == CC_PREC_MIXED, CC_ERR_INVALID_ARG, "bad precision");
  CCG_CHECK(m.num_colors > 0, CC_ERR_STATE, "cc_color must run before sweeps");
  CCG_CHECK(o.update == CC_UPDATE_CD || m.k_ring > 0, CC_ERR_STATE, "CC and JGS2 need a subspace");
  *cb = 0;
  *ce = m.num_colors;
  if (o.schedule == CC_SCHED_COLORED) {
    *cb = o.color_begin;
    *ce = o.color_end < 0 ? m.num_colors : o.color_end;
    CCG_CHECK(*cb >= 0 && *cb < *ce && *ce <= m.num_colors, CC_ERR_INVALID_ARG, "bad colour range");
  }
}


// Every mesh of a batch takes part again (cc_solve_batch may have stopped some).
void activate_all(Mesh& m) {
  const size_t B = m.mesh_vptr.size() - 1;
  CCG_CUDA(cudaMemcpyAsync(m.d_mesh_active.p, m.d_mesh_ones.p, B * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                           m.stream));
}

// Runs `chunk` sweeps over colours [cb, ce), each followed by the refresh that
// makes g and H current, then the residual reduction: the global norm into
// d_scalars[0] (per_mesh false) or every mesh's squared norm into d_mesh_gsq.
// With `graph`, the whole chunk is captured once per key and replayed.
void run_chunk(Mesh& m, double* x, const double* xt, const cc_sweep_opts& so, int cb, int ce, int chunk,
               bool graph, const std::string& key, bool per_mesh) {
  cudaStream_t s = m.stream;
  auto body = [&]() {
    for (int k = 0; k < chunk; ++k) {
      sweep_body(m, x, xt, so, cb, ce, true);
      post_refresh(m, x, xt, so, ce);
    }
    if (per_mesh) {
      const int e0 = prof_event(m);
      launch_gnorm_mesh(m, so.precision == CC_PREC_MIXED, s);
      prof_close(m, P_RED, e0, 1);
    } else {
      gnorm(m, so.precision, nullptr, m.d_scalars.p);
    }
  };
  if (!graph) {
    body();
    CCG_CUDA(cudaGetLastError());
    return;
  }
  if (m.graph_key != key) {
    drop_graph(m);
    cudaGraph_t g = nullptr;
    CCG_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    m.prof.capturing = true;
    try {
      body();
    } catch (...) {
      m.prof.capturing = false;
      cudaStreamEndCapture(s, &g);
      if (g) cudaGraphDestroy(g);
      drop_graph(m);
      throw;
    }
    m.prof.capturing = false;
    CCG_CUDA(cudaStreamEndCapture(s, &g));
    cudaError_t ie = cudaGraphInstantiate(&m.graph_exec, g, 0);
    cudaGraphDestroy(g);
    CCG_CUDA(ie);
    m.graph_key = key;
  }
  CCG_CUDA(cudaGraphLaunch(m.graph_exec, s));
}

}  // namespace
}  // namespace ccg

using namespace ccg;

struct cc_mesh : public ccg::Mesh {};

extern "C" {

const char* cc_last_error(void) { return ccg::g_last_error.c_str(); }

const char* cc_version(void) { return "cc-gb300 0.1 (sm_103a)"; }

cc_status cc_build_mesh(const double* X, int64_t n, const int32_t* tets, int64_t T, const uint8_t* pinned,
                        const cc_material* mat, double h, const double* gravity, void* stream, cc_mesh** out) {
  cc_mesh* m = nullptr;
  try {
    ccg::g_last_error.clear();
    CCG_CHECK(out != nullptr, CC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    CCG_CHECK(X && tets && mat, CC_ERR_INVALID_ARG, "NULL input array");
    CCG_CHECK(n >= 4 && T >= 1 && n < (int64_t(1) << 31) && T < (int64_t(1) << 29), CC_ERR_INVALID_ARG,
              "n or T out of range");
    CCG_CHECK(mat->E > 0 && mat->nu > -1.0 && mat->nu < 0.5 && mat->rho >= 0 && std::isfinite(mat->E),
              CC_ERR_INVALID_ARG, "bad material");
    CCG_CHECK(mat->model == CC_MODEL_SNH || mat->model == CC_MODEL_FCR, CC_ERR_INVALID_ARG, "unknown material model");
    CCG_CHECK(h >= 0 && std::isfinite(h), CC_ERR_INVALID_ARG, "bad time step");
    m = new cc_mesh();
    m->n = n;
    m->T = T;
    m->E = mat->E;
    m->nu = mat->nu;
    m->rho = mat->rho;
    m->mu = mat->E / (2.0 * (1.0 + mat->nu));
    const double lam = mat->E * mat->nu / ((1.0 + mat->nu) * (1.0 - 2.0 * mat->nu));
    m->model = mat->model;
    m->lam_hat = m->model == CC_MODEL_FCR ? lam : lam + m->mu;  // the density's second parameter
    m->h = h;
    if (gravity && h > 0)
      for (int a = 0; a < 3; ++a) m->grav[a] = gravity[a];
    m->stream = (cudaStream_t)stream;
    m->X.assign(X, X + 3 * n);
    for (int64_t k = 0; k < 3 * n; ++k) CCG_CHECK(std::isfinite(X[k]), CC_ERR_INVALID_ARG, "non-finite rest position");
    m->tets.assign(tets, tets + 4 * T);
    m->pinned.assign(n, 0);
    if (pinned)
      for (int64_t v = 0; v < n; ++v) m->pinned[v] = pinned[v] ? 1 : 0;
    m->tet_mu.assign(T, m->mu);
    m->tet_lh.assign(T, m->lam_hat);
    m->tet_rho.assign(T, m->rho);
    m->tet_E.assign(T, mat->E);
    m->tet_nu.assign(T, mat->nu);
    ccg::build_topology(*m);
    CCG_CHECK(m->n_free > 0, CC_ERR_INVALID_ARG, "every vertex is pinned");
    m->d_red.alloc(4096);
    m->d_scalars.alloc(8);
    m->d_counters.alloc(8);
    CCG_CUDA(cudaMemsetAsync(m->d_counters.p, 0, 8 * sizeof(unsigned long long), m->stream));
    CCG_CUDA(cudaMallocHost((void**)&m->h_pinned_scalars, 8 * sizeof(double)));
    *out = m;
    return CC_OK;
  } catch (const ccg::Fail& f) {
    cc_destroy_mesh(m);
    return f.st;
  } catch (...) {
    cc_destroy_mesh(m);
    ccg::g_last_error = "cc_build_mesh: unexpected error";
    return CC_ERR_STATE;
  }
}

void cc_destroy_mesh(cc_mesh* m) {
  if (!m) return;
  if (m->stream) cudaStreamSynchronize(m->stream);
  else cudaDeviceSynchronize();
  drop_graph(*m);
  for (cudaEvent_t e : m->prof.pool) cudaEventDestroy(e);
  auto rel = [](auto& b) { b.release(); };
  rel(m->d_tets); rel(m->d_tslot); rel(m->d_Bm); rel(m->d_Bm_df); rel(m->d_Bm32); rel(m->d_vol); rel(m->d_mat64); rel(m->d_matdf); rel(m->d_vert_mesh);
  rel(m->d_mesh_fptr); rel(m->d_mesh_active); rel(m->d_mesh_ones); rel(m->d_mesh_gsq); rel(m->d_volw); rel(m->d_volw32); rel(m->d_volw_df); rel(m->d_mass);
  rel(m->d_mass32); rel(m->d_mass_df);
  rel(m->d_pinned); rel(m->d_vt_ptr); rel(m->d_nbr_ptr); rel(m->d_nbr_idx); rel(m->d_vt_tet); rel(m->d_vt_corner);
  rel(m->d_up_ptr); rel(m->d_up_col); rel(m->d_rs_ptr); rel(m->d_rs_src); rel(m->d_free_rows); rel(m->d_row_hdr);
  rel(m->d_color); rel(m->d_cv_idx); rel(m->d_tl); rel(m->d_all_tets); rel(m->d_sup_ptr); rel(m->d_sup_idx); rel(m->d_smap_ptr);
  rel(m->d_smap8); rel(m->d_smap16); rel(m->d_vt_ids);
  rel(m->f64.gcon); rel(m->f64.hten); rel(m->f64.g); rel(m->f64.cpl); rel(m->f64.bsr); rel(m->f64.U);
  rel(m->mx.gcon); rel(m->mx.hten); rel(m->mx.cpl); rel(m->mx.g_hi); rel(m->mx.g_lo); rel(m->mx.bsr); rel(m->mx.U);
  rel(m->mx.x_hi); rel(m->mx.x_lo); rel(m->mx.xt_hi); rel(m->mx.xt_lo);
  rel(m->d_red); rel(m->d_scalars); rel(m->d_counters); rel(m->d_xtilde); rel(m->d_xold);
  if (m->h_pinned_scalars) cudaFreeHost(m->h_pinned_scalars);
  delete m;
}

cc_status cc_color(cc_mesh* m, int32_t* colors_out, int32_t* num_colors) {
  CC_API_BODY("cc_color", {
    CCG_CHECK(m, CC_ERR_INVALID_ARG, "mesh is NULL");
    drop_graph(*m);
    ccg::run_coloring(*m);
    if (colors_out) std::memcpy(colors_out, m->color.data(), m->n * sizeof(int32_t));
    if (num_colors) *num_colors = m->num_colors;
  })
}

cc_status cc_set_colors(cc_mesh* m, const int32_t* colors, int32_t num_colors) {
  CC_API_BODY("cc_set_colors", {
    CCG_CHECK(m && colors, CC_ERR_INVALID_ARG, "NULL argument");
    drop_graph(*m);
    ccg::set_coloring(*m, colors, num_colors);
  })
}

cc_status cc_build_subspace(cc_mesh* m, int32_t k) {
  CC_API_BODY("cc_build_subspace", {
    CCG_CHECK(m, CC_ERR_INVALID_ARG, "mesh is NULL");
    CCG_CHECK(k >= 1 && k <= 4, CC_ERR_INVALID_ARG, "k_ring must be in [1, 4]");
    CCG_CHECK(m->num_colors > 0, CC_ERR_STATE, "cc_color must run before cc_build_subspace");
    ensure_state(*m, CC_PREC_FP64);
    drop_graph(*m);
    ccg::run_subspace_build(*m, k);
  })
}

cc_status cc_build_subspace_at(cc_mesh* m, const double* x, int64_t* kept) {
  CC_API_BODY("cc_build_subspace_at", {
    CCG_CHECK(m && x, CC_ERR_INVALID_ARG, "NULL argument");
    CCG_CHECK(m->k_ring != 0 && m->f64.U.p, CC_ERR_STATE, "cc_build_subspace must run first");
    ensure_state(*m, CC_PREC_FP64);
    const int64_t k = ccg::rebuild_bases_at(*m, x);
    if (kept) *kept = k;
  })
}

cc_status cc_set_subspace(cc_mesh* m, const int64_t* sup_ptr, const int32_t* sup_idx, const double* U) {
  CC_API_BODY("cc_set_subspace", {
    CCG_CHECK(m && sup_ptr && U, CC_ERR_INVALID_ARG, "NULL argument");
    const int64_t n = m->n;
    CCG_CHECK(sup_ptr[0] == 0, CC_ERR_INVALID_ARG, "sup_ptr[0] must be 0");
    int32_t supmax = 0;
    for (int64_t v = 0; v < n; ++v) {
      CCG_CHECK(sup_ptr[v + 1] >= sup_ptr[v], CC_ERR_INVALID_ARG, "sup_ptr not monotone");
      const int64_t len = sup_ptr[v + 1] - sup_ptr[v];
      CCG_CHECK(!m->pinned[v] || len == 0, CC_ERR_INVALID_ARG, "pinned vertex with a non-empty support");
      for (int64_t p = sup_ptr[v]; p < sup_ptr[v + 1]; ++p) {
        const int32_t j = sup_idx[p];
        CCG_CHECK(j >= 0 && j < n && j != v && !m->pinned[j], CC_ERR_INVALID_ARG, "bad support vertex");
        CCG_CHECK(p == sup_ptr[v] || sup_idx[p - 1] < j, CC_ERR_INVALID_ARG, "support not ascending");
      }
      supmax = std::max<int32_t>(supmax, (int32_t)len);
    }
    const int64_t total = sup_ptr[n];
    CCG_CHECK(total < (int64_t(1) << 31) && supmax < 32768, CC_ERR_INVALID_ARG, "support too large");
    drop_graph(*m);
    m->sup_ptr.assign(sup_ptr, sup_ptr + n + 1);
    m->sup_idx.assign(sup_idx, sup_idx + total);
    m->sup_max = supmax;
    int hs = 32;
    while (hs < 2 * std::max(supmax, 1)) hs <<= 1;
    m->hash_size = hs;
    if (m->k_ring == 0) m->k_ring = -1;  // custom
    std::vector<int32_t> sp32(n + 1);
    for (int64_t v = 0; v <= n; ++v) sp32[v] = (int32_t)sup_ptr[v];
    m->d_sup_ptr.upload(sp32, m->stream);
    m->d_sup_idx.upload(m->sup_idx, m->stream);
    ccg::build_slot_maps(*m);
    m->f64.U.alloc(9 * std::max<int64_t>(total, 1));
    if (total) CCG_CUDA(cudaMemcpyAsync(m->f64.U.p, U, 9 * total * sizeof(double), cudaMemcpyHostToDevice, m->stream));
    m->mx.U.alloc(9 * std::max<int64_t>(total, 1));
    ccg::bases_to_f32(*m);
    CCG_CUDA(cudaStreamSynchronize(m->stream));
  })
}

cc_status cc_energy_grad(cc_mesh* m, const double* x, const double* xt, cc_precision p, double* energy,
                         double* grad, double* grad_norm) {
  CC_API_BODY("cc_energy_grad", {
    CCG_CHECK(m && x, CC_ERR_INVALID_ARG, "NULL argument");
    CCG_CHECK(p == CC_PREC_FP64 || p == CC_PREC_MIXED, CC_ERR_INVALID_ARG, "bad precision");
    CCG_CHECK(m->h == 0.0 || xt, CC_ERR_INVALID_ARG, "dynamic mesh needs xtilde");
    ensure_state(*m, p);
    cudaStream_t s = m->stream;
    if (p == CC_PREC_MIXED) {
      split(*m, x, m->mx.x_hi.p, m->mx.x_lo.p);
      if (m->h > 0.0) split(*m, xt, m->mx.xt_hi.p, m->mx.xt_lo.p);
    }
    refresh_all(*m, p, x, xt);
    if (grad) CCG_CUDA(cudaMemsetAsync(grad, 0, 3 * m->n * sizeof(double), s));
    gnorm(*m, p, grad, m->d_scalars.p);
    launch_energy(*m, x, m->h > 0.0 ? xt : nullptr, m->d_scalars.p + 1, s);
    CCG_CUDA(cudaGetLastError());
    CCG_CUDA(cudaMemcpyAsync(m->h_pinned_scalars, m->d_scalars.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CCG_CUDA(cudaStreamSynchronize(s));
    if (grad_norm) *grad_norm = std::sqrt(m->h_pinned_scalars[0]);
    if (energy) *energy = m->h_pinned_scalars[1];
  })
}

cc_status cc_sweep(cc_mesh* m, double* x, const double* xt, const cc_sweep_opts* opts, cc_sweep_stats* stats) {
  CC_API_BODY("cc_sweep", {
    CCG_CHECK(m && x && opts, CC_ERR_INVALID_ARG, "NULL argument");
    CCG_CHECK(m->h == 0.0 || xt, CC_ERR_INVALID_ARG, "dynamic mesh needs xtilde");
    int cb, ce;
    check_sweep_opts(*m, *opts, &cb, &ce);
    ensure_state(*m, opts->precision);
    cudaStream_t s = m->stream;
    CCG_CUDA(cudaMemsetAsync(m->d_counters.p, 0, 8 * sizeof(unsigned long long), s));
    activate_all(*m);
    if (opts->precision == CC_PREC_MIXED) {
      split(*m, x, m->mx.x_hi.p, m->mx.x_lo.p);
      if (m->h > 0.0) split(*m, xt, m->mx.xt_hi.p, m->mx.xt_lo.p);
    }
    sweep_body(*m, x, xt, *opts, cb, ce, false);
    CCG_CUDA(cudaGetLastError());
    int64_t upd = opts->schedule == CC_SCHED_JACOBI ? m->n_free : (int64_t)(m->cv_ptr[ce] - m->cv_ptr[cb]);
    read_counters(*m, stats, upd);
  })
}

cc_status cc_solve_step(cc_mesh* m, double* x, double* v, const cc_step_opts* o, cc_step_stats* st) {
  cc_status rc = CC_OK;
  try {
    ccg::g_last_error.clear();
    CCG_CHECK(m && x && o, CC_ERR_INVALID_ARG, "NULL argument");
    CCG_CHECK(o->max_iters >= 0 && o->min_iters >= 0 && o->tol >= 0, CC_ERR_INVALID_ARG, "bad iteration limits");
    CCG_CHECK((m->h > 0.0) == (v != nullptr), CC_ERR_INVALID_ARG,
              "v must be given exactly for dynamic meshes (h > 0)");
    cc_sweep_opts so{o->update, o->schedule, o->precision, 0, -1, o->corotated};
    int cb, ce;
    check_sweep_opts(*m, so, &cb, &ce);
    ensure_state(*m, o->precision);
    cudaStream_t s = m->stream;
    const int64_t n = m->n;
    const bool dyn = m->h > 0.0;
    const double* xt = nullptr;
    if (dyn) {
      if (!m->d_xtilde.p) {
        m->d_xtilde.alloc(3 * n);
        m->d_xold.alloc(3 * n);
      }
      CCG_CUDA(cudaMemcpyAsync(m->d_xold.p, x, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      const int e0 = prof_event(*m);
      launch_inertial_target(x, v, n, m->h, m->grav, m->d_xtilde.p, s);
      prof_close(*m, P_OTHER, e0, 1);
      xt = m->d_xtilde.p;
    }
    CCG_CUDA(cudaMemsetAsync(m->d_counters.p, 0, 8 * sizeof(unsigned long long), s));
    activate_all(*m);
    if (o->precision == CC_PREC_MIXED) {
      split(*m, x, m->mx.x_hi.p, m->mx.x_lo.p);
      if (dyn) split(*m, xt, m->mx.xt_hi.p, m->mx.xt_lo.p);
    }
    refresh_all(*m, o->precision, x, xt);
    gnorm(*m, o->precision, nullptr, m->d_scalars.p);
    const double g0 = std::sqrt(read_scalar(*m, m->d_scalars.p));
    CCG_CHECK(std::isfinite(g0), CC_ERR_NUMERIC, "non-finite initial residual");
    if (o->residual_history) {
      o->residual_history[0] = g0;
      for (int k = 1; k <= o->max_iters; ++k) o->residual_history[k] = -1.0;
    }
    const int every = std::max(1, o->check_every);
    double gcur = g0;
    int it = 0;
    bool conv = (g0 == 0.0);
    // Graph mode: the `every` sweeps and the residual reduction between two
    // host checks are captured once and replayed.  The first chunk always runs
    // launch by launch (it sets kernel attributes outside any capture), and
    // the legacy default stream cannot be captured, so it never uses graphs.
    const bool graph = o->use_graph && s != nullptr;
    std::string key;
    if (graph) {
      char buf[256];
      std::snprintf(buf, sizeof(buf), "step %p %p %d %d %d %d %d %d", (void*)x, (const void*)xt, (int)o->precision,
                    (int)o->schedule, (int)o->update, every, m->prof.on ? 1 : 0, (int)o->corotated);
      key = buf;
    }
    const int restart = std::max(0, o->restart_every);
    auto maybe_restart = [&]() {
      if (restart > 0 && it > 0 && it % restart == 0) {
        // restarted CC: bases from the Hessian at the current x, then the
        // solver state is brought back to x (the rebuild overwrote float64 rows)
        ensure_state(*m, CC_PREC_FP64);
        rebuild_bases_at(*m, x);
        refresh_all(*m, o->precision, x, xt);
      }
    };
    while (!conv && it < o->max_iters && !o->line_search) {
      maybe_restart();
      int chunk = std::min(every, o->max_iters - it);
      if (restart > 0) chunk = std::min(chunk, restart - it % restart);
      const bool replay = graph && chunk == every && it > 0;
      run_chunk(*m, x, xt, so, cb, ce, chunk, replay, key, false);
      it += chunk;
      gcur = std::sqrt(read_scalar(*m, m->d_scalars.p));
      if (replay) prof_after_replay(*m);
      if (o->residual_history) o->residual_history[it] = gcur;
      CCG_CHECK(std::isfinite(gcur), CC_ERR_NUMERIC, "non-finite residual");
      if (it >= o->min_iters && gcur <= o->tol * g0) conv = true;
    }
    // Global backtracking line search (Sec. 4.4): the sweep's displacement is
    // the direction, the step the largest 2^-k (k < 30) that does not raise E.
    if (o->line_search && !conv && it < o->max_iters) {
      if (!m->d_xls0.p) {
        m->d_xls0.alloc(3 * n);
        m->d_xls1.alloc(3 * n);
      }
      auto energy_at = [&](const double* xe) {
        const int ee = prof_event(*m);
        launch_energy(*m, xe, xt, m->d_scalars.p + 1, s);
        prof_close(*m, P_RED, ee, dyn ? 3 : 2);
        return read_scalar(*m, m->d_scalars.p + 1);
      };
      while (!conv && it < o->max_iters) {
        maybe_restart();
        CCG_CUDA(cudaMemcpyAsync(m->d_xls0.p, x, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        const double E0 = energy_at(x);
        sweep_body(*m, x, xt, so, cb, ce, true);  // g, H are current at x (refreshed below)
        CCG_CUDA(cudaMemcpyAsync(m->d_xls1.p, x, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        double a = 1.0;
        bool found = false;
        for (int k = 0; k < 30; ++k) {
          if (k > 0) launch_line_point(m->d_xls0.p, m->d_xls1.p, n, a, x, s);
          const double E1 = energy_at(x);
          if (E1 <= E0) {
            found = true;
            break;
          }
          a *= 0.5;
        }
        if (!found) CCG_CUDA(cudaMemcpyAsync(x, m->d_xls0.p, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        if (o->precision == CC_PREC_MIXED) split(*m, x, m->mx.x_hi.p, m->mx.x_lo.p);
        refresh_all(*m, o->precision, x, xt);
        gnorm(*m, o->precision, nullptr, m->d_scalars.p);
        ++it;
        gcur = std::sqrt(read_scalar(*m, m->d_scalars.p));
        if (o->residual_history) o->residual_history[it] = gcur;
        CCG_CHECK(std::isfinite(gcur), CC_ERR_NUMERIC, "non-finite residual");
        if (it >= o->min_iters && gcur <= o->tol * g0) conv = true;
      }
    }
    int e1 = prof_event(*m);
    launch_energy(*m, x, xt, m->d_scalars.p + 1, s);
    prof_close(*m, P_RED, e1, dyn ? 3 : 2);
    const double energy = read_scalar(*m, m->d_scalars.p + 1);
    if (dyn) {
      e1 = prof_event(*m);
      launch_velocity(x, m->d_xold.p, n, m->h, v, s);
      prof_close(*m, P_OTHER, e1, 1);
    }
    cc_step_stats tmp{};
    read_counters(*m, &tmp.sweeps, (int64_t)it * m->n_free);
    tmp.iterations = it;
    tmp.converged = conv ? 1 : 0;
    tmp.g0 = g0;
    tmp.g_final = gcur;
    tmp.energy_final = energy;
    CCG_CUDA(cudaStreamSynchronize(s));
    if (st) *st = tmp;
    if (!conv) {
      ccg::g_last_error = "cc_solve_step: max_iters reached before the tolerance";
      rc = CC_ERR_NOT_CONVERGED;
    }
    return rc;
  } catch (const ccg::Fail& f) {
    if (ccg::g_last_error.empty()) ccg::g_last_error = "cc_solve_step";
    return f.st;
  } catch (...) {
    ccg::g_last_error = "cc_solve_step: unexpected error";
    return CC_ERR_STATE;
  }
}

cc_status cc_build_batch(const cc_mesh_desc* meshes, int32_t count, double h, const double* gravity, void* stream,
                         cc_mesh** out) {
  cc_mesh* m = nullptr;
  try {
    ccg::g_last_error.clear();
    CCG_CHECK(out != nullptr, CC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    CCG_CHECK(meshes && count >= 1, CC_ERR_INVALID_ARG, "need at least one mesh");
    CCG_CHECK(h >= 0 && std::isfinite(h), CC_ERR_INVALID_ARG, "bad time step");
    int64_t n = 0, T = 0;
    for (int32_t b = 0; b < count; ++b) {
      const cc_mesh_desc& d = meshes[b];
      CCG_CHECK(d.X && d.tets && d.n >= 4 && d.T >= 1, CC_ERR_INVALID_ARG, "bad mesh in batch");
      CCG_CHECK(d.mat.E > 0 && d.mat.nu > -1.0 && d.mat.nu < 0.5 && d.mat.rho >= 0 && std::isfinite(d.mat.E),
                CC_ERR_INVALID_ARG, "bad material in batch");
      CCG_CHECK(d.mat.model == meshes[0].mat.model && (d.mat.model == CC_MODEL_SNH || d.mat.model == CC_MODEL_FCR),
                CC_ERR_INVALID_ARG, "the meshes of a batch must share one known material model");
      n += d.n;
      T += d.T;
    }
    CCG_CHECK(n < (int64_t(1) << 31) && T < (int64_t(1) << 29), CC_ERR_INVALID_ARG, "batch too large");
    m = new cc_mesh();
    m->n = n;
    m->T = T;
    const cc_material& m0 = meshes[0].mat;
    m->E = m0.E;
    m->nu = m0.nu;
    m->rho = m0.rho;
    m->mu = m0.E / (2.0 * (1.0 + m0.nu));
    m->model = m0.model;
    m->lam_hat = m0.E * m0.nu / ((1.0 + m0.nu) * (1.0 - 2.0 * m0.nu)) + (m->model == CC_MODEL_FCR ? 0.0 : m->mu);
    m->h = h;
    if (gravity && h > 0)
      for (int a = 0; a < 3; ++a) m->grav[a] = gravity[a];
    m->stream = (cudaStream_t)stream;
    m->X.resize(3 * n);
    m->tets.resize(4 * T);
    m->pinned.assign(n, 0);
    m->tet_mu.resize(T);
    m->tet_lh.resize(T);
    m->tet_rho.resize(T);
    m->tet_E.resize(T);
    m->tet_nu.resize(T);
    m->mesh_vptr.assign(count + 1, 0);
    m->mesh_tptr.assign(count + 1, 0);
    int64_t vo = 0, to = 0;
    for (int32_t b = 0; b < count; ++b) {
      const cc_mesh_desc& d = meshes[b];
      for (int64_t k = 0; k < 3 * d.n; ++k) {
        CCG_CHECK(std::isfinite(d.X[k]), CC_ERR_INVALID_ARG, "non-finite rest position");
        m->X[3 * vo + k] = d.X[k];
      }
      for (int64_t k = 0; k < 4 * d.T; ++k) {
        CCG_CHECK(d.tets[k] >= 0 && d.tets[k] < d.n, CC_ERR_INVALID_ARG, "tet vertex id out of range");
        m->tets[4 * to + k] = (int32_t)(d.tets[k] + vo);
      }
      if (d.pinned)
        for (int64_t v = 0; v < d.n; ++v) m->pinned[vo + v] = d.pinned[v] ? 1 : 0;
      const double mu = d.mat.E / (2.0 * (1.0 + d.mat.nu));
      const double lh = d.mat.E * d.mat.nu / ((1.0 + d.mat.nu) * (1.0 - 2.0 * d.mat.nu)) +
                        (m->model == CC_MODEL_FCR ? 0.0 : mu);
      for (int64_t t = 0; t < d.T; ++t) {
        m->tet_mu[to + t] = mu;
        m->tet_lh[to + t] = lh;
        m->tet_rho[to + t] = d.mat.rho;
        m->tet_E[to + t] = d.mat.E;
        m->tet_nu[to + t] = d.mat.nu;
      }
      vo += d.n;
      to += d.T;
      m->mesh_vptr[b + 1] = vo;
      m->mesh_tptr[b + 1] = to;
    }
    ccg::build_topology(*m);
    CCG_CHECK(m->n_free > 0, CC_ERR_INVALID_ARG, "every vertex is pinned");
    m->d_red.alloc(4096);
    m->d_scalars.alloc(8);
    m->d_counters.alloc(8);
    CCG_CUDA(cudaMemsetAsync(m->d_counters.p, 0, 8 * sizeof(unsigned long long), m->stream));
    CCG_CUDA(cudaMallocHost((void**)&m->h_pinned_scalars, 8 * sizeof(double)));
    *out = m;
    return CC_OK;
  } catch (const ccg::Fail& f) {
    cc_destroy_mesh(m);
    return f.st;
  } catch (...) {
    cc_destroy_mesh(m);
    ccg::g_last_error = "cc_build_batch: unexpected error";
    return CC_ERR_STATE;
  }
}

cc_status cc_batch_offsets(const cc_mesh* m, int64_t* offsets, int32_t* count) {
  CC_API_BODY("cc_batch_offsets", {
    CCG_CHECK(m, CC_ERR_INVALID_ARG, "mesh is NULL");
    const int32_t B = (int32_t)m->mesh_vptr.size() - 1;
    if (count) *count = B;
    if (offsets) std::memcpy(offsets, m->mesh_vptr.data(), (B + 1) * sizeof(int64_t));
  })
}

cc_status cc_solve_batch(cc_mesh* m, double* x, double* v, const cc_step_opts* o, cc_batch_stats* st) {
  try {
    ccg::g_last_error.clear();
    CCG_CHECK(m && x && o && st && st->iterations && st->status && st->g0 && st->g_final, CC_ERR_INVALID_ARG,
              "NULL argument");
    CCG_CHECK(o->max_iters >= 0 && o->min_iters >= 0 && o->tol >= 0, CC_ERR_INVALID_ARG, "bad iteration limits");
    CCG_CHECK((m->h > 0.0) == (v != nullptr), CC_ERR_INVALID_ARG,
              "v must be given exactly for dynamic meshes (h > 0)");
    cc_sweep_opts so{o->update, o->schedule, o->precision, 0, -1, o->corotated};
    int cb, ce;
    check_sweep_opts(*m, so, &cb, &ce);
    ensure_state(*m, o->precision);
    cudaStream_t s = m->stream;
    const int64_t n = m->n;
    const int32_t B = (int32_t)m->mesh_vptr.size() - 1;
    const bool dyn = m->h > 0.0;
    const double* xt = nullptr;
    if (dyn) {
      if (!m->d_xtilde.p) {
        m->d_xtilde.alloc(3 * n);
        m->d_xold.alloc(3 * n);
      }
      CCG_CUDA(cudaMemcpyAsync(m->d_xold.p, x, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      launch_inertial_target(x, v, n, m->h, m->grav, m->d_xtilde.p, s);
      xt = m->d_xtilde.p;
    }
    CCG_CUDA(cudaMemsetAsync(m->d_counters.p, 0, 8 * sizeof(unsigned long long), s));
    activate_all(*m);
    if (o->precision == CC_PREC_MIXED) {
      split(*m, x, m->mx.x_hi.p, m->mx.x_lo.p);
      if (dyn) split(*m, xt, m->mx.xt_hi.p, m->mx.xt_lo.p);
    }
    refresh_all(*m, o->precision, x, xt);
    launch_gnorm_mesh(*m, o->precision == CC_PREC_MIXED, s);
    std::vector<double> gsq(B);
    std::vector<int32_t> active(B, 1);
    CCG_CUDA(cudaMemcpyAsync(gsq.data(), m->d_mesh_gsq.p, B * sizeof(double), cudaMemcpyDeviceToHost, s));
    CCG_CUDA(cudaStreamSynchronize(s));
    int32_t live = 0;
    for (int32_t b = 0; b < B; ++b) {
      st->g0[b] = std::sqrt(gsq[b]);
      st->g_final[b] = st->g0[b];
      st->iterations[b] = 0;
      st->status[b] = 0;
      if (!(st->g0[b] > 0.0)) {
        active[b] = 0;
        st->status[b] = std::isfinite(st->g0[b]) ? 1 : -1;
      } else {
        ++live;
      }
    }
    const int every = std::max(1, o->check_every);
    const bool graph = o->use_graph && s != nullptr;
    std::string key;
    if (graph) {
      char buf[256];
      std::snprintf(buf, sizeof(buf), "batch %p %p %d %d %d %d %d %d", (void*)x, (const void*)xt, (int)o->precision,
                    (int)o->schedule, (int)o->update, every, m->prof.on ? 1 : 0, (int)o->corotated);
      key = buf;
    }
    int it = 0;
    // per-mesh bookkeeping after every residual check: converged, diverged
    // (non-finite or above 1e6 x its start) or still running
    auto check_meshes = [&]() {
      CCG_CUDA(cudaMemcpyAsync(gsq.data(), m->d_mesh_gsq.p, B * sizeof(double), cudaMemcpyDeviceToHost, s));
      CCG_CUDA(cudaStreamSynchronize(s));
      for (int32_t b = 0; b < B; ++b) {
        if (!active[b]) continue;
        const double g = std::sqrt(gsq[b]);
        st->iterations[b] = it;
        st->g_final[b] = g;
        if (!std::isfinite(g) || g > 1e6 * st->g0[b]) {
          st->status[b] = -1;
        } else if (it >= o->min_iters && g <= o->tol * st->g0[b]) {
          st->status[b] = 1;
        } else {
          continue;
        }
        active[b] = 0;
        --live;
      }
    };
    const int restart = std::max(0, o->restart_every);
    auto maybe_restart = [&]() {
      if (restart > 0 && it > 0 && it % restart == 0) {
        // restarted CC on the whole union: bases from the Hessian at the current x
        ensure_state(*m, CC_PREC_FP64);
        rebuild_bases_at(*m, x);
        refresh_all(*m, o->precision, x, xt);
      }
    };
    auto upload_active = [&]() {
      CCG_CUDA(cudaMemcpyAsync(m->d_mesh_active.p, active.data(), B * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    };
    while (!o->line_search && live > 0 && it < o->max_iters) {
      maybe_restart();
      upload_active();
      int chunk = std::min(every, o->max_iters - it);
      if (restart > 0) chunk = std::min(chunk, restart - it % restart);
      const bool replay = graph && chunk == every && it > 0;
      run_chunk(*m, x, xt, so, cb, ce, chunk, replay, key, true);
      it += chunk;
      if (replay) prof_after_replay(*m);
      check_meshes();
    }
    // Global backtracking line search per mesh (Sec. 4.4): each mesh takes
    // the largest 2^-k (k < 30) of its own sweep displacement that does not
    // raise its own energy, 0 if none; every trial is one launch for all.
    if (o->line_search && live > 0 && it < o->max_iters) {
      if (!m->d_xls0.p) {
        m->d_xls0.alloc(3 * n);
        m->d_xls1.alloc(3 * n);
      }
      std::vector<double> E0(B), E1(B), alpha(B);
      std::vector<char> searching(B);
      auto energies = [&](const double* xe, std::vector<double>& out) {
        launch_energy_mesh(*m, xe, xt, m->d_mesh_energy.p, s);
        CCG_CUDA(cudaMemcpyAsync(out.data(), m->d_mesh_energy.p, B * sizeof(double), cudaMemcpyDeviceToHost, s));
        CCG_CUDA(cudaStreamSynchronize(s));
      };
      auto set_alpha = [&]() {
        CCG_CUDA(cudaMemcpyAsync(m->d_mesh_alpha.p, alpha.data(), B * sizeof(double), cudaMemcpyHostToDevice, s));
        launch_line_point_mesh(*m, m->d_xls0.p, m->d_xls1.p, m->d_mesh_alpha.p, x, s);
      };
      while (live > 0 && it < o->max_iters) {
        maybe_restart();
        upload_active();
        CCG_CUDA(cudaMemcpyAsync(m->d_xls0.p, x, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        energies(x, E0);
        sweep_body(*m, x, xt, so, cb, ce, true);  // g, H are current at x (refreshed below); stopped meshes stay
        CCG_CUDA(cudaMemcpyAsync(m->d_xls1.p, x, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        for (int32_t b = 0; b < B; ++b) {
          alpha[b] = active[b] ? 1.0 : 0.0;
          searching[b] = active[b] ? 1 : 0;
        }
        for (int k = 0; k < 30; ++k) {
          if (k > 0) set_alpha();
          energies(x, E1);
          bool any = false;
          for (int32_t b = 0; b < B; ++b) {
            if (!searching[b]) continue;
            if (E1[b] <= E0[b]) {
              searching[b] = 0;
            } else {
              alpha[b] *= 0.5;
              any = true;
            }
          }
          if (!any) break;
        }
        for (int32_t b = 0; b < B; ++b)
          if (searching[b]) alpha[b] = 0.0;  // no decrease found: the mesh stays at x
        set_alpha();
        if (o->precision == CC_PREC_MIXED) split(*m, x, m->mx.x_hi.p, m->mx.x_lo.p);
        refresh_all(*m, o->precision, x, xt);
        launch_gnorm_mesh(*m, o->precision == CC_PREC_MIXED, s);
        ++it;
        check_meshes();
      }
    }
    activate_all(*m);
    if (dyn) launch_velocity(x, m->d_xold.p, n, m->h, v, s);
    unsigned long long h8[8];
    CCG_CUDA(cudaMemcpyAsync(h8, m->d_counters.p, sizeof(h8), cudaMemcpyDeviceToHost, s));
    CCG_CUDA(cudaStreamSynchronize(s));
    st->sweeps = it;
    st->totals.updates = (int64_t)it * m->n_free;
    st->totals.fallback_empty = (int64_t)h8[0];
    st->totals.fallback_reduced = (int64_t)h8[1];
    st->totals.fallback_schur = (int64_t)h8[2];
    bool all = true;
    for (int32_t b = 0; b < B; ++b) all &= st->status[b] == 1;
    if (!all) {
      ccg::g_last_error = "cc_solve_batch: some meshes did not converge";
      return CC_ERR_NOT_CONVERGED;
    }
    return CC_OK;
  } catch (const ccg::Fail& f) {
    if (ccg::g_last_error.empty()) ccg::g_last_error = "cc_solve_batch";
    return f.st;
  } catch (...) {
    ccg::g_last_error = "cc_solve_batch: unexpected error";
    return CC_ERR_STATE;
  }
}

cc_status cc_solve_concurrent(int32_t count, cc_mesh* const* meshes, double* const* x, double* const* v,
                              const cc_step_opts* o, cc_step_stats* st, cc_status* status) {
  try {
    ccg::g_last_error.clear();
    CCG_CHECK(count >= 0, CC_ERR_INVALID_ARG, "negative count");
    if (count == 0) return CC_OK;
    CCG_CHECK(meshes && x && o, CC_ERR_INVALID_ARG, "NULL argument");
    for (int32_t k = 0; k < count; ++k) {
      CCG_CHECK(meshes[k] && x[k], CC_ERR_INVALID_ARG, "NULL mesh or x");
      const cudaStream_t s = meshes[k]->stream;
      CCG_CHECK(s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread, CC_ERR_INVALID_ARG,
                "every mesh needs a stream of its own (not a default stream)");
      for (int32_t j = 0; j < k; ++j) {
        CCG_CHECK(meshes[j] != meshes[k], CC_ERR_INVALID_ARG, "a mesh appears twice");
        CCG_CHECK(meshes[j]->stream != s, CC_ERR_INVALID_ARG, "two meshes share a stream");
        CCG_CHECK(x[j] != x[k], CC_ERR_INVALID_ARG, "two meshes share x");
        CCG_CHECK(!o[k].residual_history || o[j].residual_history != o[k].residual_history, CC_ERR_INVALID_ARG,
                  "two meshes share a residual history");
      }
    }
    int dev = 0;
    CCG_CUDA(cudaGetDevice(&dev));
    std::vector<cc_status> rc(count, CC_OK);
    std::vector<std::string> msg(count);
    auto work = [&](int32_t k) {
      const cudaError_t e = cudaSetDevice(dev);
      if (e != cudaSuccess) {
        rc[k] = CC_ERR_CUDA;
        try {
          msg[k] = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
        } catch (...) {
        }
        return;
      }
      rc[k] = cc_solve_step(meshes[k], x[k], v ? v[k] : nullptr, &o[k], st ? &st[k] : nullptr);
      try {
        msg[k] = ccg::g_last_error;
      } catch (...) {  // keep the status; lose only the message
      }
    };
    // One thread per further mesh; a mesh whose thread could not be started
    // runs on the calling thread after mesh 0 (same result, less overlap).
    std::vector<std::thread> pool;
    std::vector<int32_t> here;
    pool.reserve(count - 1);
    here.reserve(count);
    here.push_back(0);
    struct JoinAll {  // started threads are joined on every way out of this scope
      std::vector<std::thread>& threads;
      ~JoinAll() {
        for (auto& t : threads)
          if (t.joinable()) t.join();
      }
    } join_all{pool};
    for (int32_t k = 1; k < count; ++k) {
      try {
        pool.emplace_back(work, k);
      } catch (const std::system_error&) {
        here.push_back(k);  // capacity reserved: cannot throw
      }
    }
    for (int32_t k : here) work(k);
    for (auto& t : pool) t.join();
    cc_status out = CC_OK;
    int32_t who = -1;
    for (int32_t k = 0; k < count; ++k) {
      if (status) status[k] = rc[k];
      if (rc[k] != CC_OK && rc[k] != CC_ERR_NOT_CONVERGED && (out == CC_OK || out == CC_ERR_NOT_CONVERGED)) {
        out = rc[k];
        who = k;
      } else if (rc[k] == CC_ERR_NOT_CONVERGED && out == CC_OK) {
        out = rc[k];
        who = k;
      }
    }
    ccg::g_last_error.clear();
    if (who >= 0) ccg::g_last_error = "cc_solve_concurrent: mesh " + std::to_string(who) + ": " + msg[who];
    return out;
  } catch (const ccg::Fail& f) {
    if (ccg::g_last_error.empty()) ccg::g_last_error = "cc_solve_concurrent";
    return f.st;
  } catch (const std::bad_alloc&) {
    ccg::g_last_error = "cc_solve_concurrent: host out of memory";
    return CC_ERR_OOM;
  } catch (...) {
    ccg::g_last_error = "cc_solve_concurrent: unexpected error";
    return CC_ERR_STATE;
  }
}

cc_status cc_autotune(cc_mesh* m, const double* x, const double* xt, cc_precision p, int32_t sweeps,
                      cc_tune_result* out) {
  CC_API_BODY("cc_autotune", {
    CCG_CHECK(m && x && out, CC_ERR_INVALID_ARG, "NULL argument");
    CCG_CHECK(sweeps >= 1 && sweeps <= 1000, CC_ERR_INVALID_ARG, "sweeps must be in [1, 1000]");
    CCG_CHECK(m->h == 0.0 || xt, CC_ERR_INVALID_ARG, "dynamic mesh needs xtilde");
    cc_sweep_opts so{CC_UPDATE_CC, CC_SCHED_COLORED, p, 0, -1};
    int cb, ce;
    check_sweep_opts(*m, so, &cb, &ce);
    ensure_state(*m, p);
    cudaStream_t s = m->stream;
    DBuf<double> tmp;
    tmp.alloc(3 * m->n);
    cudaEvent_t e0, e1;
    CCG_CUDA(cudaEventCreate(&e0));
    CCG_CUDA(cudaEventCreate(&e1));
    const bool prof = m->prof.on;
    m->prof.on = false;
    auto time_sweeps = [&]() -> double {
      CCG_CUDA(cudaMemcpyAsync(tmp.p, x, 3 * m->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      activate_all(*m);
      if (p == CC_PREC_MIXED) {
        split(*m, tmp.p, m->mx.x_hi.p, m->mx.x_lo.p);
        if (m->h > 0.0) split(*m, xt, m->mx.xt_hi.p, m->mx.xt_lo.p);
      }
      refresh_all(*m, p, tmp.p, xt);
      sweep_body(*m, tmp.p, xt, so, cb, ce, true);  // warm-up sweep
      post_refresh(*m, tmp.p, xt, so, ce);
      CCG_CUDA(cudaEventRecord(e0, s));
      for (int k = 0; k < sweeps; ++k) {
        sweep_body(*m, tmp.p, xt, so, cb, ce, true);
        post_refresh(*m, tmp.p, xt, so, ce);
      }
      CCG_CUDA(cudaEventRecord(e1, s));
      CCG_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      CCG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      return ms / sweeps;
    };
    try {
      // sweep variant first, at the current launch shapes
      {
        const bool rb0 = m->rows_build, fc0 = m->fused_condense;
        int best_v = -1;
        for (int v = 0; v < 4; ++v) {
          out->variant_ms[v] = 0.0;
          m->rows_build = (v >> 1) != 0;
          m->fused_condense = (v & 1) != 0;
          if (m->rows_build && !(p == CC_PREC_MIXED && rows_from_positions(*m))) continue;  // not applicable
          ensure_state(*m, p);
          drop_graph(*m);
          out->variant_ms[v] = time_sweeps();
          if (best_v < 0 || out->variant_ms[v] < out->variant_ms[best_v]) best_v = v;
        }
        m->rows_build = best_v >= 0 ? (best_v >> 1) != 0 : rb0;
        m->fused_condense = best_v >= 0 ? (best_v & 1) != 0 : fc0;
        ensure_state(*m, p);
      }
      const int ct[4] = {32, 64, 128, 256}, gw[3] = {2, 4, 8};
      const int ct0 = m->tune_couple_threads;
      for (int k = 0; k < 4; ++k) {
        m->tune_couple_threads = ct[k];
        try {
          out->couple_ms[k] = time_sweeps();
        } catch (const Fail& f) {
          // a shape whose shared memory this support does not fit is skipped
          if (f.st != CC_ERR_INVALID_ARG) throw;
          CCG_CUDA(cudaStreamSynchronize(s));
          out->couple_ms[k] = 1e30;
        }
      }
      m->tune_couple_threads = ct0;
      int best = 0;
      for (int k = 1; k < 4; ++k)
        if (out->couple_ms[k] < out->couple_ms[best]) best = k;
      m->tune_couple_threads = ct[best];
      const int rl[4] = {1, 2, 4, 8};
      int best_rl = -1;
      for (int k = 0; k < 4; ++k) out->row_lanes_ms[k] = 0.0;
      if (m->tune_couple_threads != 32) {  // the one-warp kernel splits blocks, not rows
        const int keep = m->tune_couple_row_lanes;
        for (int k = 0; k < 4; ++k) {
          m->tune_couple_row_lanes = rl[k];
          out->row_lanes_ms[k] = time_sweeps();
          if (best_rl < 0 || out->row_lanes_ms[k] < out->row_lanes_ms[best_rl]) best_rl = k;
        }
        m->tune_couple_row_lanes = best_rl >= 0 ? rl[best_rl] : keep;
      }
      for (int k = 0; k < 3; ++k) {
        m->tune_gather_wpb = gw[k];
        out->gather_ms[k] = time_sweeps();
      }
      best = 0;
      for (int k = 1; k < 3; ++k)
        if (out->gather_ms[k] < out->gather_ms[best]) best = k;
      m->tune_gather_wpb = gw[best];
    } catch (...) {
      m->prof.on = prof;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      throw;
    }
    m->prof.on = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    drop_graph(*m);
    CCG_CUDA(cudaMemsetAsync(m->d_counters.p, 0, 8 * sizeof(unsigned long long), s));
    CCG_CUDA(cudaStreamSynchronize(s));
    out->couple_threads = m->tune_couple_threads;
    out->couple_row_lanes = m->tune_couple_row_lanes;
    out->gather_warps = m->tune_gather_wpb;
    out->rows_from_positions = m->rows_build ? 1 : 0;
    out->fused_condense = m->fused_condense ? 1 : 0;
  })
}

cc_status cc_set_launch_shape(cc_mesh* m, int32_t couple_threads, int32_t gather_warps, int32_t couple_row_lanes) {
  CC_API_BODY("cc_set_launch_shape", {
    CCG_CHECK(m, CC_ERR_INVALID_ARG, "mesh is NULL");
    CCG_CHECK(couple_row_lanes == 0 || couple_row_lanes == 1 || couple_row_lanes == 2 || couple_row_lanes == 4 ||
                  couple_row_lanes == 8,
              CC_ERR_INVALID_ARG, "couple_row_lanes must be 1, 2, 4 or 8");
    CCG_CHECK(couple_threads == 0 || couple_threads == 32 || couple_threads == 64 || couple_threads == 128 ||
                  couple_threads == 256,
              CC_ERR_INVALID_ARG, "couple_threads must be 32, 64, 128 or 256");
    CCG_CHECK(gather_warps == 0 || gather_warps == 2 || gather_warps == 4 || gather_warps == 8, CC_ERR_INVALID_ARG,
              "gather_warps must be 2, 4 or 8");
    if (couple_threads) m->tune_couple_threads = couple_threads;
    if (gather_warps) m->tune_gather_wpb = gather_warps;
    if (couple_row_lanes) m->tune_couple_row_lanes = couple_row_lanes;
    drop_graph(*m);
  })
}

cc_status cc_set_sweep_variant(cc_mesh* m, int32_t rows_from_positions, int32_t fused_condense) {
  CC_API_BODY("cc_set_sweep_variant", {
    CCG_CHECK(m, CC_ERR_INVALID_ARG, "mesh is NULL");
    CCG_CHECK(rows_from_positions >= -1 && rows_from_positions <= 1 && fused_condense >= -1 && fused_condense <= 1,
              CC_ERR_INVALID_ARG, "variant switches are 1 (on), 0 (off) or -1 (keep)");
    if (rows_from_positions >= 0) m->rows_build = rows_from_positions != 0;
    if (fused_condense >= 0) m->fused_condense = fused_condense != 0;
    drop_graph(*m);
    if (m->mx.gcon.p) ensure_state(*m, CC_PREC_MIXED);  // allocates the per-tet store if the gather path is back
  })
}

cc_status cc_get_info(const cc_mesh* m, cc_mesh_info* info) {
  CC_API_BODY("cc_get_info", {
    CCG_CHECK(m && info, CC_ERR_INVALID_ARG, "NULL argument");
    info->n = m->n;
    info->T = m->T;
    info->n_free = m->n_free;
    info->nnz_blocks = m->nnzb;
    info->num_colors = m->num_colors;
    info->k_ring = m->k_ring;
    info->support_total = (int64_t)m->sup_idx.size();
    info->support_max = m->sup_max;
    info->max_valence = m->max_valence;
    info->patch_float64 = m->last_patch_redo;
    info->patch_solved = m->last_patch_solved;
    info->patch_shared = m->last_patch_shared;
  })
}

cc_status cc_export(const cc_mesh* m, cc_array which, void* dst, int64_t cap, int64_t* count) {
  CC_API_BODY("cc_export", {
    CCG_CHECK(m, CC_ERR_INVALID_ARG, "mesh is NULL");
    const void* src = nullptr;
    int64_t len = 0;
    size_t esz = 0;
    std::vector<int64_t> tmp64;
    switch (which) {
      case CC_ARR_VT_PTR: src = m->vt_ptr.data(); len = (int64_t)m->vt_ptr.size(); esz = 8; break;
      case CC_ARR_VT_TET: src = m->vt_tet.data(); len = (int64_t)m->vt_tet.size(); esz = 4; break;
      case CC_ARR_VT_CORNER: src = m->vt_corner.data(); len = (int64_t)m->vt_corner.size(); esz = 4; break;
      case CC_ARR_NBR_PTR: src = m->nbr_ptr.data(); len = (int64_t)m->nbr_ptr.size(); esz = 8; break;
      case CC_ARR_NBR_IDX: src = m->nbr_idx.data(); len = (int64_t)m->nbr_idx.size(); esz = 4; break;
      case CC_ARR_COLOR:
        CCG_CHECK(m->num_colors > 0, CC_ERR_STATE, "not coloured yet");
        src = m->color.data(); len = (int64_t)m->color.size(); esz = 4; break;
      case CC_ARR_SUP_PTR:
        CCG_CHECK(m->k_ring != 0, CC_ERR_STATE, "no subspace yet");
        src = m->sup_ptr.data(); len = (int64_t)m->sup_ptr.size(); esz = 8; break;
      case CC_ARR_SUP_IDX:
        CCG_CHECK(m->k_ring != 0, CC_ERR_STATE, "no subspace yet");
        src = m->sup_idx.data(); len = (int64_t)m->sup_idx.size(); esz = 4; break;
      case CC_ARR_U: {
        CCG_CHECK(m->k_ring != 0, CC_ERR_STATE, "no subspace yet");
        // the bases live on the device only
        len = 9 * (int64_t)m->sup_idx.size();
        if (count) *count = len;
        if (dst) {
          CCG_CHECK(cap >= len, CC_ERR_INVALID_ARG, "destination too small");
          if (len) {
            CCG_CUDA(cudaStreamSynchronize(m->stream));
            CCG_CUDA(cudaMemcpy(dst, m->f64.U.p, (size_t)len * sizeof(double), cudaMemcpyDeviceToHost));
          }
        }
        return CC_OK;
      }
      case CC_ARR_MASS: src = m->mass.data(); len = (int64_t)m->mass.size(); esz = 8; break;
      default: CCG_CHECK(false, CC_ERR_INVALID_ARG, "unknown array");
    }
    if (count) *count = len;
    if (dst) {
      CCG_CHECK(cap >= len, CC_ERR_INVALID_ARG, "destination too small");
      if (len) std::memcpy(dst, src, (size_t)len * esz);
    }
  })
}

cc_status cc_profile_enable(cc_mesh* m, int32_t on) {
  CC_API_BODY("cc_profile_enable", {
    CCG_CHECK(m, CC_ERR_INVALID_ARG, "mesh is NULL");
    CCG_CUDA(cudaStreamSynchronize(m->stream));
    if ((on != 0) != m->prof.on) drop_graph(*m);
    m->prof.on = on != 0;
    m->prof.used = 0;
    for (int c = 0; c < CC_PROFILE_CLASSES; ++c) {
      m->prof.acc_ms[c] = 0;
      m->prof.acc_launches[c] = 0;
    }
    m->prof.mark_cls.clear();
    m->prof.mark_begin.clear();
    m->prof.mark_end.clear();
    m->prof.mark_launches.clear();
    m->prof.total_launches = 0;
  })
}

cc_status cc_profile_read(cc_mesh* m, cc_profile* out) {
  CC_API_BODY("cc_profile_read", {
    CCG_CHECK(m && out, CC_ERR_INVALID_ARG, "NULL argument");
    CCG_CUDA(cudaStreamSynchronize(m->stream));
    std::memset(out, 0, sizeof(*out));
    for (size_t k = 0; k < m->prof.mark_cls.size(); ++k) {
      float ms = 0.f;
      CCG_CUDA(cudaEventElapsedTime(&ms, m->prof.pool[m->prof.mark_begin[k]], m->prof.pool[m->prof.mark_end[k]]));
      out->ms[m->prof.mark_cls[k]] += ms;
      out->launches[m->prof.mark_cls[k]] += m->prof.mark_launches[k];
    }
    for (int c = 0; c < CC_PROFILE_CLASSES; ++c) {
      out->ms[c] += m->prof.acc_ms[c];
      out->launches[c] += m->prof.acc_launches[c];
      m->prof.acc_ms[c] = 0;
      m->prof.acc_launches[c] = 0;
    }
    out->total_launches = m->prof.total_launches;
    m->prof.used = 0;
    m->prof.mark_cls.clear();
    m->prof.mark_begin.clear();
    m->prof.mark_end.clear();
    m->prof.mark_launches.clear();
    m->prof.total_launches = 0;
  })
}

}  // extern "C"
