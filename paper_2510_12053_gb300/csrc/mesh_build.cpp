// Rest-state preprocessing of a tet mesh on the host: orientation, shape
// matrices, volumes, lumped masses and every adjacency structure the kernels
// index with.  Integer outputs follow fixed orders (ascending ids) so that
// they can be compared bit for bit with an independent implementation.
#include <algorithm>
#include <exception>
#include <thread>
#include <functional>
#include <cmath>
#include <cstring>

#include "cc_internal.cuh"

namespace ccg {

// Host worker threads for setup passes over vertex ranges (one per hardware
// thread, at most 32; one for small inputs).
int host_threads(int64_t items) {
  if (items < 20000) return 1;
  const unsigned hc = std::thread::hardware_concurrency();
  return (int)std::max<unsigned>(1, std::min<unsigned>(hc ? hc : 1, 32));
}

void parallel_ranges(int64_t n, int nt, const std::function<void(int, int64_t, int64_t)>& f) {
  if (nt <= 1) {
    f(0, 0, n);
    return;
  }
  std::vector<std::thread> th;
  std::vector<std::exception_ptr> err(nt);
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t]() {
      try {
        f(t, n * t / nt, n * (t + 1) / nt);
      } catch (...) {
        err[t] = std::current_exception();
      }
    });
  for (auto& x : th) x.join();
  for (auto& e : err)
    if (e) std::rethrow_exception(e);
}


static void inverse3(const double* A, double* inv, double* det) {
  double c00 = A[4] * A[8] - A[5] * A[7];
  double c01 = A[5] * A[6] - A[3] * A[8];
  double c02 = A[3] * A[7] - A[4] * A[6];
  double d = A[0] * c00 + A[1] * c01 + A[2] * c02;
  *det = d;
  double id = 1.0 / d;
  inv[0] = c00 * id;
  inv[1] = (A[2] * A[7] - A[1] * A[8]) * id;
  inv[2] = (A[1] * A[5] - A[2] * A[4]) * id;
  inv[3] = c01 * id;
  inv[4] = (A[0] * A[8] - A[2] * A[6]) * id;
  inv[5] = (A[2] * A[3] - A[0] * A[5]) * id;
  inv[6] = c02 * id;
  inv[7] = (A[1] * A[6] - A[0] * A[7]) * id;
  inv[8] = (A[0] * A[4] - A[1] * A[3]) * id;
}

// D_m columns are X_{c+1} - X_0; returns det(D_m).
static double rest_matrix(const std::vector<double>& X, const int32_t* t, double* Dm) {
  for (int c = 0; c < 3; ++c)
    for (int a = 0; a < 3; ++a) Dm[3 * a + c] = X[3 * t[c + 1] + a] - X[3 * t[0] + a];
  return Dm[0] * (Dm[4] * Dm[8] - Dm[5] * Dm[7]) - Dm[1] * (Dm[3] * Dm[8] - Dm[5] * Dm[6]) +
         Dm[2] * (Dm[3] * Dm[7] - Dm[4] * Dm[6]);
}

void build_topology(Mesh& m) {
  const int64_t n = m.n, T = m.T;
  cudaStream_t s = m.stream;
  CCG_CHECK(4 * T < (int64_t(1) << 31) / 4, CC_ERR_INVALID_ARG, "mesh too large for 32-bit entry indices");

  // ---- orientation, shape matrices, volumes, masses
  std::vector<double> Bm(9 * T), vol(T);
  m.mass.assign(n, 0.0);
  for (int64_t t = 0; t < T; ++t) {
    int32_t* tv = &m.tets[4 * t];
    for (int c = 0; c < 4; ++c)
      CCG_CHECK(tv[c] >= 0 && tv[c] < n, CC_ERR_INVALID_ARG, "tet vertex id out of range");
    double Dm[9];
    double det = rest_matrix(m.X, tv, Dm);
    if (det < 0) {
      std::swap(tv[1], tv[2]);
      det = rest_matrix(m.X, tv, Dm);
    }
    CCG_CHECK(det > 0 && std::isfinite(det), CC_ERR_INVALID_ARG, "degenerate (zero-volume) tet");
    double inv[9], d2;
    inverse3(Dm, inv, &d2);
    std::memcpy(&Bm[9 * t], inv, sizeof(inv));
    vol[t] = det / 6.0;
    for (int c = 0; c < 4; ++c) m.mass[tv[c]] += m.tet_rho[t] * vol[t] / 4.0;
  }

  // ---- vertex -> tet lists (ascending tet id) and the entry of every corner
  m.vt_ptr.assign(n + 1, 0);
  for (int64_t t = 0; t < T; ++t)
    for (int c = 0; c < 4; ++c) m.vt_ptr[m.tets[4 * t + c] + 1]++;
  for (int64_t v = 0; v < n; ++v) m.vt_ptr[v + 1] += m.vt_ptr[v];
  m.vt_tet.assign(4 * T, 0);
  m.vt_corner.assign(4 * T, 0);
  std::vector<int32_t> tslot(4 * T);
  {
    std::vector<int64_t> cur(m.vt_ptr.begin(), m.vt_ptr.end() - 1);
    for (int64_t t = 0; t < T; ++t)
      for (int c = 0; c < 4; ++c) {
        int32_t v = m.tets[4 * t + c];
        int64_t e = cur[v]++;
        m.vt_tet[e] = (int32_t)t;
        m.vt_corner[e] = c;
        tslot[4 * t + c] = (int32_t)e;
      }
  }
  m.max_valence = 0;
  for (int64_t v = 0; v < n; ++v)
    m.max_valence = std::max<int32_t>(m.max_valence, (int32_t)(m.vt_ptr[v + 1] - m.vt_ptr[v]));

  // ---- 1-ring neighbours (ascending, self excluded) and the upper block
  //      pattern: row j holds columns l >= j of its 1-ring plus j itself,
  //      ascending, so the diagonal block comes first
  m.nbr_ptr.assign(n + 1, 0);
  m.nbr_idx.clear();
  m.up_ptr.assign(n + 1, 0);
  m.up_col.clear();
  std::vector<int32_t> tmp;
  for (int64_t v = 0; v < n; ++v) {
    tmp.clear();
    for (int64_t e = m.vt_ptr[v]; e < m.vt_ptr[v + 1]; ++e) {
      const int32_t* tv = &m.tets[4 * m.vt_tet[e]];
      for (int c = 0; c < 4; ++c)
        if (tv[c] != v) tmp.push_back(tv[c]);
    }
    std::sort(tmp.begin(), tmp.end());
    tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
    m.nbr_idx.insert(m.nbr_idx.end(), tmp.begin(), tmp.end());
    m.nbr_ptr[v + 1] = (int64_t)m.nbr_idx.size();
    m.up_col.push_back((int32_t)v);
    for (int32_t u : tmp)
      if (u > v) m.up_col.push_back(u);
    m.up_ptr[v + 1] = (int64_t)m.up_col.size();
  }
  m.nnz_up = (int64_t)m.up_col.size();
  m.nnzb = 2 * m.nnz_up - n;
  CCG_CHECK(m.max_valence <= 1024, CC_ERR_INVALID_ARG, "vertex valence above 1024 tets");

  // ---- per upper block (j, l) of a free row, its sources: the blocks
  //      K_{cj,w} of the incident tets t with tets[t][w] == l, as offsets of
  //      the tet's stored upper block pair (min(cj,w), max(cj,w)) in the
  //      per-tet Hessian store (kTetStore values per tet; a diagonal pair,
  //      cj == w, is stored as its upper triangle), bit 31 set when the
  //      stored block must be transposed (cj > w).  Ascending slot order.
  //      The same sources also get a row-local code k * 4 + w (k = the
  //      tet's position in the row's vertex-tet list, w = the corner of l in
  //      it) for the row build, which forms K_{cj,w} itself.
  static const int kPair[4][4] = {{0, 1, 2, 3}, {1, 4, 5, 6}, {2, 5, 7, 8}, {3, 6, 8, 9}};
  std::vector<int32_t> rs_ptr(m.nnz_up + 1, 0);
  std::vector<int32_t> rs_src;
  std::vector<uint16_t> rs_loc;
  for (int64_t v = 0; v < n; ++v) {
    const int64_t p0 = m.up_ptr[v], p1 = m.up_ptr[v + 1];
    if (m.pinned[v]) {
      for (int64_t p = p0; p < p1; ++p) rs_ptr[p + 1] = (int32_t)rs_src.size();
      continue;
    }
    for (int64_t p = p0; p < p1; ++p) {
      const int32_t col = m.up_col[p];
      for (int64_t e = m.vt_ptr[v]; e < m.vt_ptr[v + 1]; ++e) {
        const int64_t t = m.vt_tet[e];
        const int cj = m.vt_corner[e];
        const int32_t* tv = &m.tets[4 * t];
        for (int w = 0; w < 4; ++w)
          if (tv[w] == col) {
            const uint32_t off = (uint32_t)(t * kTetStore + tet_pair_offset(kPair[cj][w]));
            rs_src.push_back((int32_t)(off | (cj > w ? 0x80000000u : 0u)));
            rs_loc.push_back((uint16_t)(((e - m.vt_ptr[v]) << 2) | w));
          }
      }
      rs_ptr[p + 1] = (int32_t)rs_src.size();
    }
  }
  CCG_CHECK((int64_t)kTetStore * T < (int64_t(1) << 31), CC_ERR_INVALID_ARG,
            "mesh too large for 31-bit Hessian offsets");

  m.max_up = 0;
  m.max_rs = 0;
  for (int64_t v = 0; v < n; ++v) {
    m.max_up = std::max<int32_t>(m.max_up, (int32_t)(m.up_ptr[v + 1] - m.up_ptr[v]));
    m.max_rs = std::max<int32_t>(m.max_rs, rs_ptr[m.up_ptr[v + 1]] - rs_ptr[m.up_ptr[v]]);
  }

  // ---- free rows, tets with a free vertex
  std::vector<int32_t> free_rows, active;
  for (int64_t v = 0; v < n; ++v)
    if (!m.pinned[v]) free_rows.push_back((int32_t)v);
  for (int64_t t = 0; t < T; ++t) {
    bool any = false;
    for (int c = 0; c < 4; ++c) any |= !m.pinned[m.tets[4 * t + c]];
    if (any) active.push_back((int32_t)t);
  }
  m.n_free = (int64_t)free_rows.size();
  m.n_active_tets = (int64_t)active.size();

  // ---- upload
  std::vector<float2> Bm_df(9 * T);
  std::vector<float> Bm32(9 * T), Bm32p(12 * T, 0.0f);
  for (int64_t k = 0; k < 9 * T; ++k) {
    float hi = (float)Bm[k];
    Bm_df[k] = make_float2(hi, (float)(Bm[k] - (double)hi));
    Bm32[k] = hi;
    Bm32p[12 * (k / 9) + 4 * ((k % 9) / 3) + k % 3] = hi;  // rows padded to four for 16-byte loads
  }
  auto to32 = [&](const std::vector<int64_t>& a) {
    std::vector<int32_t> r(a.size());
    for (size_t k = 0; k < a.size(); ++k) r[k] = (int32_t)a[k];
    return r;
  };
  m.d_tets.upload(reinterpret_cast<const int4*>(m.tets.data()), T, s);
  m.d_tslot.upload(reinterpret_cast<const int4*>(tslot.data()), T, s);
  m.d_Bm.upload(Bm, s);
  m.d_Bm_df.upload(Bm_df, s);
  m.d_Bm32.upload(Bm32, s);
  m.d_Bm32p.upload(Bm32p, s);
  m.d_vol.upload(vol, s);
  {
    std::vector<double2> m64(T);
    std::vector<float4> mdf(T);
    for (int64_t t = 0; t < T; ++t) {
      const double mu = m.tet_mu[t], lh = m.tet_lh[t];
      m64[t] = make_double2(mu, lh);
      const float mh = (float)mu, lhh = (float)lh;
      mdf[t] = make_float4(mh, (float)(mu - (double)mh), lhh, (float)(lh - (double)lhh));
    }
    m.d_mat64.upload(m64, s);
    m.d_matdf.upload(mdf, s);
    CCG_CUDA(cudaStreamSynchronize(s));
  }
  {
    const double w = m.h > 0.0 ? m.h * m.h : 1.0;
    std::vector<double> vw(T);
    std::vector<float> vw32(T);
    std::vector<float2> vwdf(T);
    for (int64_t t = 0; t < T; ++t) {
      vw[t] = vol[t] * w;
      vw32[t] = (float)vw[t];
      vwdf[t] = make_float2(vw32[t], (float)(vw[t] - (double)vw32[t]));
    }
    m.d_volw.upload(vw, s);
    m.d_volw32.upload(vw32, s);
    m.d_volw_df.upload(vwdf, s);
    std::vector<float> m32(n);
    std::vector<float2> mdf(n);
    for (int64_t v = 0; v < n; ++v) {
      m32[v] = (float)m.mass[v];
      mdf[v] = make_float2(m32[v], (float)(m.mass[v] - (double)m32[v]));
    }
    m.d_mass.upload(m.mass, s);
    m.d_mass32.upload(m32, s);
    m.d_mass_df.upload(mdf, s);
    CCG_CUDA(cudaStreamSynchronize(s));
  }
  m.d_pinned.upload(m.pinned, s);
  auto vt32 = to32(m.vt_ptr), nb32 = to32(m.nbr_ptr), up32 = to32(m.up_ptr);
  m.d_vt_ptr.upload(vt32, s);
  m.d_vt_tet.upload(m.vt_tet, s);
  std::vector<uint8_t> corner8(m.vt_corner.begin(), m.vt_corner.end());
  m.d_vt_corner.upload(corner8, s);
  m.d_nbr_ptr.upload(nb32, s);
  m.d_nbr_idx.upload(m.nbr_idx, s);
  m.d_up_ptr.upload(up32, s);
  m.d_up_col.upload(m.up_col, s);
  m.d_rs_ptr.upload(rs_ptr, s);
  m.d_rs_src.upload(rs_src, s);
  m.d_rs_loc.upload(rs_loc, s);
  m.d_free_rows.upload(free_rows, s);
  {
    // per free row, what the row gather needs first, in one 32-byte record:
    // (j, first upper block, upper blocks, first source), (sources, first
    // vertex-tet entry, entries, 0)
    std::vector<int32_t> hdr(8 * free_rows.size(), 0);
    for (size_t w = 0; w < free_rows.size(); ++w) {
      const int32_t j = free_rows[w];
      const int32_t p0 = (int32_t)m.up_ptr[j], p1 = (int32_t)m.up_ptr[j + 1];
      int32_t* h = &hdr[8 * w];
      h[0] = j;
      h[1] = p0;
      h[2] = p1 - p0;
      h[3] = rs_ptr[p0];
      h[4] = rs_ptr[p1] - rs_ptr[p0];
      h[5] = (int32_t)m.vt_ptr[j];
      h[6] = (int32_t)(m.vt_ptr[j + 1] - m.vt_ptr[j]);
    }
    m.d_row_hdr.upload(reinterpret_cast<const int4*>(hdr.data()), 2 * (int64_t)free_rows.size(), s);
    CCG_CUDA(cudaStreamSynchronize(s));
  }
  m.d_all_tets.upload(active, s);
  {
    if (m.mesh_vptr.empty()) {
      m.mesh_vptr = {0, n};
      m.mesh_tptr = {0, T};
    }
    const int64_t B = (int64_t)m.mesh_vptr.size() - 1;
    std::vector<int32_t> vmesh(n);
    m.mesh_fptr.assign(B + 1, 0);
    for (int64_t b = 0; b < B; ++b)
      for (int64_t v = m.mesh_vptr[b]; v < m.mesh_vptr[b + 1]; ++v) vmesh[v] = (int32_t)b;
    // free rows ascend, and vertex ranges ascend with b, so each mesh's free rows are contiguous
    int64_t f = 0;
    for (int64_t b = 0; b < B; ++b) {
      while (f < (int64_t)free_rows.size() && free_rows[f] < m.mesh_vptr[b + 1]) ++f;
      m.mesh_fptr[b + 1] = (int32_t)f;
    }
    m.d_vert_mesh.upload(vmesh, s);
    m.d_mesh_fptr.upload(m.mesh_fptr, s);
    std::vector<int32_t> ones(B, 1);
    m.d_mesh_active.upload(ones, s);
    m.d_mesh_ones.upload(ones, s);
    m.d_mesh_gsq.alloc(B);
    m.d_mesh_vptr.upload(m.mesh_vptr, s);
    m.d_mesh_tptr.upload(m.mesh_tptr, s);
    m.d_mesh_energy.alloc(B);
    m.d_mesh_alpha.alloc(B);
    CCG_CUDA(cudaStreamSynchronize(s));
  }
  {
    std::vector<int32_t> ids(16 * T);
    for (int64_t e = 0; e < 4 * T; ++e)
      for (int c = 0; c < 4; ++c) ids[4 * e + c] = m.tets[4 * (int64_t)m.vt_tet[e] + c];
    m.d_vt_ids.upload(reinterpret_cast<const int4*>(ids.data()), 4 * T, s);
    CCG_CUDA(cudaStreamSynchronize(s));
  }
  CCG_CUDA(cudaStreamSynchronize(s));  // host vectors above go out of scope
}

}  // namespace ccg
