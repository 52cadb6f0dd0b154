// C ABI of the library: mesh topology (host), operator lifecycle, data
// movement between the caller's panel numbering and the internal order.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "stbem_internal.h"

namespace stbem {
static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }
}  // namespace stbem

using namespace stbem;

namespace {

template <typename T>
bem_status dalloc(T** p, size_t n) {
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) {
    set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? BEM_ERR_OUT_OF_MEMORY : BEM_ERR_CUDA;
  }
  return BEM_OK;
}

template <typename T>
struct DevBuf {
  T* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
  bem_status alloc(size_t n) { return dalloc(&p, n); }
};

#define TRY(x)                        \
  do {                                \
    bem_status s_ = (x);              \
    if (s_ != BEM_OK) return s_;      \
  } while (0)

bool g_tables_ready = false;

cudaStream_t pick(const bem_context* ctx, void* stream) {
  return stream ? (cudaStream_t)stream : ctx->stream;
}

}  // namespace

extern "C" {

const char* bem_last_error(void) { return g_last_error.c_str(); }
const char* bem_version(void) { return "stbem-gb300 0.1 (sm_103a)"; }

bem_status bem_context_create(int device, bem_context** out) {
  if (!out) { set_error("null out"); return BEM_ERR_INVALID_ARG; }
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) {
    set_error(std::string("no CUDA device: ") + cudaGetErrorString(e));
    return BEM_ERR_CUDA;
  }
  if (device < 0 || device >= n) { set_error("device index out of range"); return BEM_ERR_INVALID_ARG; }
  STBEM_CUDA(cudaSetDevice(device));
  std::unique_ptr<bem_context> ctx(new bem_context());
  ctx->device = device;
  STBEM_CUDA(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  ctx->sm_count = sms;
  if (!g_tables_ready) {
    TRY(upload_gauss_tables());
    g_tables_ready = true;
  }
  *out = ctx.release();
  return BEM_OK;
}

void bem_context_destroy(bem_context* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

bem_status bem_mesh_create(bem_context* ctx, int64_t n_sv, const double* sv_xyz, int64_t n_stv, const int32_t* stv_sv,
                           const double* stv_t, int64_t n_tet, const int32_t* tets, bem_mesh** out) {
  if (!ctx || !out || !sv_xyz || !stv_sv || !stv_t || !tets || n_sv <= 0 || n_stv <= 0 || n_tet <= 0) {
    set_error("bem_mesh_create: invalid argument");
    return BEM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  STBEM_CUDA(cudaSetDevice(ctx->device));
  for (int64_t v = 0; v < n_stv; ++v)
    if (stv_sv[v] < 0 || stv_sv[v] >= n_sv) { set_error("stv_sv out of range"); return BEM_ERR_BAD_MESH; }
  struct TetH {
    int col, dup;
    int cs[3];      // corner spatial ids ascending
    int lo_v[3], hi_v[3];  // space-time vertex at each corner for the lower / upper face
    double tmin, tmax;
    int user;
  };
  std::vector<TetH> T(n_tet);
  std::map<std::array<int, 3>, int> colmap;
  std::vector<std::array<int, 3>> col_corners;
  double scale = 0.0;
  for (int64_t v = 0; v < n_stv; ++v) scale = std::max(scale, std::fabs(stv_t[v]));
  for (int64_t v = 0; v < 3 * n_sv; ++v) scale = std::max(scale, std::fabs(sv_xyz[v]));
  for (int64_t i = 0; i < n_tet; ++i) {
    const int32_t* tv = tets + 4 * i;
    int sid[4];
    for (int k = 0; k < 4; ++k) {
      if (tv[k] < 0 || tv[k] >= n_stv) { set_error("tet vertex out of range"); return BEM_ERR_BAD_MESH; }
      sid[k] = stv_sv[tv[k]];
    }
    std::array<int, 3> cs{};
    int nc = 0;
    for (int k = 0; k < 4; ++k) {
      bool seen = false;
      for (int q = 0; q < nc; ++q) seen |= cs[q] == sid[k];
      if (!seen) {
        if (nc == 3) { nc = 4; break; }
        cs[nc++] = sid[k];
      }
    }
    if (nc != 3) {
      set_error("panel " + std::to_string(i) + " is not flat in Gamma_K x R (needs exactly 3 spatial vertices)");
      return BEM_ERR_BAD_MESH;
    }
    std::sort(cs.begin(), cs.end());
    TetH& h = T[i];
    h.user = (int)i;
    h.dup = -1;
    for (int c = 0; c < 3; ++c) {
      h.cs[c] = cs[c];
      int vs[2], nv = 0;
      for (int k = 0; k < 4; ++k)
        if (sid[k] == cs[c]) vs[nv++] = tv[k];
      if (nv == 1) { h.lo_v[c] = h.hi_v[c] = vs[0]; }
      else {
        if (stv_t[vs[0]] == stv_t[vs[1]]) {
          set_error("panel " + std::to_string(i) + " has a vertical edge of zero length");
          return BEM_ERR_BAD_MESH;
        }
        bool first_lo = stv_t[vs[0]] < stv_t[vs[1]];
        h.lo_v[c] = first_lo ? vs[0] : vs[1];
        h.hi_v[c] = first_lo ? vs[1] : vs[0];
        h.dup = c;
      }
    }
    // non-degenerate triangle
    const double* a = sv_xyz + 3 * cs[0];
    const double* b = sv_xyz + 3 * cs[1];
    const double* cc = sv_xyz + 3 * cs[2];
    double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, w[3] = {cc[0] - a[0], cc[1] - a[1], cc[2] - a[2]};
    double nx = u[1] * w[2] - u[2] * w[1], ny = u[2] * w[0] - u[0] * w[2], nz = u[0] * w[1] - u[1] * w[0];
    double l2 = std::max(u[0] * u[0] + u[1] * u[1] + u[2] * u[2], w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    if (!(std::sqrt(nx * nx + ny * ny + nz * nz) > 1e-12 * l2)) {
      set_error("panel " + std::to_string(i) + " has a degenerate spatial triangle");
      return BEM_ERR_BAD_MESH;
    }
    h.tmin = 1e300; h.tmax = -1e300;
    for (int k = 0; k < 4; ++k) {
      h.tmin = std::min(h.tmin, stv_t[tv[k]]);
      h.tmax = std::max(h.tmax, stv_t[tv[k]]);
    }
    auto it = colmap.find(cs);
    if (it == colmap.end()) {
      it = colmap.emplace(cs, (int)col_corners.size()).first;
      col_corners.push_back(cs);
    }
    h.col = it->second;
  }
  const int64_t n_col = (int64_t)col_corners.size();
  // internal order: column, then time
  std::vector<int32_t> perm(n_tet);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) {
    const TetH &A = T[a], &B = T[b];
    if (A.col != B.col) return A.col < B.col;
    if (A.tmin != B.tmin) return A.tmin < B.tmin;
    return A.tmax < B.tmax;
  });
  std::vector<int32_t> iperm(n_tet);
  for (int64_t i = 0; i < n_tet; ++i) iperm[perm[i]] = (int32_t)i;
  std::vector<int32_t> col_tet_begin(n_col + 1, 0);
  for (int64_t i = 0; i < n_tet; ++i) col_tet_begin[T[perm[i]].col + 1]++;
  for (int64_t c = 0; c < n_col; ++c) col_tet_begin[c + 1] += col_tet_begin[c];
  // faces with nu_t != 0, numbered per column in order of first appearance
  std::vector<std::map<std::array<int, 3>, int>> smap(n_col);
  std::vector<std::vector<std::array<int, 3>>> scols(n_col);
  std::vector<int> tlo(n_tet), thi(n_tet);
  for (int64_t i = 0; i < n_tet; ++i) {
    const TetH& h = T[perm[i]];
    std::array<int, 3> klo{h.lo_v[0], h.lo_v[1], h.lo_v[2]}, khi{h.hi_v[0], h.hi_v[1], h.hi_v[2]};
    for (int pass = 0; pass < 2; ++pass) {
      auto& key = pass ? khi : klo;
      auto it = smap[h.col].find(key);
      if (it == smap[h.col].end()) {
        it = smap[h.col].emplace(key, (int)scols[h.col].size()).first;
        scols[h.col].push_back(key);
      }
      (pass ? thi : tlo)[i] = it->second;
    }
  }
  std::vector<int32_t> col_surf_begin(n_col + 1, 0);
  int max_tets = 0, max_surf = 0;
  for (int64_t c = 0; c < n_col; ++c) {
    col_surf_begin[c + 1] = col_surf_begin[c] + (int)scols[c].size();
    max_tets = std::max(max_tets, col_tet_begin[c + 1] - col_tet_begin[c]);
    max_surf = std::max(max_surf, (int)scols[c].size());
  }
  if (max_tets > MAX_COL_TETS || max_surf > MAX_COL_SURF) {
    set_error("more than " + std::to_string(MAX_COL_TETS) + " panels over one spatial triangle");
    return BEM_ERR_UNSUPPORTED;
  }
  const int64_t n_surf = col_surf_begin[n_col];
  std::vector<int32_t> surf_col(n_surf);
  std::vector<double> surf_p(3 * n_surf);
  for (int64_t c = 0; c < n_col; ++c)
    for (size_t s = 0; s < scols[c].size(); ++s) {
      int64_t g = col_surf_begin[c] + s;
      surf_col[g] = (int32_t)c;
      for (int k = 0; k < 3; ++k) surf_p[3 * g + k] = stv_t[scols[c][s][k]];
    }
  std::vector<TetDev> td(n_tet);
  std::vector<double> tvx(16 * n_tet);
  for (int64_t i = 0; i < n_tet; ++i) {
    const TetH& h = T[perm[i]];
    TetDev& d = td[i];
    d.col = h.col;
    d.lo = col_surf_begin[h.col] + tlo[i];
    d.hi = col_surf_begin[h.col] + thi[i];
    d.dup = h.dup;
    d.tmin = h.tmin;
    d.tmax = h.tmax;
    bool first = i == col_tet_begin[h.col];
    d.pmax = first ? h.tmax : std::max(td[i - 1].pmax, h.tmax);
    for (int c = 0; c < 3; ++c) d.vt[c] = stv_t[h.lo_v[c]];
    d.vt[3] = stv_t[h.hi_v[h.dup]];
    for (int k = 0; k < 5; ++k) d.ball[k] = 0.0;
    const int32_t* tv = tets + 4 * (int64_t)perm[i];
    for (int k = 0; k < 4; ++k) {
      tvx[16 * i + 4 * k] = stv_t[tv[k]];
      for (int q = 0; q < 3; ++q) tvx[16 * i + 4 * k + 1 + q] = sv_xyz[3 * stv_sv[tv[k]] + q];
    }
  }
  std::vector<int32_t> corner_sv(3 * n_col);
  for (int64_t c = 0; c < n_col; ++c)
    for (int k = 0; k < 3; ++k) corner_sv[3 * c + k] = col_corners[c][k];
  std::unique_ptr<bem_mesh> m(new bem_mesh());
  m->ctx = ctx;
  m->n_tet = n_tet; m->n_col = n_col; m->n_surf = n_surf;
  m->max_col_tets = max_tets; m->max_col_surf = max_surf;
  m->perm = perm; m->iperm = iperm;
  m->col_tet_begin = col_tet_begin; m->col_surf_begin = col_surf_begin;
  m->coord_scale = std::max(scale, 1e-300);
  cudaStream_t s = ctx->stream;
  TRY(dalloc(&m->d_col, n_col));
  TRY(dalloc(&m->d_col_tet_begin, n_col + 1));
  TRY(dalloc(&m->d_col_surf_begin, n_col + 1));
  TRY(dalloc(&m->d_surf, n_surf));
  TRY(dalloc(&m->d_tet, n_tet));
  TRY(dalloc(&m->d_perm, n_tet));
  DevBuf<double> d_sv, d_tvx, d_sp;
  DevBuf<int32_t> d_cs, d_scol;
  TRY(d_sv.alloc(3 * n_sv));
  TRY(d_tvx.alloc(16 * n_tet));
  TRY(d_sp.alloc(3 * n_surf));
  TRY(d_cs.alloc(3 * n_col));
  TRY(d_scol.alloc(n_surf));
  STBEM_CUDA(cudaMemcpyAsync(d_sv.p, sv_xyz, sizeof(double) * 3 * n_sv, cudaMemcpyHostToDevice, s));
  STBEM_CUDA(cudaMemcpyAsync(d_tvx.p, tvx.data(), sizeof(double) * 16 * n_tet, cudaMemcpyHostToDevice, s));
  STBEM_CUDA(cudaMemcpyAsync(d_sp.p, surf_p.data(), sizeof(double) * 3 * n_surf, cudaMemcpyHostToDevice, s));
  STBEM_CUDA(cudaMemcpyAsync(d_cs.p, corner_sv.data(), sizeof(int32_t) * 3 * n_col, cudaMemcpyHostToDevice, s));
  STBEM_CUDA(cudaMemcpyAsync(d_scol.p, surf_col.data(), sizeof(int32_t) * n_surf, cudaMemcpyHostToDevice, s));
  STBEM_CUDA(cudaMemcpyAsync(m->d_tet, td.data(), sizeof(TetDev) * n_tet, cudaMemcpyHostToDevice, s));
  STBEM_CUDA(cudaMemcpyAsync(m->d_col_tet_begin, col_tet_begin.data(), sizeof(int32_t) * (n_col + 1),
                             cudaMemcpyHostToDevice, s));
  STBEM_CUDA(cudaMemcpyAsync(m->d_col_surf_begin, col_surf_begin.data(), sizeof(int32_t) * (n_col + 1),
                             cudaMemcpyHostToDevice, s));
  STBEM_CUDA(cudaMemcpyAsync(m->d_perm, perm.data(), sizeof(int32_t) * n_tet, cudaMemcpyHostToDevice, s));
  TRY(mesh_device_geometry(m.get(), d_sv.p, d_cs.p, d_tvx.p, d_scol.p, d_sp.p));
  STBEM_CUDA(cudaStreamSynchronize(s));
  *out = m.release();
  return BEM_OK;
}

bem_status bem_mesh_create_prisms(bem_context* ctx, int64_t n_sv, const double* sv_xyz, int64_t n_tri,
                                  const int32_t* tri, int32_t n_slabs, const double* time_nodes, bem_mesh** out) {
  if (!ctx || !sv_xyz || !tri || !time_nodes || !out || n_sv <= 0 || n_tri <= 0 || n_slabs <= 0) {
    set_error("bem_mesh_create_prisms: invalid argument");
    return BEM_ERR_INVALID_ARG;
  }
  const int64_t ns1 = n_slabs + 1;
  std::vector<int32_t> stv_sv(n_sv * ns1);
  std::vector<double> stv_t(n_sv * ns1);
  for (int64_t v = 0; v < n_sv; ++v)
    for (int64_t n = 0; n < ns1; ++n) {
      stv_sv[v * ns1 + n] = (int32_t)v;
      stv_t[v * ns1 + n] = time_nodes[v * ns1 + n];
      if (n > 0 && !(time_nodes[v * ns1 + n] > time_nodes[v * ns1 + n - 1])) {
        set_error("time nodes must increase");
        return BEM_ERR_BAD_MESH;
      }
    }
  std::vector<int32_t> tets(12 * n_tri * n_slabs);
  for (int64_t k = 0; k < n_tri; ++k) {
    int v[3] = {tri[3 * k], tri[3 * k + 1], tri[3 * k + 2]};
    std::sort(v, v + 3);
    for (int64_t n = 0; n < n_slabs; ++n) {
      int32_t A0 = (int32_t)(v[0] * ns1 + n), B0 = (int32_t)(v[1] * ns1 + n), C0 = (int32_t)(v[2] * ns1 + n);
      int32_t* t = tets.data() + 12 * (k * n_slabs + n);
      int32_t loc[12] = {A0, B0, C0, A0 + 1, B0, C0, A0 + 1, B0 + 1, C0, A0 + 1, B0 + 1, C0 + 1};
      std::memcpy(t, loc, sizeof(loc));
    }
  }
  return bem_mesh_create(ctx, n_sv, sv_xyz, n_sv * ns1, stv_sv.data(), stv_t.data(), 3 * n_tri * n_slabs,
                         tets.data(), out);
}

bem_status bem_mesh_info(const bem_mesh* m, int64_t* n_tet, int64_t* n_columns, int64_t* n_surfaces) {
  if (!m) { set_error("null mesh"); return BEM_ERR_INVALID_ARG; }
  if (n_tet) *n_tet = m->n_tet;
  if (n_columns) *n_columns = m->n_col;
  if (n_surfaces) *n_surfaces = m->n_surf;
  return BEM_OK;
}

void bem_mesh_destroy(bem_mesh* m) {
  if (!m) return;
  cudaFree(m->d_col); cudaFree(m->d_col_tet_begin); cudaFree(m->d_col_surf_begin);
  cudaFree(m->d_surf); cudaFree(m->d_tet); cudaFree(m->d_perm);
  delete m;
}

}  // extern "C"

bem_status stbem::op_layout(bem_operator* op, const int32_t* bw, const int64_t* bnnz, bool first, bool own_scratch,
                           cudaStream_t s) {
  const bem_mesh* m = op->mesh;
  const int64_t nb = m->n_col * m->n_col;
  std::vector<int64_t> boff(nb), rsoff(nb);
  int64_t vo = 0, ro = 0, nnz = 0, nblk = 0;
  int wmax = 0;
  for (int64_t I = 0; I < m->n_col; ++I) {
    int R = m->col_tet_begin[I + 1] - m->col_tet_begin[I];
    for (int64_t J = 0; J < m->n_col; ++J) {
      int64_t b = I * m->n_col + J;
      boff[b] = vo;
      rsoff[b] = ro;
      if (bw[b] > 0) {
        vo += (int64_t)R * bw[b];
        ro += R;
        ++nblk;
        wmax = std::max(wmax, bw[b]);
      }
      nnz += bnnz[b];
    }
  }
  if (first) {
    op->nstored = vo; op->nrows_stored = ro; op->nnz = nnz; op->nblocks = nblk;
    op->max_bw = wmax;
    if (own_scratch) {
      const int64_t grid = (int64_t)op->ctx->sm_count * quad_max_per_sm(op, 0);
      op->tmp_len = std::max<int64_t>((int64_t)grid * m->max_col_surf * m->max_col_tets, 2 * m->n_tet * 8);
    } else {
      op->tmp_len = 0;
    }
    if (op->opts.matrix_free) op->nstored = 0;
    if (op->admit) TRY(op->admit(op));
    if (!op->opts.matrix_free) {
      // mixed-precision values carry FP32 accuracy: FP32 storage only
      if (op->opts.precision == BEM_PREC_FP64) TRY(dalloc(&op->d_val, (size_t)vo));
      // (8 floats of tail room: the tensor-core product copies whole 16-byte granules)
      if (op->opts.store_fp32 || op->opts.precision == BEM_PREC_MIXED) TRY(dalloc(&op->d_val32, (size_t)vo + 8));
      TRY(dalloc(&op->d_rs, (size_t)ro + 4));   // (tail room as for the values)
    }
    if (own_scratch) TRY(dalloc(&op->d_tmp, (size_t)op->tmp_len));
  } else if ((!op->opts.matrix_free && vo != op->nstored) || nnz != op->nnz) {
    set_error("reassembly changed the sparsity structure");
    return BEM_ERR_INTERNAL;
  }
  STBEM_CUDA(cudaMemcpyAsync(op->d_boff, boff.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice, s));
  STBEM_CUDA(cudaMemcpyAsync(op->d_rsoff, rsoff.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice, s));
  // the host offsets must stay alive until the copies are done
  STBEM_CUDA(cudaStreamSynchronize(s));
  return BEM_OK;
}

bem_status stbem::op_structure_alloc(bem_context* ctx, const bem_mesh* mesh, const bem_op_opts* opts,
                                     std::unique_ptr<bem_operator>& op) {
  bem_op_opts o{};
  o.precision = BEM_PREC_FP64; o.m_q = 3; o.n_theta = 0; o.store_fp32 = 1;
  if (opts) o = *opts;
  if (o.precision != BEM_PREC_FP64 && o.precision != BEM_PREC_MIXED) {
    set_error("unknown precision"); return BEM_ERR_INVALID_ARG;
  }
  if (o.m_q < 1 || o.m_q > 4) { set_error("m_q must be in 1..4"); return BEM_ERR_UNSUPPORTED; }
  if (o.trial_space == BEM_TRIAL_P1) {
    set_error("trial space P1 (V_h^1) is not built; only P0 (S_h^0)");
    return BEM_ERR_UNSUPPORTED;
  }
  if (o.trial_space != BEM_TRIAL_P0) { set_error("unknown trial_space"); return BEM_ERR_INVALID_ARG; }
  if (o.n_theta != 0 && (o.n_theta < 4 || o.n_theta > MAX_NTHETA)) {
    set_error("n_theta must be 0 or in 4..32");
    return BEM_ERR_INVALID_ARG;
  }
  op.reset(new bem_operator());
  op->ctx = ctx; op->mesh = mesh; op->opts = o;
  op->mq = o.m_q; op->nq = o.m_q * o.m_q; op->n_theta = o.n_theta;
  const int64_t nb = mesh->n_col * mesh->n_col;
  TRY(dalloc(&op->d_pts, (size_t)mesh->n_surf * op->nq * 4));
  TRY(dalloc(&op->d_ptsf, (size_t)mesh->n_surf * op->nq * 4));
  TRY(dalloc(&op->d_pts_trange, (size_t)mesh->n_surf * 2));
  TRY(dalloc(&op->d_bw, (size_t)nb));
  TRY(dalloc(&op->d_bnnz, (size_t)nb));
  TRY(dalloc(&op->d_boff, (size_t)nb));
  TRY(dalloc(&op->d_rsoff, (size_t)nb));
  TRY(dalloc(&op->d_counter, 4));
  return BEM_OK;
}

namespace {

bem_status assemble(bem_operator* op, cudaStream_t s, bool first) {
  const bem_mesh* m = op->mesh;
  const int64_t nb = m->n_col * m->n_col;
  cudaEvent_t e0, e1, ea, eb, ec;
  STBEM_CUDA(cudaEventCreate(&e0));
  STBEM_CUDA(cudaEventCreate(&e1));
  STBEM_CUDA(cudaEventCreate(&ea));
  STBEM_CUDA(cudaEventCreate(&eb));
  STBEM_CUDA(cudaEventCreate(&ec));
  STBEM_CUDA(cudaEventRecord(e0, s));
  TRY(op_outer_points(op, s));
  STBEM_CUDA(cudaEventRecord(ea, s));
  TRY(op_pattern(op, s));
  STBEM_CUDA(cudaEventRecord(eb, s));
  std::vector<int32_t> bw(nb);
  std::vector<int64_t> bnnz(nb);
  STBEM_CUDA(cudaMemcpyAsync(bw.data(), op->d_bw, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaMemcpyAsync(bnnz.data(), op->d_bnnz, sizeof(int64_t) * nb, cudaMemcpyDeviceToHost, s));
  unsigned long long n_inner = 0;
  STBEM_CUDA(cudaMemcpyAsync(&n_inner, op->d_counter + 1, sizeof(n_inner), cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaStreamSynchronize(s));
  op->n_inner = (int64_t)n_inner;
  TRY(op_layout(op, bw.data(), bnnz.data(), first, true, s));
  STBEM_CUDA(cudaEventRecord(ec, s));
  if (!op->opts.matrix_free) TRY(op_quadrature(op, s));
  op->tcv_stale[0] = op->tcv_stale[1] = true;   // the tensor-core product's slots are remade on next use
  STBEM_CUDA(cudaEventRecord(e1, s));
  STBEM_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f, m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventElapsedTime(&m0, e0, ea);
  cudaEventElapsedTime(&m1, ea, eb);
  cudaEventElapsedTime(&m2, eb, ec);
  cudaEventElapsedTime(&m3, ec, e1);
  op->assemble_ms = ms;
  op->phase_ms[0] = m0; op->phase_ms[1] = m1; op->phase_ms[2] = m2; op->phase_ms[3] = m3;
  for (cudaEvent_t e : {e0, e1, ea, eb, ec}) cudaEventDestroy(e);
  STBEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

}  // namespace

int64_t stbem::operator_value_bytes(const bem_operator* op) {
  int64_t b = 0;
  if (op->opts.precision == BEM_PREC_FP64) b += 8 * op->nstored;
  if (op->opts.store_fp32 || op->opts.precision == BEM_PREC_MIXED) b += 4 * op->nstored;
  return b + 4 * op->nrows_stored + 8 * op->tmp_len;
}

extern "C" {

bem_status bem_operator_create(bem_context* ctx, const bem_mesh* mesh, const bem_op_opts* opts, bem_operator** out) {
  return stbem::operator_create(ctx, mesh, opts, nullptr, out);
}

}  // extern "C"

bem_status stbem::operator_create(bem_context* ctx, const bem_mesh* mesh, const bem_op_opts* opts,
                                  std::function<bem_status(const bem_operator*)> admit, bem_operator** out) {
  if (!ctx || !mesh || !out) { set_error("bem_operator_create: invalid argument"); return BEM_ERR_INVALID_ARG; }
  *out = nullptr;
  bem_op_opts o{};
  o.precision = BEM_PREC_FP64; o.m_q = 3; o.n_theta = 0; o.store_fp32 = 1;
  if (opts) o = *opts;
  if (o.precision != BEM_PREC_FP64 && o.precision != BEM_PREC_MIXED) {
    set_error("unknown precision"); return BEM_ERR_INVALID_ARG;
  }
  if (o.m_q < 1 || o.m_q > 4) { set_error("m_q must be in 1..4"); return BEM_ERR_UNSUPPORTED; }
  if (o.trial_space == BEM_TRIAL_P1) {
    set_error("trial space P1 (V_h^1) is not built; only P0 (S_h^0)");
    return BEM_ERR_UNSUPPORTED;
  }
  if (o.trial_space != BEM_TRIAL_P0) { set_error("unknown trial_space"); return BEM_ERR_INVALID_ARG; }
  if (o.n_theta != 0 && (o.n_theta < 4 || o.n_theta > MAX_NTHETA)) {
    set_error("n_theta must be 0 or in 4..32");
    return BEM_ERR_INVALID_ARG;
  }
  STBEM_CUDA(cudaSetDevice(ctx->device));
  std::unique_ptr<bem_operator> op;
  bem_status st = op_structure_alloc(ctx, mesh, &o, op);
  if (st != BEM_OK) { if (op) bem_operator_destroy(op.release()); return st; }
  op->admit = std::move(admit);
  st = assemble(op.get(), ctx->stream, true);
  if (st != BEM_OK) { bem_operator_destroy(op.release()); return st; }
  int64_t nbad = 0;
  double mx = 0.0;
  if (!op->opts.matrix_free) st = op_value_scan(op.get(), &nbad, &mx, ctx->stream);
  if (st == BEM_OK && nbad > 0) {
    set_error(std::to_string(nbad) + " assembled values are not finite");
    st = BEM_ERR_INTERNAL;
  }
  if (st != BEM_OK) { bem_operator_destroy(op.release()); return st; }
  op->admit = nullptr;
  *out = op.release();
  return BEM_OK;
}

extern "C" {

bem_status bem_operator_work(const bem_operator* op, int64_t* inner_integrals) {
  if (!op || !inner_integrals) { set_error("bem_operator_work: invalid argument"); return BEM_ERR_INVALID_ARG; }
  *inner_integrals = op->n_inner;
  return BEM_OK;
}

bem_status bem_operator_check(const bem_operator* op, int64_t* n_nonfinite, double* max_abs) {
  if (op && op->opts.matrix_free) {
    set_error("matrix-free operator: no stored values");
    return BEM_ERR_UNSUPPORTED;
  }
  if (!op) { set_error("null operator"); return BEM_ERR_INVALID_ARG; }
  int64_t nb = 0;
  double mx = 0.0;
  TRY(op_value_scan(op, &nb, &mx, op->ctx->stream));
  if (n_nonfinite) *n_nonfinite = nb;
  if (max_abs) *max_abs = mx;
  int tc_flag = 0;
  TRY(op_tc_error(op, &tc_flag));
  if (tc_flag) {
    set_error("a tensor-core product gave up waiting for its pipeline (its output was set to NaN)");
    return BEM_ERR_DEVICE_TIMEOUT;
  }
  return BEM_OK;
}

bem_status bem_operator_timings(const bem_operator* op, double* ms) {
  if (!op || !ms) { set_error("invalid argument"); return BEM_ERR_INVALID_ARG; }
  for (int k = 0; k < 4; ++k) ms[k] = op->phase_ms[k];
  return BEM_OK;
}

bem_status bem_operator_reassemble(bem_operator* op, void* stream) {
  if (!op) { set_error("null operator"); return BEM_ERR_INVALID_ARG; }
  return assemble(op, pick(op->ctx, stream), false);
}

bem_status bem_operator_stats(const bem_operator* op, int64_t* nnz, int64_t* stored, int64_t* nblocks, double* ms) {
  if (!op) { set_error("null operator"); return BEM_ERR_INVALID_ARG; }
  if (nnz) *nnz = op->nnz;
  if (stored) *stored = op->nstored;
  if (nblocks) *nblocks = op->nblocks;
  if (ms) *ms = op->assemble_ms;
  return BEM_OK;
}

void bem_operator_destroy(bem_operator* op) {
  if (!op) return;
  cudaFree(op->d_pts); cudaFree(op->d_ptsf); cudaFree(op->d_pts_trange); cudaFree(op->d_bw); cudaFree(op->d_bnnz);
  cudaFree(op->d_boff); cudaFree(op->d_rsoff); cudaFree(op->d_rs); cudaFree(op->d_val);
  cudaFree(op->d_val32); cudaFree(op->d_tmp); cudaFree(op->d_counter);
  cudaFree(op->d_ws); cudaFree(op->d_pv);
  cudaFree(op->d_tc_colptr); cudaFree(op->d_tc_blk); cudaFree(op->d_tc_err);
  cudaFree(op->d_tcv[0]); cudaFree(op->d_tcv[1]);
  delete op;
}

bem_status bem_operator_export_pattern(const bem_operator* op, int64_t* rowptr, int32_t* cols) {
  if (!op || !rowptr || !cols) { set_error("invalid argument"); return BEM_ERR_INVALID_ARG; }
  const bem_mesh* m = op->mesh;
  cudaStream_t s = op->ctx->stream;
  const int64_t n = m->n_tet;
  DevBuf<int64_t> cnt, rp;
  DevBuf<int32_t> cl;
  TRY(cnt.alloc(n)); TRY(rp.alloc(n + 1)); TRY(cl.alloc(std::max<int64_t>(op->nnz, 1)));
  STBEM_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int64_t) * n, s));
  TRY(op_pattern_csr(op, cnt.p, rp.p, cl.p, false, s));
  std::vector<int64_t> hc(n), hp(n + 1, 0);
  STBEM_CUDA(cudaMemcpyAsync(hc.data(), cnt.p, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaStreamSynchronize(s));
  for (int64_t i = 0; i < n; ++i) hp[i + 1] = hp[i] + hc[i];
  if (hp[n] != op->nnz) { set_error("pattern count mismatch"); return BEM_ERR_INTERNAL; }
  STBEM_CUDA(cudaMemcpyAsync(rp.p, hp.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s));
  STBEM_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int64_t) * n, s));
  TRY(op_pattern_csr(op, cnt.p, rp.p, cl.p, true, s));
  std::vector<int32_t> hcl(std::max<int64_t>(op->nnz, 1));
  STBEM_CUDA(cudaMemcpyAsync(hcl.data(), cl.p, sizeof(int32_t) * op->nnz, cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaStreamSynchronize(s));
  // caller numbering: row p = perm[i], columns perm[j], sorted
  std::vector<int64_t> ucount(n + 1, 0);
  for (int64_t i = 0; i < n; ++i) ucount[m->perm[i] + 1] = hc[i];
  for (int64_t i = 0; i < n; ++i) ucount[i + 1] += ucount[i];
  for (int64_t i = 0; i <= n; ++i) rowptr[i] = ucount[i];
  for (int64_t i = 0; i < n; ++i) {
    int64_t dst = rowptr[m->perm[i]];
    for (int64_t k = hp[i]; k < hp[i + 1]; ++k) cols[dst + (k - hp[i])] = m->perm[hcl[k]];
    std::sort(cols + dst, cols + dst + hc[i]);
  }
  return BEM_OK;
}

bem_status bem_operator_pattern_rows(const bem_operator* op, int64_t n, const int32_t* rows, int64_t cap,
                                     int64_t* counts, int32_t* cols) {
  if (!op || n < 0 || (n > 0 && (!rows || !counts || (cap > 0 && !cols))) || cap < 0) {
    set_error("bem_operator_pattern_rows: invalid argument");
    return BEM_ERR_INVALID_ARG;
  }
  const bem_mesh* m = op->mesh;
  cudaStream_t s = op->ctx->stream;
  std::vector<int32_t> internal(n);
  std::vector<int64_t> colset;
  for (int64_t k = 0; k < n; ++k) {
    if (rows[k] < 0 || rows[k] >= m->n_tet) { set_error("row out of range"); return BEM_ERR_INVALID_ARG; }
    internal[k] = m->iperm[rows[k]];
    auto it = std::upper_bound(m->col_tet_begin.begin(), m->col_tet_begin.end(), internal[k]);
    colset.push_back((int64_t)(it - m->col_tet_begin.begin()) - 1);
  }
  std::sort(colset.begin(), colset.end());
  colset.erase(std::unique(colset.begin(), colset.end()), colset.end());
  const int64_t nt = m->n_tet;
  DevBuf<int64_t> cnt, rp;
  TRY(cnt.alloc(nt)); TRY(rp.alloc(nt + 1));
  STBEM_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int64_t) * nt, s));
  for (int64_t I : colset) TRY(op_pattern_csr(op, cnt.p, rp.p, nullptr, false, s, I));
  std::vector<int64_t> hc(nt), hp(nt + 1, 0);
  STBEM_CUDA(cudaMemcpyAsync(hc.data(), cnt.p, sizeof(int64_t) * nt, cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaStreamSynchronize(s));
  for (int64_t i = 0; i < nt; ++i) hp[i + 1] = hp[i] + hc[i];
  DevBuf<int32_t> cl;
  TRY(cl.alloc(std::max<int64_t>(hp[nt], 1)));
  STBEM_CUDA(cudaMemcpyAsync(rp.p, hp.data(), sizeof(int64_t) * (nt + 1), cudaMemcpyHostToDevice, s));
  STBEM_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int64_t) * nt, s));
  for (int64_t I : colset) TRY(op_pattern_csr(op, cnt.p, rp.p, cl.p, true, s, I));
  std::vector<int32_t> hcl(std::max<int64_t>(hp[nt], 1));
  STBEM_CUDA(cudaMemcpyAsync(hcl.data(), cl.p, sizeof(int32_t) * hp[nt], cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaStreamSynchronize(s));
  for (int64_t k = 0; k < n; ++k) {
    int32_t i = internal[k];
    std::vector<int32_t> row(hcl.begin() + hp[i], hcl.begin() + hp[i + 1]);
    for (auto& j : row) j = m->perm[j];
    std::sort(row.begin(), row.end());
    counts[k] = (int64_t)row.size();
    for (int64_t q = 0; q < std::min<int64_t>(cap, (int64_t)row.size()); ++q) cols[k * cap + q] = row[q];
  }
  return BEM_OK;
}

bem_status bem_operator_export_dense(const bem_operator* op, double* A) {
  if (op && op->opts.matrix_free) {
    set_error("matrix-free operator: no stored values");
    return BEM_ERR_UNSUPPORTED;
  }
  if (!op || !A) { set_error("invalid argument"); return BEM_ERR_INVALID_ARG; }
  const bem_mesh* m = op->mesh;
  const int64_t n = m->n_tet, nb = m->n_col * m->n_col;
  if (n > 20000) { set_error("export_dense: mesh too large"); return BEM_ERR_UNSUPPORTED; }
  cudaStream_t s = op->ctx->stream;
  std::vector<int32_t> bw(nb), rs(std::max<int64_t>(op->nrows_stored, 1));
  std::vector<int64_t> boff(nb), rsoff(nb);
  std::vector<double> val(std::max<int64_t>(op->nstored, 1));
  std::vector<float> val32(op->d_val ? 1 : std::max<int64_t>(op->nstored, 1));
  STBEM_CUDA(cudaMemcpyAsync(bw.data(), op->d_bw, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaMemcpyAsync(boff.data(), op->d_boff, sizeof(int64_t) * nb, cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaMemcpyAsync(rsoff.data(), op->d_rsoff, sizeof(int64_t) * nb, cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaMemcpyAsync(rs.data(), op->d_rs, sizeof(int32_t) * op->nrows_stored, cudaMemcpyDeviceToHost, s));
  if (op->d_val)
    STBEM_CUDA(cudaMemcpyAsync(val.data(), op->d_val, sizeof(double) * op->nstored, cudaMemcpyDeviceToHost, s));
  else
    STBEM_CUDA(cudaMemcpyAsync(val32.data(), op->d_val32, sizeof(float) * op->nstored, cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaStreamSynchronize(s));
  if (!op->d_val)
    for (int64_t k = 0; k < op->nstored; ++k) val[k] = (double)val32[k];
  std::memset(A, 0, sizeof(double) * n * n);
  for (int64_t I = 0; I < m->n_col; ++I) {
    int t0 = m->col_tet_begin[I], R = m->col_tet_begin[I + 1] - t0;
    for (int64_t J = 0; J < m->n_col; ++J) {
      int64_t b = I * m->n_col + J;
      if (!bw[b]) continue;
      int jend = m->col_tet_begin[J + 1];
      for (int r = 0; r < R; ++r) {
        int st = rs[rsoff[b] + r];
        for (int w = 0; w < bw[b]; ++w) {
          int j = st + w;
          if (j >= jend) break;
          A[(int64_t)m->perm[t0 + r] * n + m->perm[j]] = val[boff[b] + (int64_t)w * R + r];
        }
      }
    }
  }
  return BEM_OK;
}

bem_status bem_operator_entries(const bem_operator* op, int64_t n, const int32_t* ij, double* out) {
  if (op && op->opts.matrix_free) {
    set_error("matrix-free operator: no stored values");
    return BEM_ERR_UNSUPPORTED;
  }
  if (!op || (n > 0 && (!ij || !out)) || n < 0) { set_error("invalid argument"); return BEM_ERR_INVALID_ARG; }
  if (n == 0) return BEM_OK;
  const bem_mesh* m = op->mesh;
  std::vector<int32_t> in(2 * n);
  for (int64_t k = 0; k < 2 * n; ++k) {
    if (ij[k] < 0 || ij[k] >= m->n_tet) { set_error("entry index out of range"); return BEM_ERR_INVALID_ARG; }
    in[k] = m->iperm[ij[k]];
  }
  cudaStream_t s = op->ctx->stream;
  DevBuf<int32_t> dij;
  DevBuf<double> dout;
  TRY(dij.alloc(2 * n)); TRY(dout.alloc(n));
  STBEM_CUDA(cudaMemcpyAsync(dij.p, in.data(), sizeof(int32_t) * 2 * n, cudaMemcpyHostToDevice, s));
  TRY(op_entries(op, n, dij.p, dout.p, s));
  STBEM_CUDA(cudaMemcpyAsync(out, dout.p, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaStreamSynchronize(s));
  return BEM_OK;
}

bem_status bem_rhs(const bem_operator* op, int32_t kind, int32_t nrhs, const double* params, double* b) {
  if (!op || !b || nrhs <= 0 || (kind != BEM_DATA_SIN2_UNIFORM && kind != BEM_DATA_PULSE) ||
      (kind == BEM_DATA_PULSE && !params)) {
    set_error("bem_rhs: invalid argument");
    return BEM_ERR_INVALID_ARG;
  }
  const bem_mesh* m = op->mesh;
  cudaStream_t s = op->ctx->stream;
  const int64_t nn = m->n_tet * nrhs;
  DevBuf<double> dp, db, du;
  TRY(db.alloc(nn)); TRY(du.alloc(nn));
  if (params) {
    TRY(dp.alloc(5 * nrhs));
    STBEM_CUDA(cudaMemcpyAsync(dp.p, params, sizeof(double) * 5 * nrhs, cudaMemcpyHostToDevice, s));
  }
  TRY(op_rhs(op, kind, nrhs, dp.p, db.p, s));
  TRY(permute(m->d_perm, db.p, du.p, m->n_tet, nrhs, false, s));
  STBEM_CUDA(cudaMemcpyAsync(b, du.p, sizeof(double) * nn, cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaStreamSynchronize(s));
  return BEM_OK;
}

// Room for the two reordered vectors of a product of nn entries each in the
// operator's workspace; grown stream-ordered on s (the previous block is
// released on s after the work already enqueued there).
static bem_status ensure_pv(const bem_operator* op, int64_t nn, cudaStream_t s) {
  if (op->pv_len >= 2 * nn) return BEM_OK;
  if (op->d_pv) STBEM_CUDA(cudaFreeAsync(op->d_pv, s));
  op->d_pv = nullptr;
  op->pv_len = 0;
  cudaError_t e = cudaMallocAsync((void**)&op->d_pv, sizeof(double) * 2 * nn, s);
  if (e != cudaSuccess) {
    op->d_pv = nullptr;
    set_error(std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? BEM_ERR_OUT_OF_MEMORY : BEM_ERR_CUDA;
  }
  op->pv_len = 2 * nn;
  return BEM_OK;
}

static bem_status rhs_rule_args(const bem_operator* op, int32_t level, int32_t n_gauss, int64_t* npps) {
  if (!op || level < 0 || level > 4 || n_gauss < 1 || n_gauss > 16) {
    set_error("bem_rhs_points: level must be in 0..4 and n_gauss in 1..16");
    return BEM_ERR_INVALID_ARG;
  }
  *npps = ((int64_t)1 << (2 * level)) * n_gauss * n_gauss;
  return BEM_OK;
}

bem_status bem_rhs_points(const bem_operator* op, int32_t level, int32_t n_gauss, int64_t* n_pts, double* pts_txyz,
                          double* w) {
  int64_t npps = 0;
  TRY(rhs_rule_args(op, level, n_gauss, &npps));
  if (!n_pts) { set_error("bem_rhs_points: n_pts is null"); return BEM_ERR_INVALID_ARG; }
  const bem_mesh* m = op->mesh;
  const int64_t n = m->n_surf * npps;
  *n_pts = n;
  if (!pts_txyz && !w) return BEM_OK;
  if (!pts_txyz || !w) { set_error("bem_rhs_points: give both arrays or neither"); return BEM_ERR_INVALID_ARG; }
  STBEM_CUDA(cudaSetDevice(op->ctx->device));
  cudaStream_t s = op->ctx->stream;
  DevBuf<double> dp, dw;
  TRY(dp.alloc(4 * n)); TRY(dw.alloc(n));
  TRY(op_rhs_points(op, level, n_gauss, dp.p, dw.p, s));
  STBEM_CUDA(cudaMemcpyAsync(pts_txyz, dp.p, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaMemcpyAsync(w, dw.p, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaStreamSynchronize(s));
  return BEM_OK;
}

bem_status bem_rhs_from_samples(const bem_operator* op, int32_t level, int32_t n_gauss, const double* g,
                                int32_t nrhs, double* b) {
  int64_t npps = 0;
  TRY(rhs_rule_args(op, level, n_gauss, &npps));
  if (!g || !b || nrhs <= 0) { set_error("bem_rhs_from_samples: invalid argument"); return BEM_ERR_INVALID_ARG; }
  const bem_mesh* m = op->mesh;
  const int64_t n = m->n_surf * npps, nn = m->n_tet * (int64_t)nrhs;
  STBEM_CUDA(cudaSetDevice(op->ctx->device));
  cudaStream_t s = op->ctx->stream;
  DevBuf<double> dw, dg, dS, dbi, db;
  TRY(dw.alloc(n)); TRY(dg.alloc(n * nrhs)); TRY(dS.alloc(m->n_surf * nrhs)); TRY(dbi.alloc(nn)); TRY(db.alloc(nn));
  STBEM_CUDA(cudaMemcpyAsync(dg.p, g, sizeof(double) * n * nrhs, cudaMemcpyHostToDevice, s));
  TRY(op_rhs_points(op, level, n_gauss, nullptr, dw.p, s));
  TRY(op_rhs_samples(op, level, n_gauss, dw.p, dg.p, nrhs, dS.p, dbi.p, s));
  TRY(permute(m->d_perm, dbi.p, db.p, m->n_tet, nrhs, false, s));
  STBEM_CUDA(cudaMemcpyAsync(b, db.p, sizeof(double) * nn, cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaStreamSynchronize(s));
  return BEM_OK;
}

bem_status bem_matvec(const bem_operator* op, const double* x_dev, double* y_dev, int32_t nrhs, void* stream) {
  if (!op || !x_dev || !y_dev || nrhs <= 0) { set_error("bem_matvec: invalid argument"); return BEM_ERR_INVALID_ARG; }
  const bem_mesh* m = op->mesh;
  cudaStream_t s = pick(op->ctx, stream);
  const int64_t nn = m->n_tet * nrhs;
  TRY(ensure_pv(op, nn, s));
  double* xi = op->d_pv;
  double* yi = op->d_pv + nn;
  TRY(permute(m->d_perm, x_dev, xi, m->n_tet, nrhs, true, s));
  TRY(op_matvec(op, xi, yi, nrhs, false, s));
  TRY(permute(m->d_perm, yi, y_dev, m->n_tet, nrhs, false, s));
  return BEM_OK;
}

bem_status bem_matvec_dtype(const bem_operator* op, const double* x_dev, double* y_dev, int32_t nrhs, int32_t dtype,
                            void* stream) {
  if (!op || !x_dev || !y_dev || nrhs <= 0 || dtype < BEM_DTYPE_FP64 || dtype > BEM_DTYPE_BF16) {
    set_error("bem_matvec_dtype: invalid argument");
    return BEM_ERR_INVALID_ARG;
  }
  const bem_mesh* m = op->mesh;
  cudaStream_t s = pick(op->ctx, stream);
  const int64_t nn = m->n_tet * nrhs;
  TRY(ensure_pv(op, nn, s));
  double* xi = op->d_pv;
  double* yi = op->d_pv + nn;
  TRY(permute(m->d_perm, x_dev, xi, m->n_tet, nrhs, true, s));
  TRY(op_matvec(op, xi, yi, nrhs, dtype, s));
  TRY(permute(m->d_perm, yi, y_dev, m->n_tet, nrhs, false, s));
  return BEM_OK;
}

bem_status bem_solve_device(bem_operator* op, const double* b_dev, double* w_dev, int32_t nrhs,
                            const bem_solve_opts* opts, bem_solve_info* info, void* stream) {
  if (!op || !b_dev || !w_dev || nrhs <= 0) { set_error("bem_solve: invalid argument"); return BEM_ERR_INVALID_ARG; }
  bem_solve_opts o{1e-8, 50, 2000, BEM_DTYPE_FP64, 10};
  if (opts) o = *opts;
  if (o.restart < 1 || o.restart > 200 || o.maxit < 1 || !(o.tol > 0)) {
    set_error("bem_solve: bad options");
    return BEM_ERR_INVALID_ARG;
  }
  if (o.inner_dtype < BEM_DTYPE_FP64 || o.inner_dtype > BEM_DTYPE_BF16) {
    set_error("bem_solve: unknown inner_dtype");
    return BEM_ERR_INVALID_ARG;
  }
  if ((o.inner_dtype == BEM_DTYPE_FP32 || o.inner_dtype == BEM_DTYPE_TF32) && !op->d_val32) {
    set_error("FP32 / TF32 inner solves need store_fp32 = 1");
    return BEM_ERR_INVALID_ARG;
  }
  const bem_mesh* m = op->mesh;
  cudaStream_t s = pick(op->ctx, stream);
  const int64_t nn = m->n_tet * nrhs;
  DevBuf<double> bi, xi;
  TRY(bi.alloc(nn)); TRY(xi.alloc(nn));
  TRY(permute(m->d_perm, b_dev, bi.p, m->n_tet, nrhs, true, s));
  bem_status st = gmres_solve(op, bi.p, xi.p, nrhs, &o, info, s);
  if (st != BEM_OK && st != BEM_ERR_NOT_CONVERGED && st != BEM_ERR_CANCELLED) return st;
  TRY(permute(m->d_perm, xi.p, w_dev, m->n_tet, nrhs, false, s));
  STBEM_CUDA(cudaStreamSynchronize(s));
  return st;
}

bem_status bem_solve_refined(const bem_operator* op_hi, bem_operator* op_lo, const double* b, double* w,
                             int32_t nrhs, const bem_solve_opts* opts, bem_solve_info* info) {
  if (!op_hi || !op_lo || !b || !w || nrhs <= 0 || !opts) {
    set_error("bem_solve_refined: invalid argument");
    return BEM_ERR_INVALID_ARG;
  }
  if (op_hi->mesh != op_lo->mesh) {
    set_error("bem_solve_refined: the operators must share one mesh");
    return BEM_ERR_INVALID_ARG;
  }
  const bem_solve_opts& o = *opts;
  if (o.inner_dtype != BEM_DTYPE_FP32 && o.inner_dtype != BEM_DTYPE_TF32 && o.inner_dtype != BEM_DTYPE_BF16) {
    set_error("bem_solve_refined: inner_dtype must be FP32, TF32 or BF16");
    return BEM_ERR_INVALID_ARG;
  }
  if (o.restart < 1 || o.restart > 200 || o.maxit < 1 || !(o.tol > 0)) {
    set_error("bem_solve_refined: bad options");
    return BEM_ERR_INVALID_ARG;
  }
  if ((o.inner_dtype == BEM_DTYPE_FP32 || o.inner_dtype == BEM_DTYPE_TF32) && !op_lo->d_val32) {
    set_error("FP32 / TF32 inner solves need FP32 values on op_lo");
    return BEM_ERR_INVALID_ARG;
  }
  if (!op_hi->opts.matrix_free && !op_hi->d_val) {
    set_error("bem_solve_refined: op_hi must hold FP64 values (FP64 precision) or be matrix-free");
    return BEM_ERR_INVALID_ARG;
  }
  const bem_mesh* m = op_lo->mesh;
  cudaStream_t s = op_lo->ctx->stream;
  STBEM_CUDA(cudaSetDevice(op_lo->ctx->device));
  const int64_t nn = m->n_tet * nrhs;
  DevBuf<double> db, bi, xi;
  TRY(db.alloc(nn)); TRY(bi.alloc(nn)); TRY(xi.alloc(nn));
  STBEM_CUDA(cudaMemcpyAsync(db.p, b, sizeof(double) * nn, cudaMemcpyHostToDevice, s));
  TRY(permute(m->d_perm, db.p, bi.p, m->n_tet, nrhs, true, s));
  bem_status st = gmres_solve_two(op_hi, op_lo, bi.p, xi.p, nrhs, &o, info, s);
  if (st != BEM_OK && st != BEM_ERR_NOT_CONVERGED) return st;
  TRY(permute(m->d_perm, xi.p, db.p, m->n_tet, nrhs, false, s));
  STBEM_CUDA(cudaMemcpyAsync(w, db.p, sizeof(double) * nn, cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaStreamSynchronize(s));
  return st;
}

bem_status bem_solve(bem_operator* op, const double* b, double* w, int32_t nrhs, const bem_solve_opts* opts,
                     bem_solve_info* info) {
  if (!op || !b || !w || nrhs <= 0) { set_error("bem_solve: invalid argument"); return BEM_ERR_INVALID_ARG; }
  const int64_t nn = op->mesh->n_tet * nrhs;
  cudaStream_t s = op->ctx->stream;
  DevBuf<double> db, dw;
  TRY(db.alloc(nn)); TRY(dw.alloc(nn));
  STBEM_CUDA(cudaMemcpyAsync(db.p, b, sizeof(double) * nn, cudaMemcpyHostToDevice, s));
  bem_status st = bem_solve_device(op, db.p, dw.p, nrhs, opts, info, s);
  if (st != BEM_OK && st != BEM_ERR_NOT_CONVERGED) return st;
  STBEM_CUDA(cudaMemcpyAsync(w, dw.p, sizeof(double) * nn, cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaStreamSynchronize(s));
  return st;
}

}  // extern "C"

// An asynchronous solve: bem_solve_device run by a worker thread that polls
// the request's cancellation flag between blocks of Arnoldi steps.
struct bem_request {
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv;
  bool done = false;
  bem_status status = BEM_OK;
  std::string error;
  std::vector<bem_solve_info> info;
  std::atomic<int> cancel{0};
};

extern "C" {

bem_status bem_solve_async(bem_operator* op, const double* b_dev, double* w_dev, int32_t nrhs,
                           const bem_solve_opts* opts, void* stream, bem_request** out) {
  if (!op || !b_dev || !w_dev || nrhs <= 0 || !out) {
    set_error("bem_solve_async: invalid argument");
    return BEM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  std::unique_ptr<bem_request> req(new bem_request());
  req->info.resize(nrhs);
  bem_solve_opts o{1e-8, 50, 2000, BEM_DTYPE_FP64, 10};
  if (opts) o = *opts;
  bem_request* r = req.get();
  const int dev = op->ctx->device;
  try {
    r->worker = std::thread([r, op, b_dev, w_dev, nrhs, o, stream, dev]() {
      bem_status st = BEM_OK;
      if (cudaSetDevice(dev) != cudaSuccess) {
        set_error("cudaSetDevice failed in the solve worker");
        st = BEM_ERR_CUDA;
      } else {
        set_thread_cancel_flag(&r->cancel);
        st = bem_solve_device(op, b_dev, w_dev, nrhs, &o, r->info.data(), stream);
        set_thread_cancel_flag(nullptr);
      }
      std::lock_guard<std::mutex> lk(r->mu);
      r->status = st;
      r->error = st == BEM_OK ? std::string() : std::string(bem_last_error());
      r->done = true;
      r->cv.notify_all();
    });
  } catch (...) {
    set_error("bem_solve_async: could not start the worker thread");
    return BEM_ERR_INTERNAL;
  }
  *out = req.release();
  return BEM_OK;
}

bem_status bem_request_wait(bem_request* req, int64_t timeout_ns, bem_solve_info* info) {
  if (!req || timeout_ns < 0) { set_error("bem_request_wait: invalid argument"); return BEM_ERR_INVALID_ARG; }
  std::unique_lock<std::mutex> lk(req->mu);
  if (!req->cv.wait_for(lk, std::chrono::nanoseconds(timeout_ns), [req] { return req->done; })) {
    set_error("bem_request_wait: the solve is still running");
    return BEM_ERR_DEVICE_TIMEOUT;
  }
  if (info) std::copy(req->info.begin(), req->info.end(), info);
  if (req->status != BEM_OK) set_error(req->error);
  return req->status;
}

bem_status bem_request_cancel(bem_request* req) {
  if (!req) { set_error("bem_request_cancel: null request"); return BEM_ERR_INVALID_ARG; }
  req->cancel.store(1);
  return BEM_OK;
}

void bem_request_destroy(bem_request* req) {
  if (!req) return;
  req->cancel.store(1);
  if (req->worker.joinable()) req->worker.join();
  delete req;
}

bem_status bem_inner_potentials(bem_context* ctx, int64_t n, const double* x4, const double* tets,
                                const int32_t* tet_sv, int32_t precision, int32_t n_theta, double* out) {
  if (!ctx || n < 0 || (n > 0 && (!x4 || !tets || !tet_sv || !out))) {
    set_error("bem_inner_potentials: invalid argument");
    return BEM_ERR_INVALID_ARG;
  }
  if (n_theta != 0 && (n_theta < 4 || n_theta > MAX_NTHETA)) {
    set_error("n_theta must be 0 or in 4..32");
    return BEM_ERR_INVALID_ARG;
  }
  if (n == 0) return BEM_OK;
  STBEM_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  DevBuf<double> dx, dt, dout;
  DevBuf<int32_t> dsv;
  TRY(dx.alloc(4 * n)); TRY(dt.alloc(16 * n)); TRY(dout.alloc(n)); TRY(dsv.alloc(4 * n));
  STBEM_CUDA(cudaMemcpyAsync(dx.p, x4, sizeof(double) * 4 * n, cudaMemcpyHostToDevice, s));
  STBEM_CUDA(cudaMemcpyAsync(dt.p, tets, sizeof(double) * 16 * n, cudaMemcpyHostToDevice, s));
  STBEM_CUDA(cudaMemcpyAsync(dsv.p, tet_sv, sizeof(int32_t) * 4 * n, cudaMemcpyHostToDevice, s));
  TRY(inner_potentials(n, dx.p, dt.p, dsv.p, precision, n_theta, dout.p, s));
  STBEM_CUDA(cudaMemcpyAsync(out, dout.p, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaStreamSynchronize(s));
  return BEM_OK;
}

}  // extern "C"
