// Batches of small scatterers: many independent problems of eq. df_ind,
// each on its own mesh, assembled by one persistent launch per pass over the
// blocks of all operators and solved together: the batch operator is block
// diagonal, every (right-hand side, scatterer) is its own GMRES column, and
// the Arnoldi steps of all columns run as captured CUDA graphs.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <memory>
#include <string>
#include <vector>

#include "stbem_internal.h"

using namespace stbem;

#define B_TRY(x)                     \
  do {                               \
    bem_status st_ = (x);            \
    if (st_ != BEM_OK) return st_;   \
  } while (0)

struct bem_batch {
  bem_context* ctx = nullptr;
  std::vector<bem_operator*> ops;
  BatchDev dev;
  BatchMatvec mv;
  double assemble_ms = 0.0;
  int64_t nnz = 0;
  ~bem_batch() {
    for (auto* op : ops) bem_operator_destroy(op);
    cudaFree(dev.d_ctx);
    cudaFree(dev.d_prefix);
    cudaFree(dev.d_counter);
    cudaFree(dev.d_uscratch);
  }
};

namespace {

template <typename T>
bem_status balloc(T** p, int64_t n) {
  if (cudaMalloc((void**)p, sizeof(T) * std::max<int64_t>(n, 1)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_error("out of device memory (batch)");
    return BEM_ERR_OUT_OF_MEMORY;
  }
  return BEM_OK;
}

template <typename T>
struct BBuf {
  T* p = nullptr;
  ~BBuf() { if (p) cudaFree(p); }
};

}  // namespace

extern "C" {

bem_status bem_batch_create(bem_context* ctx, int32_t n, const bem_mesh* const* meshes, const bem_op_opts* opts,
                            bem_batch** out) {
  if (!ctx || n <= 0 || !meshes || !out) { set_error("bem_batch_create: invalid argument"); return BEM_ERR_INVALID_ARG; }
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (!meshes[i] || meshes[i]->ctx->device != ctx->device) {
      set_error("bem_batch_create: null mesh or mesh of another device");
      return BEM_ERR_INVALID_ARG;
    }
  STBEM_CUDA(cudaSetDevice(ctx->device));
  std::unique_ptr<bem_batch> B(new bem_batch());
  B->ctx = ctx;
  cudaStream_t s = ctx->stream;
  for (int i = 0; i < n; ++i) {
    std::unique_ptr<bem_operator> op;
    bem_status st = op_structure_alloc(ctx, meshes[i], opts, op);
    if (st != BEM_OK) { if (op) bem_operator_destroy(op.release()); return st; }
    B->ops.push_back(op.release());
  }
  B_TRY(balloc(reinterpret_cast<unsigned char**>(&B->dev.d_ctx), (int64_t)block_ctx_size() * n));
  B_TRY(balloc(&B->dev.d_prefix, n + 1));
  B_TRY(balloc(&B->dev.d_counter, 1));
  cudaEvent_t e0, e1;
  STBEM_CUDA(cudaEventCreate(&e0));
  STBEM_CUDA(cudaEventCreate(&e1));
  STBEM_CUDA(cudaEventRecord(e0, s));
  B_TRY(op_outer_points_all(B->ops, s));
  B_TRY(op_pattern_batch(B->ops, B->dev, s));
  STBEM_CUDA(cudaStreamSynchronize(s));
  for (bem_operator* op : B->ops) {
    const int64_t nb = op->mesh->n_col * op->mesh->n_col;
    std::vector<int32_t> bw(nb);
    std::vector<int64_t> bnnz(nb);
    STBEM_CUDA(cudaMemcpyAsync(bw.data(), op->d_bw, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, s));
    STBEM_CUDA(cudaMemcpyAsync(bnnz.data(), op->d_bnnz, sizeof(int64_t) * nb, cudaMemcpyDeviceToHost, s));
    STBEM_CUDA(cudaStreamSynchronize(s));
    B_TRY(op_layout(op, bw.data(), bnnz.data(), true, false, s));
    B->nnz += op->nnz;
  }
  B->dev.uscratch_len = quad_batch_scratch(B->ops);
  B_TRY(balloc(&B->dev.d_uscratch, B->dev.uscratch_len));
  B_TRY(op_quadrature_batch(B->ops, B->dev, s));
  STBEM_CUDA(cudaEventRecord(e1, s));
  STBEM_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  B->assemble_ms = ms;
  for (bem_operator* op : B->ops) {
    int64_t nbad = 0;
    double mx = 0.0;
    B_TRY(op_value_scan(op, &nbad, &mx, s));
    if (nbad > 0) {
      set_error(std::to_string(nbad) + " assembled values of a batch operator are not finite");
      return BEM_ERR_INTERNAL;
    }
  }
  B_TRY(B->mv.init(B->ops, s));
  *out = B.release();
  return BEM_OK;
}

bem_status bem_batch_stats(const bem_batch* B, int32_t* n_ops, int64_t* n_tet_total, int64_t* nnz, double* assemble_ms) {
  if (!B) { set_error("null batch"); return BEM_ERR_INVALID_ARG; }
  if (n_ops) *n_ops = (int32_t)B->ops.size();
  if (n_tet_total) *n_tet_total = B->mv.N;
  if (nnz) *nnz = B->nnz;
  if (assemble_ms) *assemble_ms = B->assemble_ms;
  return BEM_OK;
}

bem_status bem_batch_solve(bem_batch* B, int32_t kind, const int32_t* nrhs, const double* params,
                           const bem_solve_opts* opts, double* w, bem_solve_info* info) {
  if (!B || !nrhs || !w || (kind != BEM_DATA_SIN2_UNIFORM && kind != BEM_DATA_PULSE) ||
      (kind == BEM_DATA_PULSE && !params)) {
    set_error("bem_batch_solve: invalid argument");
    return BEM_ERR_INVALID_ARG;
  }
  bem_solve_opts o{1e-8, 50, 2000, BEM_DTYPE_FP64, 10};
  if (opts) o = *opts;
  if (o.restart < 1 || o.restart > 200 || o.maxit < 1 || !(o.tol > 0) || o.inner_dtype < BEM_DTYPE_FP64 ||
      o.inner_dtype > BEM_DTYPE_FP32) {
    set_error("bem_batch_solve: bad options (inner_dtype FP64 or FP32)");
    return BEM_ERR_INVALID_ARG;
  }
  const int S = (int)B->ops.size();
  int K = 0;
  int64_t nr_total = 0;
  for (int i = 0; i < S; ++i) {
    if (nrhs[i] < 1) { set_error("bem_batch_solve: nrhs must be >= 1"); return BEM_ERR_INVALID_ARG; }
    K = std::max(K, (int)nrhs[i]);
    nr_total += nrhs[i];
  }
  STBEM_CUDA(cudaSetDevice(B->ctx->device));
  cudaStream_t s = B->ctx->stream;
  SegLayout L;
  L.N = B->mv.N;
  L.K = K;
  L.S = S;
  L.seg_off.assign(S + 1, 0);
  for (int i = 0; i < S; ++i) L.seg_off[i + 1] = L.seg_off[i] + B->ops[i]->mesh->n_tet;
  const int64_t NN = L.N * K;
  BBuf<double> db, dx, tmp, tmp2, dp;
  B_TRY(balloc(&db.p, NN));
  B_TRY(balloc(&dx.p, NN));
  int64_t max_n = 1;
  for (auto* op : B->ops) max_n = std::max(max_n, op->mesh->n_tet);
  B_TRY(balloc(&tmp.p, max_n * K));
  B_TRY(balloc(&tmp2.p, max_n * K));
  STBEM_CUDA(cudaMemsetAsync(db.p, 0, sizeof(double) * NN, s));
  if (kind == BEM_DATA_PULSE) {
    B_TRY(balloc(&dp.p, 5 * nr_total));
    STBEM_CUDA(cudaMemcpyAsync(dp.p, params, sizeof(double) * 5 * nr_total, cudaMemcpyHostToDevice, s));
  }
  // right-hand sides, operator by operator, into the [K][N] layout
  int64_t prow = 0;
  for (int i = 0; i < S; ++i) {
    const bem_operator* op = B->ops[i];
    const int64_t ni = op->mesh->n_tet;
    B_TRY(op_rhs(op, kind, nrhs[i], dp.p ? dp.p + 5 * prow : nullptr, tmp.p, s));
    STBEM_CUDA(cudaMemcpy2DAsync(db.p + L.seg_off[i], sizeof(double) * L.N, tmp.p, sizeof(double) * ni,
                                 sizeof(double) * ni, nrhs[i], cudaMemcpyDeviceToDevice, s));
    prow += nrhs[i];
  }
  BatchMatvec* mvp = &B->mv;
  const int inner = o.inner_dtype;
  MatvecFn hi = [mvp, K](const double* x, double* y, cudaStream_t st) { return mvp->apply(x, y, K, MV_FP64, st); };
  MatvecFn lo = [mvp, K, inner](const double* x, double* y, cudaStream_t st) {
    return mvp->apply(x, y, K, inner, st);
  };
  std::vector<bem_solve_info> ci((size_t)K * S);
  bem_status st = gmres_solve_layout(L, hi, lo, db.p, dx.p, &o, ci.data(), s);
  if (st != BEM_OK && st != BEM_ERR_NOT_CONVERGED) return st;
  // densities back in each operator's caller order, concatenated
  int64_t woff = 0;
  prow = 0;
  for (int i = 0; i < S; ++i) {
    const bem_operator* op = B->ops[i];
    const int64_t ni = op->mesh->n_tet;
    STBEM_CUDA(cudaMemcpy2DAsync(tmp.p, sizeof(double) * ni, dx.p + L.seg_off[i], sizeof(double) * L.N,
                                 sizeof(double) * ni, nrhs[i], cudaMemcpyDeviceToDevice, s));
    B_TRY(permute(op->mesh->d_perm, tmp.p, tmp2.p, ni, nrhs[i], false, s));
    STBEM_CUDA(cudaMemcpyAsync(w + woff, tmp2.p, sizeof(double) * ni * nrhs[i], cudaMemcpyDeviceToHost, s));
    STBEM_CUDA(cudaStreamSynchronize(s));
    if (info)
      for (int k = 0; k < nrhs[i]; ++k) info[prow + k] = ci[(size_t)k * S + i];
    woff += ni * nrhs[i];
    prow += nrhs[i];
  }
  return st;
}

void bem_batch_destroy(bem_batch* B) { delete B; }

}  // extern "C"
