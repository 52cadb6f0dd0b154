// Solve of eq. df_ind (the paper names no linear solver): restarted GMRES on
// the device (stbem_gmres.cu), either in FP64 throughout or with inner solves
// in a lower arithmetic (FP32 / TF32 / BF16 products) inside an FP64
// iterative refinement on the outer residual r = b - A x.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "stbem_internal.h"

namespace stbem {

namespace {
thread_local const std::atomic<int>* t_cancel = nullptr;
}  // namespace

void set_thread_cancel_flag(const std::atomic<int>* flag) { t_cancel = flag; }
bool cancel_requested() { return t_cancel && t_cancel->load(std::memory_order_relaxed) != 0; }

namespace {

__global__ void k_sub(const double* a, const double* b, double* out, int64_t n) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx < n) out[idx] = a[idx] - b[idx];
}

__global__ void k_axpy(double alpha, const double* x, double* y, int64_t n) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx < n) y[idx] += alpha * x[idx];
}

// refinement vectors, stream-ordered like the GMRES workspace
struct Dev {
  double* p = nullptr;
  cudaStream_t st = nullptr;
  ~Dev() { if (p) cudaFreeAsync(p, st); }
  cudaError_t alloc(int64_t n, cudaStream_t s) {
    st = s;
    return cudaMallocAsync((void**)&p, sizeof(double) * n, s);
  }
};

unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

bem_status gmres_solve_layout(const SegLayout& L, const MatvecFn& mv_hi, const MatvecFn& mv_lo,
                              const double* d_b, double* d_x, const bem_solve_opts* o, bem_solve_info* info,
                              cudaStream_t s) {
  const int64_t nn = L.N * L.K;
  const int C = L.K * L.S;
  auto t0 = std::chrono::steady_clock::now();
  STBEM_CUDA(cudaMemsetAsync(d_x, 0, sizeof(double) * nn, s));
  std::vector<int> iters, conv;
  std::vector<double> rel;
  bem_status st;
  int refinements = 0;
  std::vector<int> tot_iters(C, 0);
  if (o->inner_dtype == BEM_DTYPE_FP64) {
    st = gmres_device(L, mv_hi, d_b, d_x, o->tol, o->restart, o->maxit, iters, rel, conv, s);
    if (st != BEM_OK) return st;
    tot_iters = iters;
  } else {
    Dev r, dx, Ax;
    STBEM_CUDA(r.alloc(nn, s));
    STBEM_CUDA(dx.alloc(nn, s));
    STBEM_CUDA(Ax.alloc(nn, s));
    std::vector<double> bn;
    st = seg_norms(L, d_b, bn, s);
    if (st != BEM_OK) return st;
    rel.assign(C, 1.0);
    conv.assign(C, 0);
    // inner tolerance near the unit roundoff of the inner arithmetic: each
    // refinement step contracts the error by about cond(A) * u_inner anyway
    const double u_floor = o->inner_dtype == BEM_DTYPE_BF16 ? 1e-2 : o->inner_dtype == BEM_DTYPE_TF32 ? 1e-3 : 1e-5;
    const double inner_tol = std::max(o->tol, u_floor);
    for (int it = 0; it <= std::max(0, o->max_refine); ++it) {
      st = mv_hi(d_x, Ax.p, s);
      if (st != BEM_OK) return st;
      k_sub<<<nb(nn), 256, 0, s>>>(d_b, Ax.p, r.p, nn);
      std::vector<double> rn;
      st = seg_norms(L, r.p, rn, s);
      if (st != BEM_OK) return st;
      bool done = true;
      for (int c = 0; c < C; ++c) {
        rel[c] = bn[c] > 0 ? rn[c] / bn[c] : 0.0;
        conv[c] = rel[c] <= o->tol;
        done = done && conv[c];
      }
      if (done || it == std::max(0, o->max_refine)) break;
      if (cancel_requested()) { set_error("solve cancelled"); return BEM_ERR_CANCELLED; }
      STBEM_CUDA(cudaMemsetAsync(dx.p, 0, sizeof(double) * nn, s));
      std::vector<int> ci;
      std::vector<double> ri;
      st = gmres_device(L, mv_lo, r.p, dx.p, inner_tol, o->restart, o->maxit, iters, ri, ci, s);
      if (st != BEM_OK) return st;
      for (int c = 0; c < C; ++c) tot_iters[c] += iters[c];
      k_axpy<<<nb(nn), 256, 0, s>>>(1.0, dx.p, d_x, nn);
      ++refinements;
    }
  }
  STBEM_CUDA(cudaStreamSynchronize(s));
  double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  bool allc = true;
  for (int c = 0; c < C; ++c) {
    allc = allc && conv[c];
    if (info) {
      info[c].iterations = tot_iters[c];
      info[c].refinements = refinements;
      info[c].converged = conv[c];
      info[c].reserved = 0;
      info[c].rel_residual = rel[c];
      info[c].solve_ms = ms;
    }
  }
  if (!allc) {
    set_error("GMRES did not reach the requested tolerance");
    return BEM_ERR_NOT_CONVERGED;
  }
  return BEM_OK;
}

bem_status gmres_solve(bem_operator* op, const double* d_b, double* d_x, int nrhs, const bem_solve_opts* o,
                       bem_solve_info* info, cudaStream_t s) {
  SegLayout L;
  L.N = op->mesh->n_tet;
  L.K = nrhs;
  L.S = 1;
  L.seg_off = {0, L.N};
  const int inner = o->inner_dtype;
  MatvecFn hi = [op, nrhs](const double* x, double* y, cudaStream_t st) {
    return op_matvec(op, x, y, nrhs, MV_FP64, st);
  };
  MatvecFn lo = [op, nrhs, inner](const double* x, double* y, cudaStream_t st) {
    return op_matvec(op, x, y, nrhs, inner, st);
  };
  return gmres_solve_layout(L, hi, lo, d_b, d_x, o, info, s);
}

bem_status gmres_solve_two(const bem_operator* hi_op, bem_operator* lo_op, const double* d_b, double* d_x,
                           int nrhs, const bem_solve_opts* o, bem_solve_info* info, cudaStream_t s) {
  SegLayout L;
  L.N = lo_op->mesh->n_tet;
  L.K = nrhs;
  L.S = 1;
  L.seg_off = {0, L.N};
  const int inner = o->inner_dtype;
  MatvecFn hi = [hi_op, nrhs](const double* x, double* y, cudaStream_t st) {
    return op_matvec(hi_op, x, y, nrhs, MV_FP64, st);
  };
  MatvecFn lo = [lo_op, nrhs, inner](const double* x, double* y, cudaStream_t st) {
    return op_matvec(lo_op, x, y, nrhs, inner, st);
  };
  return gmres_solve_layout(L, hi, lo, d_b, d_x, o, info, s);
}

}  // namespace stbem
