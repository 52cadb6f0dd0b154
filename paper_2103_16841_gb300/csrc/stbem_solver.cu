// Restarted GMRES for the discrete indirect problem (eq. df_ind). The paper
// names no linear solver; GMRES(m) with classical Gram-Schmidt and one
// re-orthogonalisation pass is used, batched over independent right-hand
// sides (each has its own Krylov space). Reductions run in a fixed order, so
// a right-hand side gives the same bits whatever else is solved beside it.
// With inner_dtype = FP32 the Krylov solves use the FP32 copy of the values
// and an outer FP64 iterative refinement r = b - A x wins the accuracy back.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "stbem_internal.h"

namespace stbem {

// out[j + k*r] = <V_j(:, r), w(:, r)> for j < k; one CTA per (j, r)
__global__ void k_dots(const double* V, int64_t ldv, const double* w, int64_t n, int k, int nrhs, double* out) {
  int j = blockIdx.x % k, r = blockIdx.x / k;
  const double* a = V + (int64_t)j * ldv + (int64_t)r * n;
  const double* b = w + (int64_t)r * n;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += a[i] * b[i];
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j + k * r] = red[0];
}

// w(:, r) += alpha * sum_j h[j + k r] V_j(:, r)
__global__ void k_combine(const double* V, int64_t ldv, const double* h, int k, double alpha, double* w, int64_t n,
                          int nrhs) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * nrhs) return;
  int64_t r = idx / n, i = idx % n;
  double s = 0.0;
  for (int j = 0; j < k; ++j) s += h[j + k * r] * V[(int64_t)j * ldv + r * n + i];
  w[idx] += alpha * s;
}

// out(:, r) = scale[r] * in(:, r)
__global__ void k_scale(const double* in, const double* scale, double* out, int64_t n, int nrhs) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * nrhs) return;
  out[idx] = scale[idx / n] * in[idx];
}

// out = a - b
__global__ void k_sub(const double* a, const double* b, double* out, int64_t n) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx < n) out[idx] = a[idx] - b[idx];
}

__global__ void k_axpy(double alpha, const double* x, double* y, int64_t n) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx < n) y[idx] += alpha * x[idx];
}

namespace {
struct Dev {
  double* p = nullptr;
  ~Dev() { if (p) cudaFree(p); }
};
unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }
}  // namespace

static bem_status norms(const double* v, int64_t n, int nrhs, double* d_tmp, std::vector<double>& out,
                        cudaStream_t s) {
  k_dots<<<nrhs, 256, 0, s>>>(v, 0, v, n, 1, nrhs, d_tmp);
  // k_dots with k = 1 and ldv = 0 indexes V + r*n: the same vector
  STBEM_CUDA(cudaGetLastError());
  out.resize(nrhs);
  STBEM_CUDA(cudaMemcpyAsync(out.data(), d_tmp, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaStreamSynchronize(s));
  for (auto& x : out) x = std::sqrt(std::max(x, 0.0));
  return BEM_OK;
}

// GMRES(m) on A with products in the arithmetic `arith` (MV_*), solving A x = b for all
// columns; x holds the initial guess and the result. Returns per-rhs
// iterations and relative residual estimates.
static bem_status gmres_inner(const bem_operator* op, int arith, const double* b, double* x, int nrhs, double tol,
                              int m, int maxit, std::vector<int>& iters, std::vector<double>& relres,
                              std::vector<int>& conv, cudaStream_t s) {
  const int64_t n = op->mesh->n_tet;
  const int64_t nn = n * nrhs;
  Dev V, w, hbuf, r;
  STBEM_CUDA(cudaMalloc(&V.p, sizeof(double) * nn * (m + 1)));
  STBEM_CUDA(cudaMalloc(&w.p, sizeof(double) * nn));
  STBEM_CUDA(cudaMalloc(&r.p, sizeof(double) * nn));
  STBEM_CUDA(cudaMalloc(&hbuf.p, sizeof(double) * (m + 2) * nrhs * 2));
  std::vector<double> bnorm;
  bem_status st = norms(b, n, nrhs, hbuf.p, bnorm, s);
  if (st != BEM_OK) return st;
  iters.assign(nrhs, 0);
  relres.assign(nrhs, 1.0);
  conv.assign(nrhs, 0);
  std::vector<double> H((size_t)(m + 1) * m * nrhs), cs((size_t)m * nrhs), sn((size_t)m * nrhs),
      g((size_t)(m + 1) * nrhs), hh((size_t)(m + 1) * nrhs), hh2((size_t)(m + 1) * nrhs);
  std::vector<int> kdim(nrhs), active(nrhs);
  int total = 0;
  while (total < maxit) {
    // r = b - A x
    st = op_matvec(op, x, w.p, nrhs, arith, s);
    if (st != BEM_OK) return st;
    k_sub<<<nb(nn), 256, 0, s>>>(b, w.p, r.p, nn);
    std::vector<double> beta;
    st = norms(r.p, n, nrhs, hbuf.p, beta, s);
    if (st != BEM_OK) return st;
    bool all = true;
    std::vector<double> inv(nrhs);
    for (int k = 0; k < nrhs; ++k) {
      double rel = bnorm[k] > 0 ? beta[k] / bnorm[k] : 0.0;
      relres[k] = rel;
      active[k] = !(rel <= tol) && beta[k] > 0.0;
      if (!active[k]) conv[k] = 1;
      all = all && !active[k];
      inv[k] = active[k] ? 1.0 / beta[k] : 0.0;
      g.assign(g.size(), 0.0);
    }
    if (all) break;
    for (int k = 0; k < nrhs; ++k) g[(size_t)k * (m + 1)] = active[k] ? beta[k] : 0.0;
    STBEM_CUDA(cudaMemcpyAsync(hbuf.p, inv.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
    k_scale<<<nb(nn), 256, 0, s>>>(r.p, hbuf.p, V.p, n, nrhs);
    std::fill(kdim.begin(), kdim.end(), 0);
    int j = 0;
    for (; j < m && total < maxit; ++j, ++total) {
      double* Vj = V.p + (int64_t)j * nn;
      st = op_matvec(op, Vj, w.p, nrhs, arith, s);
      if (st != BEM_OK) return st;
      // two classical Gram-Schmidt passes
      for (int pass = 0; pass < 2; ++pass) {
        k_dots<<<(j + 1) * nrhs, 256, 0, s>>>(V.p, nn, w.p, n, j + 1, nrhs, hbuf.p);
        k_combine<<<nb(nn), 256, 0, s>>>(V.p, nn, hbuf.p, j + 1, -1.0, w.p, n, nrhs);
        std::vector<double>& dst = pass == 0 ? hh : hh2;
        STBEM_CUDA(cudaMemcpyAsync(dst.data(), hbuf.p, sizeof(double) * (j + 1) * nrhs, cudaMemcpyDeviceToHost, s));
      }
      std::vector<double> wn;
      st = norms(w.p, n, nrhs, hbuf.p + (m + 2) * nrhs, wn, s);
      if (st != BEM_OK) return st;
      std::vector<double> sc(nrhs);
      bool any = false;
      for (int k = 0; k < nrhs; ++k) {
        if (!active[k]) { sc[k] = 0.0; continue; }
        double* Hk = H.data() + (size_t)k * (m + 1) * m;
        for (int i = 0; i <= j; ++i) Hk[i + (size_t)j * (m + 1)] = hh[i + (size_t)(j + 1) * k] + hh2[i + (size_t)(j + 1) * k];
        double hn = wn[k];
        Hk[j + 1 + (size_t)j * (m + 1)] = hn;
        // apply previous rotations
        for (int i = 0; i < j; ++i) {
          double a = Hk[i + (size_t)j * (m + 1)], c2 = Hk[i + 1 + (size_t)j * (m + 1)];
          double c = cs[(size_t)k * m + i], sv = sn[(size_t)k * m + i];
          Hk[i + (size_t)j * (m + 1)] = c * a + sv * c2;
          Hk[i + 1 + (size_t)j * (m + 1)] = -sv * a + c * c2;
        }
        double a = Hk[j + (size_t)j * (m + 1)], c2 = Hk[j + 1 + (size_t)j * (m + 1)];
        double den = std::hypot(a, c2);
        double c = den > 0 ? a / den : 1.0, sv = den > 0 ? c2 / den : 0.0;
        cs[(size_t)k * m + j] = c;
        sn[(size_t)k * m + j] = sv;
        Hk[j + (size_t)j * (m + 1)] = den;
        Hk[j + 1 + (size_t)j * (m + 1)] = 0.0;
        double* gk = g.data() + (size_t)k * (m + 1);
        gk[j + 1] = -sv * gk[j];
        gk[j] = c * gk[j];
        kdim[k] = j + 1;
        ++iters[k];
        double rel = std::fabs(gk[j + 1]) / bnorm[k];
        relres[k] = rel;
        bool breakdown = !(hn > 1e-300 * std::max(1.0, bnorm[k]));
        if (rel <= tol || breakdown) active[k] = 0;
        sc[k] = active[k] ? 1.0 / hn : 0.0;
        any = any || active[k];
      }
      STBEM_CUDA(cudaMemcpyAsync(hbuf.p, sc.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s));
      k_scale<<<nb(nn), 256, 0, s>>>(w.p, hbuf.p, V.p + (int64_t)(j + 1) * nn, n, nrhs);
      if (!any) { ++j; ++total; break; }
    }
    // x += V y, y from the triangular systems
    int kmax = 0;
    for (int k = 0; k < nrhs; ++k) kmax = std::max(kmax, kdim[k]);
    std::vector<double> y((size_t)kmax * nrhs, 0.0);
    for (int k = 0; k < nrhs; ++k) {
      const double* Hk = H.data() + (size_t)k * (m + 1) * m;
      const double* gk = g.data() + (size_t)k * (m + 1);
      for (int i = kdim[k] - 1; i >= 0; --i) {
        double sum = gk[i];
        for (int q = i + 1; q < kdim[k]; ++q) sum -= Hk[i + (size_t)q * (m + 1)] * y[q + (size_t)kmax * k];
        y[i + (size_t)kmax * k] = sum / Hk[i + (size_t)i * (m + 1)];
      }
    }
    if (kmax > 0) {
      STBEM_CUDA(cudaMemcpyAsync(hbuf.p, y.data(), sizeof(double) * y.size(), cudaMemcpyHostToDevice, s));
      k_combine<<<nb(nn), 256, 0, s>>>(V.p, nn, hbuf.p, kmax, 1.0, x, n, nrhs);
    }
    STBEM_CUDA(cudaGetLastError());
    if (kmax == 0) break;
  }
  // final true residual
  st = op_matvec(op, x, w.p, nrhs, arith, s);
  if (st != BEM_OK) return st;
  k_sub<<<nb(nn), 256, 0, s>>>(b, w.p, r.p, nn);
  std::vector<double> fin;
  st = norms(r.p, n, nrhs, hbuf.p, fin, s);
  if (st != BEM_OK) return st;
  for (int k = 0; k < nrhs; ++k) {
    relres[k] = bnorm[k] > 0 ? fin[k] / bnorm[k] : 0.0;
    conv[k] = relres[k] <= tol * 1.0000001 + 1e-300;
  }
  return BEM_OK;
}

bem_status gmres_solve(bem_operator* op, const double* d_b, double* d_x, int nrhs, const bem_solve_opts* o,
                       bem_solve_info* info, cudaStream_t s) {
  const int64_t n = op->mesh->n_tet, nn = n * nrhs;
  auto t0 = std::chrono::steady_clock::now();
  STBEM_CUDA(cudaMemsetAsync(d_x, 0, sizeof(double) * nn, s));
  std::vector<int> iters, conv;
  std::vector<double> rel;
  bem_status st;
  int refinements = 0;
  std::vector<int> tot_iters(nrhs, 0);
  if (o->inner_dtype == BEM_DTYPE_FP64) {
    st = gmres_inner(op, MV_FP64, d_b, d_x, nrhs, o->tol, o->restart, o->maxit, iters, rel, conv, s);
    if (st != BEM_OK) return st;
    tot_iters = iters;
  } else {
    // FP64 iterative refinement around FP32-valued inner solves
    Dev r, dx, Ax;
    STBEM_CUDA(cudaMalloc(&r.p, sizeof(double) * nn));
    STBEM_CUDA(cudaMalloc(&dx.p, sizeof(double) * nn));
    STBEM_CUDA(cudaMalloc(&Ax.p, sizeof(double) * nn));
    Dev tmp;
    STBEM_CUDA(cudaMalloc(&tmp.p, sizeof(double) * nrhs));
    std::vector<double> bn;
    st = norms(d_b, n, nrhs, tmp.p, bn, s);
    if (st != BEM_OK) return st;
    rel.assign(nrhs, 1.0);
    conv.assign(nrhs, 0);
    // inner tolerance near the unit roundoff of the inner arithmetic: each
    // refinement step contracts the error by about cond(A) * u_inner anyway
    const double u_floor = o->inner_dtype == BEM_DTYPE_BF16 ? 1e-2 : o->inner_dtype == BEM_DTYPE_TF32 ? 1e-3 : 1e-5;
    double inner_tol = std::max(o->tol, u_floor);
    for (int it = 0; it <= std::max(0, o->max_refine); ++it) {
      st = op_matvec(op, d_x, Ax.p, nrhs, MV_FP64, s);
      if (st != BEM_OK) return st;
      k_sub<<<nb(nn), 256, 0, s>>>(d_b, Ax.p, r.p, nn);
      std::vector<double> rn;
      st = norms(r.p, n, nrhs, tmp.p, rn, s);
      if (st != BEM_OK) return st;
      bool done = true;
      for (int k = 0; k < nrhs; ++k) {
        rel[k] = bn[k] > 0 ? rn[k] / bn[k] : 0.0;
        conv[k] = rel[k] <= o->tol;
        done = done && conv[k];
      }
      if (done || it == std::max(0, o->max_refine)) break;
      STBEM_CUDA(cudaMemsetAsync(dx.p, 0, sizeof(double) * nn, s));
      std::vector<int> ci;
      std::vector<double> ri;
      st = gmres_inner(op, o->inner_dtype, r.p, dx.p, nrhs, inner_tol, o->restart, o->maxit, iters, ri, ci, s);
      if (st != BEM_OK) return st;
      for (int k = 0; k < nrhs; ++k) tot_iters[k] += iters[k];
      k_axpy<<<nb(nn), 256, 0, s>>>(1.0, dx.p, d_x, nn);
      ++refinements;
    }
  }
  STBEM_CUDA(cudaStreamSynchronize(s));
  double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  bool allc = true;
  for (int k = 0; k < nrhs; ++k) {
    allc = allc && conv[k];
    if (info) {
      info[k].iterations = tot_iters[k];
      info[k].refinements = refinements;
      info[k].converged = conv[k];
      info[k].reserved = 0;
      info[k].rel_residual = rel[k];
      info[k].solve_ms = ms;
    }
  }
  if (!allc) {
    set_error("GMRES did not reach the requested tolerance");
    return BEM_ERR_NOT_CONVERGED;
  }
  return BEM_OK;
}

}  // namespace stbem
