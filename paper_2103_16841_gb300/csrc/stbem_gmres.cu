// Restarted GMRES(m) with the whole Arnoldi step on the device (the paper
// names no linear solver). Every column (vector k, segment s) is its own
// Krylov process: a column is one right-hand side of one operator, and the
// segments are the independent operators of a batch (block-diagonal A), so
// one launch sequence advances all of them. Per step: w = A v_j, classical
// Gram-Schmidt with one re-orthogonalisation (dot products reduced in a fixed
// order: chunk partials, then per column), the Givens update of each
// column's Hessenberg column and residual estimate in a kernel with one
// thread per column, and v_{j+1} = w / h_{j+1,j}. The step index lives in
// device memory, so a block of steps is captured once as a CUDA graph and
// replayed; the host reads the number of active columns between blocks.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "stbem_internal.h"

namespace stbem {

namespace {

constexpr int CH = 2048;        // entries per dot-product chunk
constexpr int TPB = 256;


__device__ __forceinline__ int col_of(int64_t idx, int64_t N, int S, const int32_t* seg_of) {
  const int64_t k = idx / N;
  const int64_t i = idx - k * N;
  return (int)(k * S + (S > 1 ? seg_of[i] : 0));
}

// partial[i][item] = sum over the item's entries of V_i * w (i < *nvec)
__global__ void k_dot_partial(const double* __restrict__ V, int64_t ldv, const int* __restrict__ nvec_p, int nvec_add,
                              const double* __restrict__ w, const int64_t* __restrict__ it_start,
                              const int32_t* __restrict__ it_len, int64_t n_items, double* __restrict__ partial) {
  __shared__ double red[TPB / 32];
  const int64_t item = blockIdx.x;
  const int64_t st = it_start[item];
  const int len = it_len[item];
  double wv[CH / TPB];
#pragma unroll
  for (int e = 0; e < CH / TPB; ++e) {
    const int k = threadIdx.x + e * TPB;
    wv[e] = k < len ? w[st + k] : 0.0;
  }
  const int nvec = (nvec_p ? *nvec_p : 0) + nvec_add;
  for (int i = 0; i < nvec; ++i) {
    const double* v = V + (int64_t)i * ldv + st;
    double sacc = 0.0;
#pragma unroll
    for (int e = 0; e < CH / TPB; ++e) {
      const int k = threadIdx.x + e * TPB;
      if (k < len) sacc += v[k] * wv[e];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sacc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tsum = 0.0;
      for (int q = 0; q < TPB / 32; ++q) tsum += red[q];
      partial[(int64_t)i * n_items + item] = tsum;
    }
    __syncthreads();
  }
}

// out[c * ldh + i] = sum over the chunks of column c (in order) of partial[i][.]
__global__ void k_dot_final(const double* __restrict__ partial, int64_t n_items, const int32_t* __restrict__ col_begin,
                            int C, const int* __restrict__ nvec_p, int nvec_add, double* __restrict__ out, int ldh) {
  const int nvec = (nvec_p ? *nvec_p : 0) + nvec_add;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < (int64_t)C * nvec;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(q / nvec), i = (int)(q % nvec);
    double sacc = 0.0;
    for (int it = col_begin[c]; it < col_begin[c + 1]; ++it) sacc += partial[(int64_t)i * n_items + it];
    out[(int64_t)c * ldh + i] = sacc;
  }
}

// w += alpha * sum_{i < nvec} h[c][i] V_i   (c the column of each entry)
__global__ void k_combine(const double* __restrict__ V, int64_t ldv, const double* __restrict__ h, int ldh,
                          const int* __restrict__ nvec_p, int nvec_add, double alpha, double* __restrict__ w, int64_t N,
                          int K, int S, const int32_t* __restrict__ seg_of) {
  const int nvec = (nvec_p ? *nvec_p : 0) + nvec_add;
  const int64_t total = N * K;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int c = col_of(idx, N, S, seg_of);
    const double* hc = h + (int64_t)c * ldh;
    double sacc = 0.0;
    for (int i = 0; i < nvec; ++i) sacc += hc[i] * V[(int64_t)i * ldv + idx];
    w[idx] += alpha * sacc;
  }
}

struct GState {
  int* j;            // current step
  int* nactive;
  double* H;         // [C][(m+1) m] column-major Hessenberg per column
  double* g;         // [C][m+1]
  double* cs;        // [C][m]
  double* sn;
  double* h1;        // [C][m+1] first Gram-Schmidt pass
  double* h2;        // second pass
  double* hn2;       // [C] |w|^2
  double* bnorm;     // [C]
  double* relres;    // [C] residual estimate
  double* scale;     // [C]
  double* y;         // [C][m] solution of the least-squares problem
  int* active;       // [C]
  int* kdim;         // [C]
  int* iters;        // [C]
};

__global__ void k_givens(GState G, int C, int m, double tol) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const int j = *G.j;
  if (!G.active[c]) { G.scale[c] = 0.0; return; }
  double* Hc = G.H + (int64_t)c * (m + 1) * m + (int64_t)j * (m + 1);
  for (int i = 0; i <= j; ++i) Hc[i] = G.h1[(int64_t)c * (m + 1) + i] + G.h2[(int64_t)c * (m + 1) + i];
  const double hn = sqrt(fmax(G.hn2[c], 0.0));
  Hc[j + 1] = hn;
  double* csc = G.cs + (int64_t)c * m;
  double* snc = G.sn + (int64_t)c * m;
  for (int i = 0; i < j; ++i) {
    const double a = Hc[i], b = Hc[i + 1];
    Hc[i] = csc[i] * a + snc[i] * b;
    Hc[i + 1] = -snc[i] * a + csc[i] * b;
  }
  const double a = Hc[j], b = Hc[j + 1];
  const double den = hypot(a, b);
  const double co = den > 0.0 ? a / den : 1.0, si = den > 0.0 ? b / den : 0.0;
  csc[j] = co;
  snc[j] = si;
  Hc[j] = den;
  Hc[j + 1] = 0.0;
  double* gc = G.g + (int64_t)c * (m + 1);
  gc[j + 1] = -si * gc[j];
  gc[j] = co * gc[j];
  G.kdim[c] = j + 1;
  G.iters[c] += 1;
  const double bn = G.bnorm[c];
  const double rel = fabs(gc[j + 1]) / bn;
  G.relres[c] = rel;
  const bool breakdown = !(hn > 1e-300 * fmax(1.0, bn));
  if (rel <= tol || breakdown || j + 1 >= m) G.active[c] = 0;
  G.scale[c] = G.active[c] ? 1.0 / hn : 0.0;
}

// V_{j+1} = scale[c] * w and the product operand vj; then j += 1 (last block)
__global__ void k_next(const double* __restrict__ w, const double* __restrict__ scale, double* __restrict__ V,
                       int64_t ldv, double* __restrict__ vj, const int* __restrict__ jp, int64_t N, int K, int S,
                       const int32_t* __restrict__ seg_of) {
  const int j = *jp;
  const int64_t total = N * K;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const double v = scale[col_of(idx, N, S, seg_of)] * w[idx];
    V[(int64_t)(j + 1) * ldv + idx] = v;
    vj[idx] = v;
  }
}

// j += inc; nactive = number of active columns
__global__ void k_inc(int* j, int inc, const int* active, int C, int* nactive) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *j += inc;
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int n = 0;
  for (int c = threadIdx.x; c < C; c += blockDim.x) n += active[c];
  atomicAdd(&cnt, n);
  __syncthreads();
  if (threadIdx.x == 0) *nactive = cnt;
}

// cycle start: beta = |r| per column, g = beta e_1, V_0 = r / beta
__global__ void k_cycle_init(GState G, int C, int m, double tol) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c == 0) *G.j = 0;
  if (c >= C) return;
  const double beta = sqrt(fmax(G.hn2[c], 0.0));
  const double bn = G.bnorm[c];
  const double rel = bn > 0.0 ? beta / bn : 0.0;
  G.relres[c] = rel;
  const int act = (rel > tol) && beta > 0.0;
  G.active[c] = act;
  G.kdim[c] = 0;
  double* gc = G.g + (int64_t)c * (m + 1);
  for (int i = 0; i <= m; ++i) gc[i] = 0.0;
  gc[0] = act ? beta : 0.0;
  G.scale[c] = act ? 1.0 / beta : 0.0;
}

__global__ void k_scale0(const double* __restrict__ r, const double* __restrict__ scale, double* __restrict__ V0,
                         double* __restrict__ vj, int64_t N, int K, int S, const int32_t* __restrict__ seg_of) {
  const int64_t total = N * K;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const double v = scale[col_of(idx, N, S, seg_of)] * r[idx];
    V0[idx] = v;
    vj[idx] = v;
  }
}

// y = H^{-1} g on the first kdim rows (upper triangular after the rotations)
__global__ void k_backsolve(GState G, int C, int m) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  const int kd = G.kdim[c];
  const double* Hc = G.H + (int64_t)c * (m + 1) * m;
  const double* gc = G.g + (int64_t)c * (m + 1);
  double* yc = G.y + (int64_t)c * m;
  for (int i = m - 1; i >= kd; --i) yc[i] = 0.0;
  for (int i = kd - 1; i >= 0; --i) {
    double sacc = gc[i];
    for (int q = i + 1; q < kd; ++q) sacc -= Hc[i + (int64_t)q * (m + 1)] * yc[q];
    yc[i] = sacc / Hc[i + (int64_t)i * (m + 1)];
  }
}

__global__ void k_residual(const double* __restrict__ b, const double* __restrict__ ax, double* __restrict__ r,
                           int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = b[i] - ax[i];
}

unsigned grid_of(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); }

// GMRES workspace, allocated and released stream-ordered on the solve's
// stream (no device-wide synchronization when it is freed, so the solves of
// concurrent requests on other streams keep running)
template <typename T>
struct DA {
  T* p = nullptr;
  cudaStream_t st = nullptr;
  ~DA() { if (p) cudaFreeAsync(p, st); }
  bem_status alloc(int64_t n, bool zero, cudaStream_t s) {
    st = s;
    if (cudaMallocAsync((void**)&p, sizeof(T) * std::max<int64_t>(n, 1), s) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      set_error("out of device memory (GMRES workspace)");
      return BEM_ERR_OUT_OF_MEMORY;
    }
    if (zero && cudaMemsetAsync(p, 0, sizeof(T) * std::max<int64_t>(n, 1), s) != cudaSuccess) {
      set_error("cudaMemsetAsync failed");
      return BEM_ERR_CUDA;
    }
    return BEM_OK;
  }
};

#define G_TRY(x)                     \
  do {                               \
    bem_status st_ = (x);            \
    if (st_ != BEM_OK) return st_;   \
  } while (0)


// chunks of every column, column by column (host tables kept alive until
// the uploads are done: the caller synchronizes before they go)
struct ItemTables {
  std::vector<int64_t> st;
  std::vector<int32_t> ln, cb;
  DA<int64_t> d_st;
  DA<int32_t> d_ln, d_cb;
  int64_t n = 0;
  bem_status build(const SegLayout& L, cudaStream_t s) {
    const int C = L.K * L.S;
    cb.assign(C + 1, 0);
    for (int k = 0; k < L.K; ++k)
      for (int sg = 0; sg < L.S; ++sg) {
        const int c = k * L.S + sg;
        cb[c] = (int32_t)st.size();
        const int64_t off = (int64_t)k * L.N + L.seg_off[sg], len = L.seg_off[sg + 1] - L.seg_off[sg];
        for (int64_t o = 0; o < len; o += CH) {
          st.push_back(off + o);
          ln.push_back((int32_t)std::min<int64_t>(CH, len - o));
        }
      }
    cb[C] = (int32_t)st.size();
    n = (int64_t)st.size();
    G_TRY(d_st.alloc(n, false, s));
    G_TRY(d_ln.alloc(n, false, s));
    G_TRY(d_cb.alloc(C + 1, false, s));
    STBEM_CUDA(cudaMemcpyAsync(d_st.p, st.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice, s));
    STBEM_CUDA(cudaMemcpyAsync(d_ln.p, ln.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    STBEM_CUDA(cudaMemcpyAsync(d_cb.p, cb.data(), sizeof(int32_t) * (C + 1), cudaMemcpyHostToDevice, s));
    return BEM_OK;
  }
};

}  // namespace

bem_status seg_norms(const SegLayout& L, const double* v, std::vector<double>& out, cudaStream_t s) {
  const int C = L.K * L.S;
  ItemTables T;
  G_TRY(T.build(L, s));
  DA<double> partial, res;
  G_TRY(partial.alloc(T.n, false, s));
  G_TRY(res.alloc(C, false, s));
  k_dot_partial<<<(unsigned)std::max<int64_t>(T.n, 1), TPB, 0, s>>>(v, 0, nullptr, 1, v, T.d_st.p, T.d_ln.p, T.n,
                                                                     partial.p);
  k_dot_final<<<(unsigned)((C + 63) / 64), 64, 0, s>>>(partial.p, T.n, T.d_cb.p, C, nullptr, 1, res.p, 1);
  STBEM_CUDA(cudaGetLastError());
  out.resize(C);
  STBEM_CUDA(cudaMemcpyAsync(out.data(), res.p, sizeof(double) * C, cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaStreamSynchronize(s));
  for (auto& x : out) x = std::sqrt(std::max(x, 0.0));
  return BEM_OK;
}

bem_status gmres_device(const SegLayout& L, const MatvecFn& mv, const double* d_b, double* d_x, double tol, int m,
                        int maxit, std::vector<int>& iters, std::vector<double>& relres, std::vector<int>& conv,
                        cudaStream_t s) {
  const int64_t N = L.N, NN = L.N * L.K;
  const int K = L.K, S = L.S, C = K * S;
  ItemTables T;
  G_TRY(T.build(L, s));
  const int64_t n_items = T.n;
  const int64_t* it_st_p = T.d_st.p;
  const int32_t* it_ln_p = T.d_ln.p;
  const int32_t* it_cb_p = T.d_cb.p;
  DA<int32_t> seg_of;
  const int32_t* d_seg = nullptr;
  if (S > 1) {
    std::vector<int32_t> so(N);
    for (int sg = 0; sg < S; ++sg)
      for (int64_t i = L.seg_off[sg]; i < L.seg_off[sg + 1]; ++i) so[i] = sg;
    G_TRY(seg_of.alloc(N, false, s));
    STBEM_CUDA(cudaMemcpyAsync(seg_of.p, so.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, s));
    d_seg = seg_of.p;
  }
  // workspace
  DA<double> V, w, vj, r, partial, H, g, cs, sn, h1, h2, hn2, bnorm, rel, scale, y;
  DA<int> ints, active, kdim, it;
  G_TRY(V.alloc(NN * (m + 1), true, s));
  G_TRY(w.alloc(NN, false, s));
  G_TRY(vj.alloc(NN, false, s));
  G_TRY(r.alloc(NN, false, s));
  G_TRY(partial.alloc(n_items * (m + 1), false, s));
  G_TRY(H.alloc((int64_t)C * (m + 1) * m, true, s));
  G_TRY(g.alloc((int64_t)C * (m + 1), true, s));
  G_TRY(cs.alloc((int64_t)C * m, true, s));
  G_TRY(sn.alloc((int64_t)C * m, true, s));
  G_TRY(h1.alloc((int64_t)C * (m + 1), true, s));
  G_TRY(h2.alloc((int64_t)C * (m + 1), true, s));
  G_TRY(hn2.alloc(C, true, s));
  G_TRY(bnorm.alloc(C, true, s));
  G_TRY(rel.alloc(C, true, s));
  G_TRY(scale.alloc(C, true, s));
  G_TRY(y.alloc((int64_t)C * m, true, s));
  G_TRY(ints.alloc(4, true, s));
  G_TRY(active.alloc(C, true, s));
  G_TRY(kdim.alloc(C, true, s));
  G_TRY(it.alloc(C, true, s));
  GState G{ints.p, ints.p + 2, H.p, g.p, cs.p, sn.p, h1.p, h2.p, hn2.p, bnorm.p, rel.p, scale.p, y.p,
           active.p, kdim.p, it.p};
  const unsigned gN = grid_of(NN), gC = (unsigned)((C + 63) / 64);
  auto norms2 = [&](const double* v, double* out) -> bem_status {
    k_dot_partial<<<(unsigned)n_items, TPB, 0, s>>>(v, 0, nullptr, 1, v, it_st_p, it_ln_p, n_items, partial.p);
    k_dot_final<<<gC, 64, 0, s>>>(partial.p, n_items, it_cb_p, C, nullptr, 1, out, 1);
    STBEM_CUDA(cudaGetLastError());
    return BEM_OK;
  };
  // ||b|| per column
  G_TRY(norms2(d_b, bnorm.p));
  {
    std::vector<double> bn(C);
    STBEM_CUDA(cudaMemcpyAsync(bn.data(), bnorm.p, sizeof(double) * C, cudaMemcpyDeviceToHost, s));
    STBEM_CUDA(cudaStreamSynchronize(s));
    for (auto& v : bn) v = std::sqrt(std::max(v, 0.0));
    STBEM_CUDA(cudaMemcpyAsync(bnorm.p, bn.data(), sizeof(double) * C, cudaMemcpyHostToDevice, s));
  }
  // one Arnoldi step (all kernels read the step index from G.j)
  auto step = [&]() -> bem_status {
    G_TRY(mv(vj.p, w.p, s));
    for (int pass = 0; pass < 2; ++pass) {
      double* hp = pass == 0 ? h1.p : h2.p;
      k_dot_partial<<<(unsigned)n_items, TPB, 0, s>>>(V.p, NN, G.j, 1, w.p, it_st_p, it_ln_p, n_items, partial.p);
      k_dot_final<<<grid_of((int64_t)C * (m + 1)), 256, 0, s>>>(partial.p, n_items, it_cb_p, C, G.j, 1, hp, m + 1);
      k_combine<<<gN, 256, 0, s>>>(V.p, NN, hp, m + 1, G.j, 1, -1.0, w.p, N, K, S, d_seg);
    }
    G_TRY(norms2(w.p, hn2.p));
    k_givens<<<gC, 64, 0, s>>>(G, C, m, tol);
    k_next<<<gN, 256, 0, s>>>(w.p, scale.p, V.p, NN, vj.p, G.j, N, K, S, d_seg);
    k_inc<<<1, 256, 0, s>>>(G.j, 1, active.p, C, G.nactive);
    STBEM_CUDA(cudaGetLastError());
    return BEM_OK;
  };
  // steps per graph launch; the graph is captured on the first use
  const int q = std::min(m, 8);
  cudaGraphExec_t gexec = nullptr;
  struct ExecGuard {
    cudaGraphExec_t* g;
    ~ExecGuard() { if (*g) cudaGraphExecDestroy(*g); *g = nullptr; }
  } exec_guard{&gexec};
  bool graph_ok = true;
  int total = 0;
  int nact = 0;
  iters.assign(C, 0);
  while (total < maxit) {
    // r = b - A x, beta, V_0
    G_TRY(mv(d_x, w.p, s));
    k_residual<<<gN, 256, 0, s>>>(d_b, w.p, r.p, NN);
    G_TRY(norms2(r.p, hn2.p));
    k_cycle_init<<<gC, 64, 0, s>>>(G, C, m, tol);
    k_scale0<<<gN, 256, 0, s>>>(r.p, scale.p, V.p, vj.p, N, K, S, d_seg);
    k_inc<<<1, 256, 0, s>>>(G.j, 0, active.p, C, G.nactive);
    STBEM_CUDA(cudaGetLastError());
    STBEM_CUDA(cudaMemcpyAsync(&nact, G.nactive, sizeof(int), cudaMemcpyDeviceToHost, s));
    STBEM_CUDA(cudaStreamSynchronize(s));
    if (nact == 0) break;
    if (cancel_requested()) { set_error("solve cancelled"); return BEM_ERR_CANCELLED; }
    int j = 0;
    while (j < m && total < maxit && nact > 0) {
      const int nb = std::min(q, m - j);
      if (nb == q && graph_ok) {
        if (!gexec) {
          cudaGraph_t graph = nullptr;
          if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            bem_status cst = BEM_OK;
            for (int u = 0; u < q && cst == BEM_OK; ++u) cst = step();
            cudaError_t ce = cudaStreamEndCapture(s, &graph);
            if (cst == BEM_OK && ce == cudaSuccess && graph &&
                cudaGraphInstantiate(&gexec, graph, 0) == cudaSuccess) {
              cudaGraphDestroy(graph);
            } else {
              if (graph) cudaGraphDestroy(graph);
              gexec = nullptr;
              graph_ok = false;
              cudaGetLastError();
            }
          } else {
            graph_ok = false;
            cudaGetLastError();
          }
        }
        if (gexec) STBEM_CUDA(cudaGraphLaunch(gexec, s));
        else
          for (int u = 0; u < nb; ++u) G_TRY(step());
      } else {
        for (int u = 0; u < nb; ++u) G_TRY(step());
      }
      j += nb;
      total += nb;
      STBEM_CUDA(cudaMemcpyAsync(&nact, G.nactive, sizeof(int), cudaMemcpyDeviceToHost, s));
      STBEM_CUDA(cudaStreamSynchronize(s));
      if (cancel_requested()) break;   // x += V y below keeps the iterate reached
    }
    // x += V y
    k_backsolve<<<gC, 64, 0, s>>>(G, C, m);
    k_combine<<<gN, 256, 0, s>>>(V.p, NN, y.p, m, nullptr, m, 1.0, d_x, N, K, S, d_seg);
    STBEM_CUDA(cudaGetLastError());
    if (cancel_requested()) {
      STBEM_CUDA(cudaStreamSynchronize(s));
      set_error("solve cancelled");
      return BEM_ERR_CANCELLED;
    }
  }
  // true residuals
  G_TRY(mv(d_x, w.p, s));
  k_residual<<<gN, 256, 0, s>>>(d_b, w.p, r.p, NN);
  G_TRY(norms2(r.p, hn2.p));
  std::vector<double> rn(C), bn(C);
  std::vector<int> itv(C);
  STBEM_CUDA(cudaMemcpyAsync(rn.data(), hn2.p, sizeof(double) * C, cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaMemcpyAsync(bn.data(), bnorm.p, sizeof(double) * C, cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaMemcpyAsync(itv.data(), it.p, sizeof(int) * C, cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaStreamSynchronize(s));
  relres.assign(C, 0.0);
  conv.assign(C, 0);
  for (int c = 0; c < C; ++c) {
    relres[c] = bn[c] > 0 ? std::sqrt(std::max(rn[c], 0.0)) / bn[c] : 0.0;
    conv[c] = relres[c] <= tol * 1.0000001 + 1e-300;
    iters[c] = itv[c];
  }
  return BEM_OK;
}

}  // namespace stbem
