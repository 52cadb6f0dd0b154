// Kernels of the light-cone-clipped single-layer Galerkin assembly.
//
// Work decomposition: the matrix is cut into blocks (I, J) of panels over
// spatial triangle ("column") I times panels over column J. A persistent
// grid pops blocks from a device counter. For every face F with nu_{F,t} != 0
// over column I and every outer point x_q on F (composite midpoint rule,
// Fig. int_tri_mid), the kernel evaluates the potentials W of the faces over
// column J that the backward light cone of x_q cuts, and forms
//     U[F][j] = sum_q V 1_{sigma_j}(x_q) = sum_q (W_lo(j)(x_q) - W_hi(j)(x_q)),
// then the entries A_ij = |K_I| / m_Q^2 * (U[F_lo(i)][j] - U[F_hi(i)][j])
// (eq. int_bform with nu_{F,t}|F| = -|K| on the lower face, +|K| on the upper).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "stbem_internal.h"

namespace stbem {

static double __longlong_as_double_host(long long b) {
  double d;
  std::memcpy(&d, &b, sizeof(d));
  return d;
}

bem_status upload_gauss_tables() {
  std::vector<double> X(MAX_NTHETA * (MAX_NTHETA + 1) / 2), W(X.size());
  for (int n = 1; n <= MAX_NTHETA; ++n) {
    int off = n * (n - 1) / 2;
    for (int i = 0; i < n; ++i) {
      double z = std::cos(STBEM_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
          double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        if (n == 1) { p1 = z; p0 = 1.0; }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        double dz = p1 / dp;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
      }
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      X[off + i] = z;
      W[off + i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
  }
  std::copy(X.begin(), X.end(), h_gl_x);
  std::copy(W.begin(), W.end(), h_gl_w);
  std::vector<float> Xf(X.begin(), X.end()), Wf(W.begin(), W.end());
  std::copy(Xf.begin(), Xf.end(), h_gl_xf);
  std::copy(Wf.begin(), Wf.end(), h_gl_wf);
  STBEM_CUDA(cudaMemcpyToSymbol(c_gl_x, X.data(), X.size() * sizeof(double)));
  STBEM_CUDA(cudaMemcpyToSymbol(c_gl_w, W.data(), W.size() * sizeof(double)));
  STBEM_CUDA(cudaMemcpyToSymbol(c_gl_xf, Xf.data(), Xf.size() * sizeof(float)));
  STBEM_CUDA(cudaMemcpyToSymbol(c_gl_wf, Wf.data(), Wf.size() * sizeof(float)));
  return BEM_OK;
}

// ---------------------------------------------------------------------------
// Staging: column frames, face gradients, panel balls
// ---------------------------------------------------------------------------
__global__ void k_col_geom(int64_t n_col, const double* sv_xyz, const int32_t* corner_sv, ColGeom* out) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n_col) return;
  const int32_t* s = corner_sv + 3 * c;
  make_colgeom(sv_xyz + 3 * s[0], sv_xyz + 3 * s[1], sv_xyz + 3 * s[2], out[c]);
}

// surf_p [n_surf][3] corner times; surf_col [n_surf]
__global__ void k_surf_geom(int64_t n_surf, const ColGeom* cols, const double* surf_p, const int32_t* surf_col,
                            SurfDev* out) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n_surf) return;
  SurfDev S;
  S.col = surf_col[s];
  S.pad = 0;
  for (int k = 0; k < 3; ++k) S.f.p[k] = surf_p[3 * s + k];
  face_gradient(cols[S.col], S.f);
  out[s] = S;
}

// tet_vx [n_tet][4][4]: the panel's vertices (t,x,y,z) in the caller's order;
// the 4D ball is formed in that order with the fixed operation order of the
// sparsity contract: centre (((X0+X1)+X2)+X3)/4, radius max_v |X_v - c|.
__global__ void k_tet_ball(int64_t n_tet, const double* tet_vx, TetDev* tets) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_tet) return;
  const double* X = tet_vx + 16 * i;
  double c[4];
  for (int d = 0; d < 4; ++d)
    c[d] = __ddiv_rn(__dadd_rn(__dadd_rn(__dadd_rn(X[d], X[4 + d]), X[8 + d]), X[12 + d]), 4.0);
  double mx = 0.0;
  for (int v = 0; v < 4; ++v) {
    double a = __dsub_rn(X[4 * v + 0], c[0]), b = __dsub_rn(X[4 * v + 1], c[1]);
    double e = __dsub_rn(X[4 * v + 2], c[2]), f = __dsub_rn(X[4 * v + 3], c[3]);
    double l = __dsqrt_rn(__dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), __dmul_rn(e, e)),
                                    __dmul_rn(f, f)));
    if (l > mx) mx = l;
  }
  for (int d = 0; d < 4; ++d) tets[i].ball[d] = c[d];
  tets[i].ball[4] = mx;
}

bem_status mesh_device_geometry(bem_mesh* m, const double* d_sv_xyz, const int32_t* d_col_corner_sv,
                                const double* d_tet_vx, const int32_t* d_surf_col, const double* d_surf_p) {
  cudaStream_t s = m->ctx->stream;
  int th = 128;
  k_col_geom<<<(unsigned)((m->n_col + th - 1) / th), th, 0, s>>>(m->n_col, d_sv_xyz, d_col_corner_sv, m->d_col);
  k_surf_geom<<<(unsigned)((m->n_surf + th - 1) / th), th, 0, s>>>(m->n_surf, m->d_col, d_surf_p, d_surf_col,
                                                                   m->d_surf);
  k_tet_ball<<<(unsigned)((m->n_tet + th - 1) / th), th, 0, s>>>(m->n_tet, d_tet_vx, m->d_tet);
  STBEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

// ---------------------------------------------------------------------------
// Outer points (Fig. int_tri_mid): canonical corner order (ascending spatial
// id) and x = (A + xi1 (B - A)) + xi2 (C - A) without fused operations.
// ---------------------------------------------------------------------------
__global__ void k_outer_points(int64_t n_surf, int mq, const ColGeom* cols, const SurfDev* surf, double* pts,
                               float* ptsf, double* trange) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n_surf) return;
  const SurfDev S = surf[s];
  const ColGeom& G = cols[S.col];
  double A[4] = {S.f.p[0], G.X[0][0], G.X[0][1], G.X[0][2]};
  double B[4] = {S.f.p[1], G.X[1][0], G.X[1][1], G.X[1][2]};
  double C[4] = {S.f.p[2], G.X[2][0], G.X[2][1], G.X[2][2]};
  int nq = mq * mq;
  double* out = pts + (int64_t)s * nq * 4;
  double tlo = 1e300, thi = -1e300;
  int n = 0;
  for (int pass = 0; pass < 2; ++pass) {
    double off = pass == 0 ? 1.0 / 3.0 : 2.0 / 3.0;
    for (int i = 0; i < mq; ++i)
      for (int j = 0; i + j <= mq - 1 - pass; ++j) {
        double x1 = __ddiv_rn(__dadd_rn((double)i, off), (double)mq);
        double x2 = __ddiv_rn(__dadd_rn((double)j, off), (double)mq);
        for (int d = 0; d < 4; ++d) {
          double p = __dadd_rn(A[d], __dmul_rn(x1, __dsub_rn(B[d], A[d])));
          out[4 * n + d] = __dadd_rn(p, __dmul_rn(x2, __dsub_rn(C[d], A[d])));
          ptsf[(int64_t)s * nq * 4 + 4 * n + d] = (float)out[4 * n + d];
        }
        tlo = fmin(tlo, out[4 * n]);
        thi = fmax(thi, out[4 * n]);
        ++n;
      }
  }
  trange[2 * s] = tlo;
  trange[2 * s + 1] = thi;
}

bem_status op_outer_points(bem_operator* op, cudaStream_t s) {
  const bem_mesh* m = op->mesh;
  int th = 128;
  k_outer_points<<<(unsigned)((m->n_surf + th - 1) / th), th, 0, s>>>(m->n_surf, op->mq, m->d_col, m->d_surf,
                                                                      op->d_pts, op->d_ptsf, op->d_pts_trange);
  STBEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

// ---------------------------------------------------------------------------
// Sparsity predicate for one outer point and one panel (the contract):
//   C1  tau_min(j) < t_q
//   C2  max_b |x_q - y_b| - (t_q - tau_b) >= 0
//   C3  not (phi_Xi(x_q - c_j) - d_r(|x_q - c_j|) > 0)     (Theorem phi_xi_sphere)
// FP64 values with the contract's operation order decide; an FP32 estimate
// with a rigorous error margin settles the clear cases first.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double dist3x(const double* a, const double* b) {
  double dx = __dsub_rn(a[0], b[0]), dy = __dsub_rn(a[1], b[1]), dz = __dsub_rn(a[2], b[2]);
  return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
}
// (IEEE square roots here whatever the unit's FP32 flags: the filter's margin
// is set against the correctly rounded operations)
__device__ __forceinline__ float dist3f(const float* a, const float* b) {
  float dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
  return __fsqrt_rn(dx * dx + dy * dy + dz * dz);
}

struct TetSm {       // panel data kept in shared memory for a block
  double tmin, pmax;
  double vt[4];
  double ball[5];
  float vtf[4];      // FP32 copies for the filter of the sparsity predicate
  float ballf[5];
  int32_t lo, hi, dup, pad;
};

__device__ __noinline__ bool c2_exact(const double* x, const TetSm& T, const ColGeom& G) {
  double mx = -INFINITY;
  for (int b = 0; b < 4; ++b) {
    int k = b < 3 ? b : T.dup;
    double v = __dsub_rn(dist3x(x + 1, G.X[k]), __dsub_rn(x[0], T.vt[b]));
    if (v > mx) mx = v;
  }
  return mx >= 0.0;
}
__device__ __noinline__ bool c3_fail_exact(const double* x, const TetSm& T) {
  double al = dist3x(x + 1, T.ball + 1);
  double phi = __dsub_rn(al, __dsub_rn(x[0], T.ball[0]));
  double rj = T.ball[4];
  double s2 = __dsqrt_rn(2.0);
  double dr = (al < __ddiv_rn(rj, s2)) ? __dadd_rn(al, __dsqrt_rn(__dsub_rn(__dmul_rn(rj, rj), __dmul_rn(al, al))))
                                       : __dmul_rn(rj, s2);
  return __dsub_rn(phi, dr) > 0.0;
}

__device__ bool point_sees(const double* x, const float* xf, const TetSm& T, const ColGeom& G, const float (*Xf)[3],
                           float margin) {
  if (!(T.tmin < x[0])) return false;  // C1
  // C2
  {
    bool sure_true = false, sure_false = true;
    for (int b = 0; b < 4; ++b) {
      int k = b < 3 ? b : T.dup;
      float v = dist3f(xf + 1, Xf[k]) - (xf[0] - T.vtf[b]);
      if (v > margin) sure_true = true;
      if (!(v < -margin)) sure_false = false;
    }
    if (!sure_true) {
      if (sure_false) return false;
      if (!c2_exact(x, T, G)) return false;
    }
  }
  // C3
  {
    float al = dist3f(xf + 1, T.ballf + 1);
    float phi = al - (xf[0] - T.ballf[0]);
    float rj = T.ballf[4];
    float dr = (al < rj * 0.70710678f) ? al + __fsqrt_rn(fmaxf(rj * rj - al * al, 0.f)) : rj * 1.41421356f;
    float v = phi - dr;
    if (v > margin) return false;
    if (!(v < -margin)) {
      if (c3_fail_exact(x, T)) return false;
    }
  }
  return true;
}

// shared-memory image of column J
struct ColSm {
  ColGeom G;
  float Xf[3][3];
  int32_t tet0, ntet, surf0, nsurf;
  double rmax;  // max panel ball radius
};

// Trial window of column J for a face with outer-point time range [tlo, thi]:
// panels outside [jlo, jhi) are certainly outside the pattern.
__device__ inline void trial_window(const ColSm& C, const TetSm* T, double tlo, double thi, double Dmax,
                                    double Dmin_lo, double S, int& jlo, int& jhi) {
  double lim1 = tlo - Dmax * (1.0 + 1e-12) - 1e-12 * S;
  int a = 0, b = C.ntet;  // first j with pmax >= lim1
  while (a < b) { int m = (a + b) >> 1; if (T[m].pmax < lim1) a = m + 1; else b = m; }
  jlo = a;
  double lim2 = thi + fmin(0.0, C.rmax * 1.41421356237309515 * (1.0 + 1e-12) - Dmin_lo * (1.0 - 1e-12)) + 1e-12 * S;
  a = jlo; b = C.ntet;    // first j with tmin >= lim2
  while (a < b) { int m = (a + b) >> 1; if (T[m].tmin < lim2) a = m + 1; else b = m; }
  jhi = a;
}

__device__ inline void col_pair_bounds(const ColGeom& GI, const ColGeom& GJ, double& Dmax, double& Dmin_lo) {
  Dmax = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double dx = GI.X[a][0] - GJ.X[b][0], dy = GI.X[a][1] - GJ.X[b][1], dz = GI.X[a][2] - GJ.X[b][2];
      Dmax = fmax(Dmax, sqrt(dx * dx + dy * dy + dz * dz));
    }
  double dx = GI.ctr[0] - GJ.ctr[0], dy = GI.ctr[1] - GJ.ctr[1], dz = GI.ctr[2] - GJ.ctr[2];
  Dmin_lo = fmax(0.0, sqrt(dx * dx + dy * dy + dz * dz) - GI.rad - GJ.rad);
}

struct BlockCtx {
  int64_t n_col;
  int mq, nq, n_theta, prec;
  ArcRule rule;
  float margin;
  double S;
  const ColGeom* cols;
  const int32_t* col_tet_begin;
  const int32_t* col_surf_begin;
  const SurfDev* surf;
  const TetDev* tets;
  const double* pts;
  const float* ptsf;
  const double* trange;
  int32_t* bw;
  int64_t* bnnz;
  const int64_t* boff;
  const int64_t* rsoff;
  int32_t* rs;
  double* val;
  float* val32;
  double* uscratch;     // [gridDim][max_surf][max_tet]
  int max_surf, max_tet;
  unsigned long long* counter;
  int64_t end;                 // blocks [0, end) of the dense (I, J) order are processed
  unsigned long long* inner;   // pattern pass: inner integrals m_Q^2 x (test face, trial panel) (null: not counted)
  // matrix-free product: when mf_y is set the entries are not stored but
  // y[k][i] += A_ij x[k][j] is accumulated (x, y: [mf_nrhs][mf_ld], internal order)
  const double* mf_x;
  double* mf_y;
  int mf_nrhs;
  int64_t mf_ld;
};

// cooperative load of column J into shared memory
__device__ void load_column(const BlockCtx& B, int64_t J, ColSm& C, TetSm* T, FaceGeom* Fs) {
  if (threadIdx.x == 0) {
    C.G = B.cols[J];
    for (int k = 0; k < 3; ++k)
      for (int i = 0; i < 3; ++i) C.Xf[k][i] = (float)C.G.X[k][i];
    C.tet0 = B.col_tet_begin[J];
    C.ntet = B.col_tet_begin[J + 1] - C.tet0;
    C.surf0 = B.col_surf_begin[J];
    C.nsurf = B.col_surf_begin[J + 1] - C.surf0;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < C.ntet; j += blockDim.x) {
    const TetDev& D = B.tets[C.tet0 + j];
    TetSm t;
    t.tmin = D.tmin; t.pmax = D.pmax;
    for (int k = 0; k < 4; ++k) { t.vt[k] = D.vt[k]; t.vtf[k] = (float)D.vt[k]; }
    for (int k = 0; k < 5; ++k) { t.ball[k] = D.ball[k]; t.ballf[k] = (float)D.ball[k]; }
    t.lo = D.lo - C.surf0; t.hi = D.hi - C.surf0; t.dup = D.dup; t.pad = 0;
    T[j] = t;
  }
  for (int s = threadIdx.x; s < C.nsurf; s += blockDim.x) Fs[s] = B.surf[C.surf0 + s].f;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int j = 0; j < C.ntet; ++j) r = fmax(r, T[j].ball[4]);
    C.rmax = r;
  }
  __syncthreads();
}

// pattern bits of one face f' (global id) of column I against column J.
// Warp-cooperative; writes bits[0..words) and returns the trial window.
__device__ void face_bits(const BlockCtx& B, const ColSm& C, const TetSm* T, int64_t fglob, double Dmax,
                          double Dmin_lo, uint32_t* bits, int words, int& jlo, int& jhi) {
  int lane = threadIdx.x & 31;
  double tlo = B.trange[2 * fglob], thi = B.trange[2 * fglob + 1];
  trial_window(C, T, tlo, thi, Dmax, Dmin_lo, B.S, jlo, jhi);
  for (int w = lane; w < words; w += 32) bits[w] = 0u;
  __syncwarp();
  const double* P = B.pts + fglob * B.nq * 4;
  const float* Pf = B.ptsf + fglob * B.nq * 4;   // FP32 copies: no conversions in the filter
  for (int j0 = jlo; j0 < jhi; j0 += 32) {
    int j = j0 + lane;
    bool hit = false;
    if (j < jhi) {
      for (int q = 0; q < B.nq && !hit; ++q) {
        const float4 x4 = reinterpret_cast<const float4*>(Pf)[q];
        const float xf[4] = {x4.x, x4.y, x4.z, x4.w};
        hit = point_sees(P + 4 * q, xf, T[j], C.G, C.Xf, B.margin);
      }
    }
    unsigned m = __ballot_sync(0xffffffffu, hit);
    if (lane == 0 && m) {
      // j0 may not be word aligned: scatter bit by bit
      for (int l = 0; l < 32; ++l)
        if (m & (1u << l)) bits[(j0 + l) >> 5] |= 1u << ((j0 + l) & 31);
    }
    __syncwarp();
  }
}

__device__ inline int64_t pop_block(unsigned long long* counter) {
  __shared__ unsigned long long s_b;
  if (threadIdx.x == 0) s_b = atomicAdd(counter, 1ull);
  __syncthreads();
  int64_t b = (int64_t)s_b;
  __syncthreads();
  return b;
}

// Pass 1: band width and pattern count of column block b.
__device__ __forceinline__ void pattern_block(const BlockCtx& B, int64_t b, unsigned char* smem, ColSm& C, int* s_w,
                                              unsigned long long* s_n) {
  TetSm* T = reinterpret_cast<TetSm*>(smem);
  FaceGeom* Fs = reinterpret_cast<FaceGeom*>(T + B.max_tet);
  uint32_t* bits = reinterpret_cast<uint32_t*>(Fs + B.max_surf);
  const int words = (B.max_tet + 31) / 32;
  {
    int64_t I = b / B.n_col, J = b % B.n_col;
    load_column(B, J, C, T, Fs);
    const ColGeom GI = B.cols[I];
    double Dmax, Dmin_lo;
    col_pair_bounds(GI, C.G, Dmax, Dmin_lo);
    int s0 = B.col_surf_begin[I], ns = B.col_surf_begin[I + 1] - s0;
    int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int f = warp; f < ns; f += nw) {
      int jlo, jhi;
      face_bits(B, C, T, s0 + f, Dmax, Dmin_lo, bits + f * words, words, jlo, jhi);
    }
    __syncthreads();
    int t0 = B.col_tet_begin[I], nt = B.col_tet_begin[I + 1] - t0;
    int wmax = 0;
    unsigned long long cnt = 0;
    for (int r = threadIdx.x; r < nt; r += blockDim.x) {
      const TetDev& D = B.tets[t0 + r];
      int lo = D.lo - s0, hi = D.hi - s0;
      int first = -1, last = -1;
      for (int w = 0; w < words; ++w) {
        uint32_t m = bits[lo * words + w] | bits[hi * words + w];
        cnt += __popc(m);
        if (m) {
          if (first < 0) first = 32 * w + __ffs(m) - 1;
          last = 32 * w + 31 - __clz(m);
        }
      }
      if (first >= 0) wmax = max(wmax, last - first + 1);
    }
    for (int o = 16; o > 0; o >>= 1) {
      wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
      cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) { s_w[threadIdx.x >> 5] = wmax; s_n[threadIdx.x >> 5] = cnt; }
    __syncthreads();
    if (threadIdx.x == 0) {
      int w = 0;
      unsigned long long n = 0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { w = max(w, s_w[i]); n += s_n[i]; }
      B.bw[b] = w;
      B.bnnz[b] = (int64_t)n;
    }
    if (B.inner) {
      // inner integrals of the block: every outer point of a test face against
      // every trial panel the face's pattern bits admit
      unsigned long long m = 0;
      for (int f = threadIdx.x; f < ns; f += blockDim.x)
        for (int w = 0; w < words; ++w) m += __popc(bits[f * words + w]);
      for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
      if ((threadIdx.x & 31) == 0 && m) atomicAdd(B.inner, m * (unsigned long long)B.nq);
    }
    __syncthreads();
  }
}

// segment of global work item g: prefix[seg] <= g < prefix[seg + 1]
__device__ inline int find_seg(const int64_t* prefix, int S, int64_t g) {
  int lo = 0, hi = S;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (prefix[mid] <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(128) k_pattern_blocks(BlockCtx B) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ ColSm C;
  __shared__ int s_w[4];
  __shared__ unsigned long long s_n[4];
  const int64_t nblk = B.n_col * B.n_col;
  for (;;) {
    int64_t b = pop_block(B.counter);
    if (b >= nblk) break;
    pattern_block(B, b, smem, C, s_w, s_n);
  }
}

// The same over the blocks of a batch of operators (one work queue; the
// contexts share the largest column sizes so the shared layout is uniform).
__global__ void __launch_bounds__(128) k_pattern_batch(const BlockCtx* __restrict__ Bs,
                                                       const int64_t* __restrict__ prefix, int S,
                                                       unsigned long long* counter) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ ColSm C;
  __shared__ int s_w[4];
  __shared__ unsigned long long s_n[4];
  __shared__ BlockCtx sB;
  __shared__ int s_seg;
  int cur = -1;
  const int64_t total = prefix[S];
  for (;;) {
    int64_t g = pop_block(counter);
    if (g >= total) break;
    if (threadIdx.x == 0) s_seg = find_seg(prefix, S, g);
    __syncthreads();
    const int seg = s_seg;
    if (seg != cur) {
      if (threadIdx.x == 0) sB = Bs[seg];
      cur = seg;
    }
    __syncthreads();
    pattern_block(sB, g - prefix[seg], smem, C, s_w, s_n);
  }
}

// shared bytes per warp for the deferred arcs of the mixed kernel
constexpr size_t ARC_WARP_BYTES = 96 * sizeof(ArcRec<float>) + 96 * sizeof(float) + 96;
static_assert(ARC_WARP_BYTES % 16 == 0, "arc region keeps 16-byte alignment");

// Pass 2: quadrature and assembly of a non-empty block.
template <bool FP32>
__device__ __forceinline__ void quad_block(const BlockCtx& B, int64_t b, unsigned char* smem, ColSm& C,
                                           ColR<typename std::conditional<FP32, float, double>::type>& CR) {
  typedef typename std::conditional<FP32, float, double>::type R;
  TetSm* T = reinterpret_cast<TetSm*>(smem);
  FaceGeom* Fs = reinterpret_cast<FaceGeom*>(T + B.max_tet);
  uint32_t* bits = reinterpret_cast<uint32_t*>(Fs + B.max_surf);
  const int words = (B.max_tet + 31) / 32;
  PointCol* pc = reinterpret_cast<PointCol*>(bits + ((B.max_surf * words + 3) & ~3));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  PointCol* mypc = pc + warp * B.nq;
  R* Wsc0 = reinterpret_cast<R*>(pc + nw * B.nq);
  R* Wsc = Wsc0 + (size_t)warp * B.nq * B.max_surf;
  uint16_t* cut0 = reinterpret_cast<uint16_t*>(Wsc0 + (size_t)nw * B.nq * B.max_surf);
  uint16_t* mycut = cut0 + (size_t)warp * B.nq * B.max_surf;
  FaceF* Ff = reinterpret_cast<FaceF*>(cut0 + ((size_t)nw * B.nq * B.max_surf + 7) / 8 * 8);
  // mixed: per warp 96 deferred arcs (3 per lane), their values and the compacted order
  unsigned char* arc0 = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(Ff + B.max_surf) + 15) & ~static_cast<uintptr_t>(15));
  ArcRec<float>* myarc = reinterpret_cast<ArcRec<float>*>(arc0 + (size_t)warp * ARC_WARP_BYTES);
  float* myval = reinterpret_cast<float*>(myarc + 96);
  uint8_t* myidx = reinterpret_cast<uint8_t*>(myval + 96);
  R* U = reinterpret_cast<R*>(B.uscratch) + (size_t)blockIdx.x * B.max_surf * B.max_tet;
  {
    int W = B.bw[b];
    if (W == 0) return;
    int64_t I = b / B.n_col, J = b % B.n_col;
    load_column(B, J, C, T, Fs);
    if (threadIdx.x == 0) make_colr<R>(C.G, CR);
    if (FP32)
      for (int s = threadIdx.x; s < C.nsurf; s += blockDim.x) make_facef(Fs[s], Ff[s]);
    __syncthreads();
    const ColGeom GI = B.cols[I];
    double Dmax, Dmin_lo;
    col_pair_bounds(GI, C.G, Dmax, Dmin_lo);
    const int s0 = B.col_surf_begin[I], ns = B.col_surf_begin[I + 1] - s0;
    const int ntJ = C.ntet;
    const float fdiam = (float)C.G.diam;
    // The warps take the phases of their surfaces in lockstep (a CTA barrier
    // between face bits, point geometry, classification, the cut pass and the
    // U rows): all warps of the CTA then run the same code region, and the
    // instruction fetches they share hit (level-3 sphere, 16 slabs: 2,373 ->
    // 1,766 ms; benchmark mesh 5.83 -> 4.11 s).
    for (int f0 = 0; f0 < ns; f0 += nw) {
      const int f = f0 + warp;
      int jlo = 0, jhi = 0;
      const int64_t fg = s0 + f;
      R* Urow = U + (size_t)f * B.max_tet;
      if (f < ns) {
        face_bits(B, C, T, fg, Dmax, Dmin_lo, bits + f * words, words, jlo, jhi);
        for (int j = lane; j < ntJ; j += 32) Urow[j] = R(0);
      }
      const bool skip = f >= ns || jhi <= jlo;
      int slo = 1 << 30, shi = -1, nsw = 0, ncut = 0;
      const double* P = B.pts + fg * B.nq * 4;
      __syncthreads();
      if (!skip) {
      // surface window of the trial panels
      for (int j = jlo + lane; j < jhi; j += 32) {
        slo = min(slo, min(T[j].lo, T[j].hi));
        shi = max(shi, max(T[j].lo, T[j].hi));
      }
      for (int o = 16; o > 0; o >>= 1) {
        slo = min(slo, __shfl_xor_sync(0xffffffffu, slo, o));
        shi = max(shi, __shfl_xor_sync(0xffffffffu, shi, o));
      }
      nsw = shi - slo + 1;
      // per-point geometry against column J
      if constexpr (FP32) {
        for (int q = lane; q < B.nq; q += 32) point_col(P + 4 * q, C.G, mypc[q], true, true, &CR);
      } else {
        for (int q = lane; q < B.nq; q += 32) point_col(P + 4 * q, C.G, mypc[q], false);
      }
      if constexpr (FP32) {
        // the whole-edge integrals of the points' fully lit triangle, lane per (point, edge)
        __syncwarp();
        for (int e = lane; e < 3 * B.nq; e += 32) {
          const int q = e / 3, k = e - 3 * q;
          mypc[q].F.Efull[k] = edge_full_mixed(mypc[q], CR, k);
        }
        __syncwarp();
        for (int q = lane; q < B.nq; q += 32) point_col_finish(mypc[q]);
      }
      __syncwarp();
      }
      __syncthreads();
      if (!skip) {
      // pass 1: classify every (point, face) pair from the cone-function values
      // at the corners; fully lit and dark pairs are final, cut pairs are listed
      const int nit = B.nq * nsw;
      for (int base = 0; base < nit; base += 32) {
        int it = base + lane;
        bool cut = false;
        if (it < nit) {
          int q = it / nsw, s = it - q * nsw;
          int cls;
          if (FP32) {
            float Fv[3], cc = 0.f;
            cls = face_class_mixed(mypc[q], Ff[slo + s], Fv, cc, fdiam);
          } else {
            double Fv[3], cc = 0.0;
            cls = face_class(C.G, mypc[q], Fs[slo + s], Fv, cc);
          }
          if (cls == FACE_CUT) cut = true;
          else Wsc[q * B.max_surf + s] = cls == FACE_LIT ? (FP32 ? (R)mypc[q].Wst_f : (R)mypc[q].Wst) : R(0);
        }
        unsigned mk = __ballot_sync(0xffffffffu, cut);
        if (cut) mycut[ncut + __popc(mk & ((1u << lane) - 1u))] = (uint16_t)it;
        ncut += __popc(mk);
      }
      __syncwarp();
      }
      __syncthreads();
      if (!skip) {
      // pass 2: the cut pairs, converged across the warp
      if constexpr (FP32) {
        // mixed: the geometry and edge pieces lane per cut pair; the conic
        // arcs they need (at most 3 per pair, the larger part of the work)
        // are collected and integrated lane per arc over the compacted list,
        // then each pair adds its arcs in order (the same sum as in face_cut)
        for (int base = 0; base < ncut; base += 32) {
          const int k = base + lane;
          int na = 0, q = 0, s = 0;
          float et = 0.f;
          bool need64 = false;
          if (k < ncut) {
            const int it = mycut[k];
            q = it / nsw;
            s = it - q * nsw;
            float Fv[3], cc = 0.f;
            face_class_mixed(mypc[q], Ff[slo + s], Fv, cc, fdiam);
            need64 = near_singular_mixed(cc, mypc[q].F.d, fdiam);
            if (!need64) {
              FaceCutIn<float> in;
              cut_in_mixed(mypc[q], Ff[slo + s], Fv, cc, Fs[slo + s], in);
              et = (float)face_cut<float>(CR, mypc[q], in, B.rule, myarc + 3 * lane, &na);
            }
          }
          int incl = na;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
          }
          const int off = incl - na, total = __shfl_sync(0xffffffffu, incl, 31);
          for (int i = 0; i < na; ++i) myidx[off + i] = (uint8_t)(3 * lane + i);
          __syncwarp();
          for (int a = lane; a < total; a += 32) {
            const int slot = myidx[a];
            myval[slot] = arc_value<float>(myarc[slot], B.rule);
          }
          __syncwarp();
          if (k < ncut) {
            float v = et;
            for (int i = 0; i < na; ++i) v += myval[3 * lane + i];
            if (need64 || !isfinite(v))   // near-singular or degenerate FP32 geometry: this face in FP64
              v = (float)face_W_fp64(P + 4 * q, C.G, Fs[slo + s], B.n_theta);
            Wsc[q * B.max_surf + s] = v;
          }
          __syncwarp();
        }
      } else
      for (int k = lane; k < ncut; k += 32) {
        int it = mycut[k];
        int q = it / nsw, s = it - q * nsw;
        FaceCutIn<R> in;
        if constexpr (FP32) {
          float Fv[3], cc = 0.f;
          face_class_mixed(mypc[q], Ff[slo + s], Fv, cc, fdiam);
          cut_in_mixed(mypc[q], Ff[slo + s], Fv, cc, Fs[slo + s], in);
        } else {
          double Fv[3], cc = 0.0;
          face_class(C.G, mypc[q], Fs[slo + s], Fv, cc);
          cut_in_fp64(mypc[q], Fs[slo + s], Fv, cc, in);
        }
        Wsc[q * B.max_surf + s] = (R)face_cut<R>(CR, mypc[q], in, B.rule);
      }
      __syncwarp();
      }
      __syncthreads();
      if (!skip) {
      const uint32_t* fb = bits + f * words;
      for (int j = jlo + lane; j < jhi; j += 32) {
        if (!((fb[j >> 5] >> (j & 31)) & 1u)) continue;
        int lo = T[j].lo - slo, hi = T[j].hi - slo;
        R u = R(0);
        for (int q = 0; q < B.nq; ++q) u += Wsc[q * B.max_surf + lo] - Wsc[q * B.max_surf + hi];
        Urow[j] = u;
      }
      __syncwarp();
    }
    }
    __syncthreads();
    // entries of the block rows
    const int t0 = B.col_tet_begin[I], nt = B.col_tet_begin[I + 1] - t0;
    const R scale = (R)(GI.area / (4.0 * STBEM_PI * B.nq));
    const int64_t voff = B.boff[b], roff = B.rsoff[b];
    for (int r = threadIdx.x; r < nt; r += blockDim.x) {
      const TetDev& D = B.tets[t0 + r];
      int lo = D.lo - s0, hi = D.hi - s0;
      int first = -1;
      for (int w = 0; w < words && first < 0; ++w) {
        uint32_t m = bits[lo * words + w] | bits[hi * words + w];
        if (m) first = 32 * w + __ffs(m) - 1;
      }
      if (first < 0) first = 0;
      const R* Ulo = U + (size_t)lo * B.max_tet;
      const R* Uhi = U + (size_t)hi * B.max_tet;
      if (B.mf_y) {
        // fused product: the row's band times x, one atomic add per right-hand side
        for (int k = 0; k < B.mf_nrhs; ++k) {
          const double* xk = B.mf_x + (int64_t)k * B.mf_ld + C.tet0;
          double sacc = 0.0;
          for (int w = 0; w < W; ++w) {
            const int j = first + w;
            if (j < ntJ) sacc += (double)(scale * (Ulo[j] - Uhi[j])) * xk[j];
          }
          atomicAdd(B.mf_y + (int64_t)k * B.mf_ld + t0 + r, sacc);
        }
        continue;
      }
      B.rs[roff + r] = C.tet0 + first;
      for (int w = 0; w < W; ++w) {
        int j = first + w;
        R v = R(0);
        if (j < ntJ) v = scale * (Ulo[j] - Uhi[j]);
        if (B.val) B.val[voff + (int64_t)w * nt + r] = (double)v;
        if (B.val32) B.val32[voff + (int64_t)w * nt + r] = (float)v;
      }
    }
    __syncthreads();
  }
}

// STBEM_QUAD_MIN_CTAS (stbem_internal.h): CTAs of 128 threads resident per
// SM that the default register budget is cut for (quadrature of the level-3,
// 32-slab sphere in mixed precision with an earlier build: 4 / 5 / 6 CTAs
// took 6.83 / 6.91 / 7.56 s)
// warps per quadrature CTA
#ifndef STBEM_QUAD_WARPS
#define STBEM_QUAD_WARPS 4
#endif
constexpr int kQuadThreads = 32 * STBEM_QUAD_WARPS;

// MINB: CTAs per SM the register budget is cut for (STBEM_QUAD_MIN_CTAS: 128
// registers; 2: up to 255, no spills, for meshes whose shared memory per CTA
// lets no more than 2 CTAs share an SM anyway)
template <bool FP32, int MINB>
__global__ void __launch_bounds__(kQuadThreads, MINB) k_quad_blocks(BlockCtx B) {
  typedef typename std::conditional<FP32, float, double>::type R;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ ColSm C;
  __shared__ ColR<R> CR;
  const int64_t nblk = B.end;
  for (;;) {
    int64_t b = pop_block(B.counter);
    if (b >= nblk) break;
    quad_block<FP32>(B, b, smem, C, CR);
  }
}

template <bool FP32>
__global__ void __launch_bounds__(kQuadThreads, STBEM_QUAD_MIN_CTAS) k_quad_batch(const BlockCtx* __restrict__ Bs,
                                                       const int64_t* __restrict__ prefix, int S,
                                                       unsigned long long* counter, int64_t end) {
  typedef typename std::conditional<FP32, float, double>::type R;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ ColSm C;
  __shared__ ColR<R> CR;
  __shared__ BlockCtx sB;
  __shared__ int s_seg;
  int cur = -1;
  const int64_t total = min(prefix[S], end);
  for (;;) {
    int64_t g = pop_block(counter);
    if (g >= total) break;
    if (threadIdx.x == 0) s_seg = find_seg(prefix, S, g);
    __syncthreads();
    const int seg = s_seg;
    if (seg != cur) {
      if (threadIdx.x == 0) sB = Bs[seg];
      cur = seg;
    }
    __syncthreads();
    quad_block<FP32>(sB, g - prefix[seg], smem, C, CR);
  }
}

static size_t block_smem(const bem_operator* op, bool quad) {
  const bem_mesh* m = op->mesh;
  int words = (m->max_col_tets + 31) / 32;
  size_t s = sizeof(TetSm) * m->max_col_tets + sizeof(FaceGeom) * m->max_col_surf;
  s += sizeof(uint32_t) * ((m->max_col_surf * words + 3) & ~3);
  if (quad) {
    s += sizeof(PointCol) * STBEM_QUAD_WARPS * op->nq;
    s += (op->opts.precision == BEM_PREC_MIXED ? sizeof(float) : sizeof(double)) * STBEM_QUAD_WARPS * op->nq *
         m->max_col_surf;
    s += sizeof(uint16_t) * (((size_t)STBEM_QUAD_WARPS * op->nq * m->max_col_surf + 7) / 8 * 8);
    s += sizeof(FaceF) * m->max_col_surf;
    if (op->opts.precision == BEM_PREC_MIXED) s += 16 + STBEM_QUAD_WARPS * ARC_WARP_BYTES;
  }
  return s;
}

// The dynamic shared-memory limit of a kernel is state of the device shared by
// every host thread: operators of different sizes launching the same kernel
// concurrently (server slots) must never lower it under another's launch, so
// it only grows, under a lock.
bem_status ensure_smem_attr(const void* kern, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> set_to;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = set_to[std::make_pair(dev, kern)];
  if (bytes <= cur) return BEM_OK;
  STBEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  cur = bytes;
  return BEM_OK;
}

static int persistent_grid(const void* kern, size_t smem, int threads) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem);
  if (per < 1) per = 1;
  return sms * per;
}

static BlockCtx make_ctx(bem_operator* op) {
  const bem_mesh* m = op->mesh;
  BlockCtx B;
  B.n_col = m->n_col;
  B.mq = op->mq; B.nq = op->nq; B.n_theta = op->n_theta; B.prec = op->opts.precision;
  B.rule = make_rule(op->opts.precision, op->n_theta);
  B.S = m->coord_scale;
  B.margin = (float)(1.6e-5 * m->coord_scale);  // > 4x the FP32 error bound of C2 and C3
  B.cols = m->d_col; B.col_tet_begin = m->d_col_tet_begin; B.col_surf_begin = m->d_col_surf_begin;
  B.surf = m->d_surf; B.tets = m->d_tet; B.pts = op->d_pts; B.ptsf = op->d_ptsf; B.trange = op->d_pts_trange;
  B.bw = op->d_bw; B.bnnz = op->d_bnnz; B.boff = op->d_boff; B.rsoff = op->d_rsoff; B.rs = op->d_rs;
  B.val = op->d_val; B.val32 = op->d_val32; B.uscratch = op->d_tmp;
  B.max_surf = m->max_col_surf; B.max_tet = m->max_col_tets;
  B.counter = nullptr;
  B.end = m->n_col * m->n_col;
  B.inner = nullptr;
  B.mf_x = nullptr; B.mf_y = nullptr; B.mf_nrhs = 0; B.mf_ld = m->n_tet;
  return B;
}

static bem_status get_counter(const bem_operator* op, unsigned long long** out, cudaStream_t s) {
  STBEM_CUDA(cudaMemsetAsync(op->d_counter, 0, sizeof(unsigned long long), s));
  *out = op->d_counter;
  return BEM_OK;
}

bem_status op_pattern(bem_operator* op, cudaStream_t s) {
  BlockCtx B = make_ctx(op);
  bem_status st = get_counter(op, &B.counter, s);
  if (st != BEM_OK) return st;
  STBEM_CUDA(cudaMemsetAsync(op->d_counter + 1, 0, sizeof(unsigned long long), s));
  B.inner = op->d_counter + 1;
  size_t smem = block_smem(op, false);
  st = ensure_smem_attr((const void*)k_pattern_blocks, smem);
  if (st != BEM_OK) return st;
  int grid = persistent_grid((const void*)k_pattern_blocks, smem, 128);
  k_pattern_blocks<<<grid, 128, smem, s>>>(B);
  STBEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

// quadrature kernel of a precision and register budget (variant 0: the
// STBEM_QUAD_MIN_CTAS budget; variant 1: the 2-CTA budget, mixed precision only)
static const void* quad_kernel(const bem_operator* op, int variant) {
  if (op->opts.precision != BEM_PREC_MIXED) return (const void*)k_quad_blocks<false, STBEM_QUAD_MIN_CTAS>;
  return variant ? (const void*)k_quad_blocks<true, 2> : (const void*)k_quad_blocks<true, STBEM_QUAD_MIN_CTAS>;
}

int quad_variants(const bem_operator* op) { return op->opts.precision == BEM_PREC_MIXED ? 2 : 1; }

int quad_max_per_sm(const bem_operator* op, int variant) {
  const size_t smem = block_smem(op, true);
  const void* kern = quad_kernel(op, variant);
  ensure_smem_attr(kern, smem);
  return std::max(1, persistent_grid(kern, smem, kQuadThreads) / std::max(1, (int)op->ctx->sm_count));
}

bem_status quad_launch(const bem_operator* op, int per_sm, int64_t end, const double* mf_x, double* mf_y, int nrhs,
                       cudaStream_t s, int variant) {
  BlockCtx B = make_ctx(const_cast<bem_operator*>(op));
  bem_status st = get_counter(op, &B.counter, s);
  if (st != BEM_OK) return st;
  B.end = std::min<int64_t>(end, B.end);
  B.mf_x = mf_x;
  B.mf_y = mf_y;
  B.mf_nrhs = nrhs;
  B.mf_ld = op->mesh->n_tet;
  if (variant >= quad_variants(op)) variant = 0;
  const size_t smem = block_smem(op, true);
  const int max_per = quad_max_per_sm(op, variant);
  const int grid = (int)op->ctx->sm_count * std::max(1, std::min(per_sm, max_per));
  if ((int64_t)grid * op->mesh->max_col_surf * op->mesh->max_col_tets > op->tmp_len) {
    set_error("quadrature scratch too small");
    return BEM_ERR_INTERNAL;
  }
  if (op->opts.precision != BEM_PREC_MIXED) k_quad_blocks<false, STBEM_QUAD_MIN_CTAS><<<grid, kQuadThreads, smem, s>>>(B);
  else if (variant) k_quad_blocks<true, 2><<<grid, kQuadThreads, smem, s>>>(B);
  else k_quad_blocks<true, STBEM_QUAD_MIN_CTAS><<<grid, kQuadThreads, smem, s>>>(B);
  STBEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

bem_status op_quadrature(bem_operator* op, cudaStream_t s) {
  bem_status st = choose_quad_shape(op, s);
  if (st != BEM_OK) return st;
  return quad_launch(op, op->quad_per_sm, op->mesh->n_col * op->mesh->n_col, nullptr, nullptr, 0, s,
                     op->quad_variant);
}

// Matrix-free product y = A x (internal order, [nrhs][n_tet]): the quadrature
// pass with the entries summed against x instead of stored.
bem_status op_matvec_free(const bem_operator* op, const double* x, double* y, int nrhs, cudaStream_t s) {
  STBEM_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * op->mesh->n_tet * nrhs, s));
  int per_sm = op->quad_per_sm, variant = op->quad_variant;
  if (per_sm <= 0) default_quad_shape(op, &per_sm, &variant);
  return quad_launch(op, per_sm, op->mesh->n_col * op->mesh->n_col, x, y, nrhs, s, variant);
}

// ---------------------------------------------------------------------------
// Batched passes: one persistent launch over the blocks of several operators.
// All contexts take the largest column sizes of the batch, so the shared
// memory layout is the same for every block, and the quadrature scratch
// (one slab per CTA) is shared.
// ---------------------------------------------------------------------------
bem_status op_outer_points_all(const std::vector<bem_operator*>& ops, cudaStream_t s) {
  for (bem_operator* op : ops) {
    bem_status st = op_outer_points(op, s);
    if (st != BEM_OK) return st;
  }
  return BEM_OK;
}

static void batch_dims(const std::vector<bem_operator*>& ops, int& max_tet, int& max_surf) {
  max_tet = 1;
  max_surf = 1;
  for (const bem_operator* op : ops) {
    max_tet = std::max(max_tet, op->mesh->max_col_tets);
    max_surf = std::max(max_surf, op->mesh->max_col_surf);
  }
}

static size_t batch_smem(int max_tet, int max_surf, int nq, bool quad, bool fp32 = false) {
  int words = (max_tet + 31) / 32;
  size_t s = sizeof(TetSm) * max_tet + sizeof(FaceGeom) * max_surf;
  s += sizeof(uint32_t) * ((max_surf * words + 3) & ~3);
  if (quad) {
    s += sizeof(PointCol) * STBEM_QUAD_WARPS * nq;
    s += (fp32 ? sizeof(float) : sizeof(double)) * STBEM_QUAD_WARPS * nq * max_surf;
    s += sizeof(uint16_t) * (((size_t)STBEM_QUAD_WARPS * nq * max_surf + 7) / 8 * 8);
    s += sizeof(FaceF) * max_surf;
    if (fp32) s += 16 + STBEM_QUAD_WARPS * ARC_WARP_BYTES;
  }
  return s;
}

static bem_status upload_batch(const std::vector<bem_operator*>& ops, BatchDev& dev, int max_tet, int max_surf,
                               cudaStream_t s) {
  const int S = (int)ops.size();
  std::vector<BlockCtx> ctx(S);
  std::vector<int64_t> prefix(S + 1, 0);
  for (int i = 0; i < S; ++i) {
    ctx[i] = make_ctx(ops[i]);
    ctx[i].max_tet = max_tet;
    ctx[i].max_surf = max_surf;
    ctx[i].uscratch = dev.d_uscratch;
    ctx[i].counter = dev.d_counter;
    prefix[i + 1] = prefix[i] + ops[i]->mesh->n_col * ops[i]->mesh->n_col;
  }
  STBEM_CUDA(cudaMemcpyAsync(dev.d_ctx, ctx.data(), sizeof(BlockCtx) * S, cudaMemcpyHostToDevice, s));
  STBEM_CUDA(cudaMemcpyAsync(dev.d_prefix, prefix.data(), sizeof(int64_t) * (S + 1), cudaMemcpyHostToDevice, s));
  STBEM_CUDA(cudaMemsetAsync(dev.d_counter, 0, sizeof(unsigned long long), s));
  STBEM_CUDA(cudaStreamSynchronize(s));   // the host arrays above go out of scope
  return BEM_OK;
}

bem_status op_pattern_batch(const std::vector<bem_operator*>& ops, BatchDev& dev, cudaStream_t s) {
  if (ops.empty()) return BEM_OK;
  int mt, ms;
  batch_dims(ops, mt, ms);
  bem_status st = upload_batch(ops, dev, mt, ms, s);
  if (st != BEM_OK) return st;
  const size_t smem = batch_smem(mt, ms, ops[0]->nq, false);
  st = ensure_smem_attr((const void*)k_pattern_batch, smem);
  if (st != BEM_OK) return st;
  const int grid = persistent_grid((const void*)k_pattern_batch, smem, 128);
  k_pattern_batch<<<grid, 128, smem, s>>>(static_cast<const BlockCtx*>(dev.d_ctx), dev.d_prefix, (int)ops.size(),
                                          dev.d_counter);
  STBEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

static int quad_batch_grid(const std::vector<bem_operator*>& ops, size_t& smem) {
  int mt, ms;
  batch_dims(ops, mt, ms);
  smem = batch_smem(mt, ms, ops[0]->nq, true, ops[0]->opts.precision == BEM_PREC_MIXED);
  if (ops[0]->opts.precision == BEM_PREC_MIXED) {
    ensure_smem_attr((const void*)k_quad_batch<true>, smem);
    return persistent_grid((const void*)k_quad_batch<true>, smem, kQuadThreads);
  }
  ensure_smem_attr((const void*)k_quad_batch<false>, smem);
  return persistent_grid((const void*)k_quad_batch<false>, smem, kQuadThreads);
}

int64_t quad_batch_scratch(const std::vector<bem_operator*>& ops) {
  if (ops.empty()) return 0;
  int mt, ms;
  batch_dims(ops, mt, ms);
  size_t smem = 0;
  return (int64_t)quad_batch_grid(ops, smem) * mt * ms;
}

bem_status op_quadrature_batch(const std::vector<bem_operator*>& ops, BatchDev& dev, cudaStream_t s) {
  if (ops.empty()) return BEM_OK;
  for (const bem_operator* op : ops)
    if (op->opts.precision != ops[0]->opts.precision || op->nq != ops[0]->nq || op->n_theta != ops[0]->n_theta) {
      set_error("a batch takes one precision, m_Q and n_theta");
      return BEM_ERR_INVALID_ARG;
    }
  if (dev.uscratch_len < quad_batch_scratch(ops)) {
    set_error("batch quadrature scratch too small");
    return BEM_ERR_INTERNAL;
  }
  int mt, ms;
  batch_dims(ops, mt, ms);
  bem_status st = upload_batch(ops, dev, mt, ms, s);
  if (st != BEM_OK) return st;
  size_t smem = 0;
  const int max_grid = quad_batch_grid(ops, smem);
  const int sms = (int)ops[0]->ctx->sm_count;
  const int occ = std::max(1, max_grid / std::max(1, sms));
  const BlockCtx* d = static_cast<const BlockCtx*>(dev.d_ctx);
  auto launch = [&](int per, int64_t end) -> bem_status {
    STBEM_CUDA(cudaMemsetAsync(dev.d_counter, 0, sizeof(unsigned long long), s));
    const int grid = sms * std::max(1, std::min(per, occ));
    if (ops[0]->opts.precision == BEM_PREC_MIXED)
      k_quad_batch<true><<<grid, kQuadThreads, smem, s>>>(d, dev.d_prefix, (int)ops.size(), dev.d_counter, end);
    else
      k_quad_batch<false><<<grid, kQuadThreads, smem, s>>>(d, dev.d_prefix, (int)ops.size(), dev.d_counter, end);
    STBEM_CUDA(cudaGetLastError());
    return BEM_OK;
  };
  int64_t total = 0;
  for (const bem_operator* op : ops) total += op->mesh->n_col * op->mesh->n_col;
  int per = occ, how = 0;
  if (ops[0]->ctx->tune_mode) {
    // the batch's own shape class; sample: 1/32 of the block queue
    const std::string key = batch_shape_class(ops[0]->ctx, ops[0]->opts.precision, ops[0]->nq, ops[0]->n_theta, mt,
                                              ms, (int64_t)ops.size(), total);
    std::vector<int> codes;
    for (int p = std::max(1, occ - 2); p <= occ; ++p) codes.push_back(p);
    st = tune_launch_shape(ops[0]->ctx, key, codes, std::max<int64_t>(total / 32, 1), launch, s, &per, &how, nullptr);
    if (st != BEM_OK) return st;
  }
  return launch(per, total);
}

size_t block_ctx_size() { return sizeof(BlockCtx); }

// ---------------------------------------------------------------------------
// Value scan: non-finite count and largest magnitude
// ---------------------------------------------------------------------------
template <typename V>
__global__ void k_value_scan(const V* v, int64_t n, unsigned long long* bad, unsigned long long* maxbits) {
  unsigned long long nb = 0;
  double mx = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double x = (double)v[i];
    if (!isfinite(x)) ++nb;
    else mx = fmax(mx, fabs(x));
  }
  for (int o = 16; o > 0; o >>= 1) {
    nb += __shfl_xor_sync(0xffffffffu, nb, o);
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (nb) atomicAdd(bad, nb);
    atomicMax(maxbits, (unsigned long long)__double_as_longlong(mx));  // non-negative doubles order as integers
  }
}

bem_status op_value_scan(const bem_operator* op, int64_t* nbad, double* maxabs, cudaStream_t s) {
  unsigned long long* d;
  STBEM_CUDA(cudaMalloc(&d, 2 * sizeof(unsigned long long)));
  STBEM_CUDA(cudaMemsetAsync(d, 0, 2 * sizeof(unsigned long long), s));
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (op->nstored > 0) {
    if (op->d_val) k_value_scan<double><<<sms * 8, 256, 0, s>>>(op->d_val, op->nstored, d, d + 1);
    else k_value_scan<float><<<sms * 8, 256, 0, s>>>(op->d_val32, op->nstored, d, d + 1);
  }
  unsigned long long h[2];
  cudaError_t e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return BEM_ERR_CUDA; }
  *nbad = (int64_t)h[0];
  long long bits = (long long)h[1];
  *maxabs = __longlong_as_double_host(bits);
  return BEM_OK;
}

// ---------------------------------------------------------------------------
// Entry lookup (internal indices) and pattern CSR export
// ---------------------------------------------------------------------------
__global__ void k_entries(int64_t n, const int32_t* ij, const float* val32, const TetDev* tets, int64_t n_col,
                          const int32_t* col_tet_begin, const int32_t* bw, const int64_t* boff, const int64_t* rsoff,
                          const int32_t* rs, const double* val, double* out) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  int i = ij[2 * k], j = ij[2 * k + 1];
  int I = tets[i].col, J = tets[j].col;
  int64_t b = (int64_t)I * n_col + J;
  int W = bw[b];
  double v = 0.0;
  if (W > 0) {
    int r = i - col_tet_begin[I];
    int nt = col_tet_begin[I + 1] - col_tet_begin[I];
    int start = rs[rsoff[b] + r];
    int w = j - start;
    if (w >= 0 && w < W) v = val ? val[boff[b] + (int64_t)w * nt + r] : (double)val32[boff[b] + (int64_t)w * nt + r];
  }
  out[k] = v;
}

bem_status op_entries(const bem_operator* op, int64_t n, const int32_t* d_ij, double* d_out, cudaStream_t s) {
  const bem_mesh* m = op->mesh;
  if (n == 0) return BEM_OK;
  k_entries<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, d_ij, op->d_val32, m->d_tet, m->n_col, m->d_col_tet_begin,
                                                       op->d_bw, op->d_boff, op->d_rsoff, op->d_rs, op->d_val, d_out);
  STBEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

// Pattern rows (internal numbering): count pass, then fill pass (columns are
// written in internal order; the caller permutes and sorts).
__global__ void __launch_bounds__(128) k_pattern_rows(BlockCtx B, int64_t* rowcount, const int64_t* rowptr,
                                                      int32_t* cols, int fill, int64_t I_only) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ ColSm C;
  TetSm* T = reinterpret_cast<TetSm*>(smem);
  FaceGeom* Fs = reinterpret_cast<FaceGeom*>(T + B.max_tet);
  uint32_t* bits = reinterpret_cast<uint32_t*>(Fs + B.max_surf);
  const int words = (B.max_tet + 31) / 32;
  const int64_t nblk = I_only >= 0 ? B.n_col : B.n_col * B.n_col;
  for (;;) {
    int64_t b = pop_block(B.counter);
    if (b >= nblk) break;
    if (I_only >= 0) b += I_only * B.n_col;
    if (B.bw[b] == 0) continue;
    int64_t I = b / B.n_col, J = b % B.n_col;
    load_column(B, J, C, T, Fs);
    const ColGeom GI = B.cols[I];
    double Dmax, Dmin_lo;
    col_pair_bounds(GI, C.G, Dmax, Dmin_lo);
    int s0 = B.col_surf_begin[I], ns = B.col_surf_begin[I + 1] - s0;
    int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int f = warp; f < ns; f += nw) {
      int jlo, jhi;
      face_bits(B, C, T, s0 + f, Dmax, Dmin_lo, bits + f * words, words, jlo, jhi);
    }
    __syncthreads();
    int t0 = B.col_tet_begin[I], nt = B.col_tet_begin[I + 1] - t0;
    for (int r = threadIdx.x; r < nt; r += blockDim.x) {
      const TetDev& D = B.tets[t0 + r];
      int lo = D.lo - s0, hi = D.hi - s0;
      int cnt = 0;
      for (int w = 0; w < words; ++w) cnt += __popc(bits[lo * words + w] | bits[hi * words + w]);
      if (!cnt) continue;
      unsigned long long pos = atomicAdd((unsigned long long*)&rowcount[t0 + r], (unsigned long long)cnt);
      if (fill) {
        for (int w = 0; w < words; ++w) {
          uint32_t m = bits[lo * words + w] | bits[hi * words + w];
          while (m) {
            int l = __ffs(m) - 1;
            m &= m - 1;
            cols[rowptr[t0 + r] + (int64_t)pos++] = C.tet0 + 32 * w + l;
          }
        }
      }
    }
    __syncthreads();
  }
}

bem_status op_pattern_csr(const bem_operator* op, int64_t* d_rowcount, int64_t* d_rowptr, int32_t* d_cols, bool fill,
                          cudaStream_t s, int64_t I_only) {
  BlockCtx B = make_ctx(const_cast<bem_operator*>(op));
  bem_status st = get_counter(op, &B.counter, s);
  if (st != BEM_OK) return st;
  size_t smem = block_smem(op, false);
  {
    bem_status sa = ensure_smem_attr((const void*)k_pattern_rows, smem);
    if (sa != BEM_OK) return sa;
  }
  int grid = persistent_grid((const void*)k_pattern_rows, smem, 128);
  k_pattern_rows<<<grid, 128, smem, s>>>(B, d_rowcount, d_rowptr, d_cols, fill ? 1 : 0, I_only);
  STBEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

// ---------------------------------------------------------------------------
// Right-hand side: b_i = int_K [g(P_lo(y), y) - g(P_hi(y), y)] dA
// (= -sum_F nu_{F,t} int_F g dS, eq. int_bform with A = Id). K is split into
// 4^k congruent sub-triangles, k chosen so that a sub-triangle spans at most
// half the data's length scale (pulse width, or 0.5 for the sin^2 data), and
// each gets a Duffy-collapsed 8 x 8 Gauss-Legendre rule.
// ---------------------------------------------------------------------------
__device__ inline double data_g(int kind, const double* prm, double t, const double* x) {
  if (kind == BEM_DATA_SIN2_UNIFORM) {
    if (!(t > 0.0 && t < 2.0)) return 0.0;
    double s = sin(0.5 * STBEM_PI * t);
    return s * s;
  }
  double a = (t - (x[0] * prm[0] + x[1] * prm[1] + x[2] * prm[2]) - prm[3]) / prm[4];
  return exp(-a * a);
}

__device__ inline double rhs_subtri(const ColGeom& G, const FaceGeom& Flo, const FaceGeom& Fhi, int kind,
                                    const double* prm, const double* B0, const double* B1, const double* B2) {
  const int n = 8;
  const double* X = gl_x() + n * (n - 1) / 2;
  const double* Wt = gl_w() + n * (n - 1) / 2;
  double acc = 0.0;
  for (int a = 0; a < n; ++a) {
    double u = 0.5 * (X[a] + 1.0), wu = 0.5 * Wt[a];
    for (int c = 0; c < n; ++c) {
      double v = 0.5 * (X[c] + 1.0), wv = 0.5 * Wt[c];
      double m0 = 1.0 - u, m1 = u * (1.0 - v), m2 = u * v;   // Duffy: Jacobian 2 |sub| u
      double l[3];
      for (int k = 0; k < 3; ++k) l[k] = m0 * B0[k] + m1 * B1[k] + m2 * B2[k];
      double y[3];
      for (int k = 0; k < 3; ++k) y[k] = l[0] * G.X[0][k] + l[1] * G.X[1][k] + l[2] * G.X[2][k];
      double tlo = l[0] * Flo.p[0] + l[1] * Flo.p[1] + l[2] * Flo.p[2];
      double thi = l[0] * Fhi.p[0] + l[1] * Fhi.p[1] + l[2] * Fhi.p[2];
      acc += wu * wv * u * (data_g(kind, prm, tlo, y) - data_g(kind, prm, thi, y));
    }
  }
  return acc;
}

__global__ void k_rhs(int64_t n_tet, const TetDev* tets, const SurfDev* surf, const ColGeom* cols, int kind, int nrhs,
                      const double* params, double* b) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n_tet) return;
  const TetDev D = tets[i];
  const ColGeom& G = cols[D.col];
  const FaceGeom Flo = surf[D.lo].f, Fhi = surf[D.hi].f;
  for (int r = 0; r < nrhs; ++r) {
    const double* prm = params ? params + 5 * r : nullptr;
    double scale = kind == BEM_DATA_PULSE ? 0.5 * prm[4] : 0.5;
    int lev = 0;
    while (lev < 4 && G.diam / (double)(1 << lev) > scale) ++lev;
    int m = 1 << lev;
    double acc = 0.0;
    for (int p = 0; p < m; ++p)
      for (int q = 0; p + q < m; ++q) {
        double a0[3] = {1.0 - (double)(p + q) / m, (double)p / m, (double)q / m};
        double a1[3] = {1.0 - (double)(p + q + 1) / m, (double)(p + 1) / m, (double)q / m};
        double a2[3] = {1.0 - (double)(p + q + 1) / m, (double)p / m, (double)(q + 1) / m};
        acc += rhs_subtri(G, Flo, Fhi, kind, prm, a0, a1, a2);
        if (p + q + 2 <= m) {
          double c0[3] = {1.0 - (double)(p + q + 2) / m, (double)(p + 1) / m, (double)(q + 1) / m};
          acc += rhs_subtri(G, Flo, Fhi, kind, prm, a1, c0, a2);
        }
      }
    // each sub-triangle has area |K| / m^2; Duffy Jacobian 2 |sub| u
    b[i + n_tet * (int64_t)r] = 2.0 * G.area / ((double)m * m) * acc;
  }
}

bem_status op_rhs(const bem_operator* op, int kind, int nrhs, const double* d_params, double* d_b, cudaStream_t s) {
  const bem_mesh* m = op->mesh;
  k_rhs<<<(unsigned)((m->n_tet + 127) / 128), 128, 0, s>>>(m->n_tet, m->d_tet, m->d_surf, m->d_col, kind, nrhs,
                                                           d_params, d_b);
  STBEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

// Points and weights of the right-hand side rule for arbitrary data: per
// surface (a face tau = P(y) over K), K split into 4^level congruent
// triangles in the order of k_rhs (row p, then q; upright, then inverted),
// each with a Duffy-collapsed ng x ng Gauss-Legendre rule. One thread per
// (surface, sub-triangle); pts may be null (weights only).
__global__ void k_rhs_points(int64_t n_surf, const SurfDev* surf, const ColGeom* cols, int level, int ng,
                             double* pts, double* wts) {
  const int m = 1 << level, nsub = m * m;
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= n_surf * nsub) return;
  const int64_t sidx = tid / nsub;
  const int k = (int)(tid - sidx * nsub);
  // sub-triangle k -> corners (barycentric)
  double a0[3], a1[3], a2[3];
  int cnt = 0;
  bool found = false;
  for (int p = 0; p < m && !found; ++p)
    for (int q = 0; p + q < m && !found; ++q) {
      double u0[3] = {1.0 - (double)(p + q) / m, (double)p / m, (double)q / m};
      double u1[3] = {1.0 - (double)(p + q + 1) / m, (double)(p + 1) / m, (double)q / m};
      double u2[3] = {1.0 - (double)(p + q + 1) / m, (double)p / m, (double)(q + 1) / m};
      if (cnt++ == k) {
        for (int c = 0; c < 3; ++c) { a0[c] = u0[c]; a1[c] = u1[c]; a2[c] = u2[c]; }
        found = true;
      } else if (p + q + 2 <= m) {
        if (cnt++ == k) {
          double v0[3] = {1.0 - (double)(p + q + 2) / m, (double)(p + 1) / m, (double)(q + 1) / m};
          for (int c = 0; c < 3; ++c) { a0[c] = u1[c]; a1[c] = v0[c]; a2[c] = u2[c]; }
          found = true;
        }
      }
    }
  const SurfDev S = surf[sidx];
  const ColGeom& G = cols[S.col];
  const double* X = gl_x() + ng * (ng - 1) / 2;
  const double* Wt = gl_w() + ng * (ng - 1) / 2;
  const double jac = 2.0 * G.area / (double)nsub;   // Duffy: 2 |sub| u
  int64_t o = (sidx * nsub + k) * (int64_t)ng * ng;
  for (int a = 0; a < ng; ++a) {
    const double u = 0.5 * (X[a] + 1.0), wu = 0.5 * Wt[a];
    for (int c = 0; c < ng; ++c, ++o) {
      const double v = 0.5 * (X[c] + 1.0), wv = 0.5 * Wt[c];
      const double m0 = 1.0 - u, m1 = u * (1.0 - v), m2 = u * v;
      double l[3];
      for (int e = 0; e < 3; ++e) l[e] = m0 * a0[e] + m1 * a1[e] + m2 * a2[e];
      wts[o] = jac * wu * wv * u;
      if (pts) {
        pts[4 * o] = l[0] * S.f.p[0] + l[1] * S.f.p[1] + l[2] * S.f.p[2];
        for (int e = 0; e < 3; ++e) pts[4 * o + 1 + e] = l[0] * G.X[0][e] + l[1] * G.X[1][e] + l[2] * G.X[2][e];
      }
    }
  }
}

// S[r][s] = sum_q w_q g[r][s * npps + q] in ascending q (one thread per (r, s))
__global__ void k_rhs_face_sums(int64_t n_surf, int64_t npps, int nrhs, const double* wts, const double* g,
                                double* S) {
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= n_surf * nrhs) return;
  const int64_t r = tid / n_surf, sidx = tid - r * n_surf;
  const double* gw = g + r * n_surf * npps + sidx * npps;
  const double* ww = wts + sidx * npps;
  double acc = 0.0;
  for (int64_t q = 0; q < npps; ++q) acc += ww[q] * gw[q];
  S[tid] = acc;
}

// b[r][i] = S[r][lo(i)] - S[r][hi(i)] (internal panel order)
__global__ void k_rhs_combine(int64_t n_tet, int64_t n_surf, int nrhs, const TetDev* tets, const double* S, double* b) {
  int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (tid >= n_tet * nrhs) return;
  const int64_t r = tid / n_tet, i = tid - r * n_tet;
  const TetDev& D = tets[i];
  b[tid] = S[r * n_surf + D.lo] - S[r * n_surf + D.hi];
}

bem_status op_rhs_points(const bem_operator* op, int level, int ng, double* d_pts, double* d_wts, cudaStream_t s) {
  const bem_mesh* m = op->mesh;
  const int64_t n = m->n_surf * ((int64_t)1 << (2 * level));
  if (n == 0) return BEM_OK;
  k_rhs_points<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(m->n_surf, m->d_surf, m->d_col, level, ng, d_pts, d_wts);
  STBEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

bem_status op_rhs_samples(const bem_operator* op, int level, int ng, const double* d_wts, const double* d_g, int nrhs,
                          double* d_S, double* d_b, cudaStream_t s) {
  const bem_mesh* m = op->mesh;
  const int64_t npps = ((int64_t)1 << (2 * level)) * ng * ng;
  const int64_t ns = m->n_surf * nrhs, nb = m->n_tet * nrhs;
  if (ns > 0)
    k_rhs_face_sums<<<(unsigned)((ns + 127) / 128), 128, 0, s>>>(m->n_surf, npps, nrhs, d_wts, d_g, d_S);
  if (nb > 0)
    k_rhs_combine<<<(unsigned)((nb + 127) / 128), 128, 0, s>>>(m->n_tet, m->n_surf, nrhs, m->d_tet, d_S, d_b);
  STBEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

// ---------------------------------------------------------------------------
// Kernel-level inner potentials for arbitrary (point, panel) pairs
// ---------------------------------------------------------------------------
template <bool FP32>
__global__ void k_inner(int64_t n, const double* x4, const double* tv, const int32_t* sv, int n_theta, double* out) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double* X = tv + 16 * k;
  const int32_t* s = sv + 4 * k;
  // corners: distinct spatial ids ascending; lower / upper times per corner
  int ids[3], nid = 0;
  for (int v = 0; v < 4; ++v) {
    bool dup = false;
    for (int q = 0; q < nid; ++q) dup |= ids[q] == s[v];
    if (!dup && nid < 3) ids[nid++] = s[v];
  }
  if (nid != 3) { out[k] = nan(""); return; }
  for (int a = 1; a < 3; ++a)
    for (int b = a; b > 0 && ids[b - 1] > ids[b]; --b) { int t = ids[b]; ids[b] = ids[b - 1]; ids[b - 1] = t; }
  double cx[3][3];
  FaceGeom Flo, Fhi;
  for (int c = 0; c < 3; ++c) {
    double lo = 1e300, hi = -1e300;
    for (int v = 0; v < 4; ++v)
      if (s[v] == ids[c]) {
        for (int i = 0; i < 3; ++i) cx[c][i] = X[4 * v + 1 + i];
        lo = fmin(lo, X[4 * v]);
        hi = fmax(hi, X[4 * v]);
      }
    Flo.p[c] = lo;
    Fhi.p[c] = hi;
  }
  ColGeom G;
  make_colgeom(cx[0], cx[1], cx[2], G);
  face_gradient(G, Flo);
  face_gradient(G, Fhi);
  PointCol P;
  point_col(x4 + 4 * k, G, P, FP32);
  const ArcRule rule = make_rule(FP32 ? BEM_PREC_MIXED : BEM_PREC_FP64, n_theta);
  double wl = face_W<FP32>(G, P, Flo, rule), wh = face_W<FP32>(G, P, Fhi, rule);
  if (FP32 && !isfinite(wl)) wl = face_W_fp64(x4 + 4 * k, G, Flo, n_theta);
  if (FP32 && !isfinite(wh)) wh = face_W_fp64(x4 + 4 * k, G, Fhi, n_theta);
  out[k] = (wl - wh) / (4.0 * STBEM_PI);
}

bem_status inner_potentials(int64_t n, const double* d_x4, const double* d_tets, const int32_t* d_sv, int prec,
                            int n_theta, double* d_out, cudaStream_t s) {
  if (n == 0) return BEM_OK;
  unsigned g = (unsigned)((n + 127) / 128);
  if (prec == BEM_PREC_MIXED) k_inner<true><<<g, 128, 0, s>>>(n, d_x4, d_tets, d_sv, n_theta, d_out);
  else k_inner<false><<<g, 128, 0, s>>>(n, d_x4, d_tets, d_sv, n_theta, d_out);
  STBEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

// ---------------------------------------------------------------------------
// Permutations between caller and internal panel order
// ---------------------------------------------------------------------------
__global__ void k_permute(const int32_t* perm, const double* in, double* out, int64_t n, int nrhs, int to_internal) {
  int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= n * nrhs) return;
  int64_t r = k / n, i = k % n;
  int64_t p = perm[i];  // internal i -> caller p
  if (to_internal) out[r * n + i] = in[r * n + p];
  else out[r * n + p] = in[r * n + i];
}

bem_status permute(const int32_t* d_perm, const double* in, double* out, int64_t n, int nrhs, bool to_internal,
                   cudaStream_t s) {
  int64_t tot = n * nrhs;
  if (tot == 0) return BEM_OK;
  k_permute<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(d_perm, in, out, n, nrhs, to_internal ? 1 : 0);
  STBEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

}  // namespace stbem
