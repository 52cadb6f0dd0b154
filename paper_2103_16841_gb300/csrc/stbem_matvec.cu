// Products with the assembled operator over the block-banded storage.
//
// Storage (built by the quadrature epilogue): for the block of test column I
// and trial column J, every test row r of column I owns a band of W_IJ
// consecutive trial panels starting at rs[r]; the band values are stored
// column-major, value (r, w) at val[boff + w * R_I + r].
//
// Arithmetic choices, y = A x with x, y in FP64 at the boundary:
//   MV_FP64  FP64 accumulation of FP64 values (or of FP32 values when the
//            operator keeps FP32 values only) - residuals, FP64 solves;
//   MV_FP32  FP32 values, x rounded to FP32, FP32 accumulation - inner solves;
//   MV_TF32  tensor-core SpMM: FP32 values and x rounded to TF32 (10-bit
//            mantissa), FP32 accumulation (mma m16n8k8);
//   MV_BF16  tensor-core SpMM on a BF16 copy of the values, x in BF16, FP32
//            accumulation (mma m16n8k16).
// The tensor-core path treats every 16-row strip of a block as a dense
// 16 x K tile over the union of its rows' bands (K rounded up to the MMA
// depth) and multiplies it with the K x nrhs slab of x; each stored value is
// read from HBM once per product, whatever the number of right-hand sides.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <type_traits>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "stbem_internal.h"

namespace stbem {

// ---------------------------------------------------------------------------
// SpMV for one to a few right-hand sides (NR at a time, the matrix is read
// once per NR). One CTA per test column I; G groups of R_I threads split the
// trial columns J (g, g+G, ...), each thread owns one row.
// ---------------------------------------------------------------------------
template <typename V, typename Acc, typename XT, int NR>
__device__ __forceinline__ void matvec_col(int64_t n_col, const int32_t* __restrict__ ctb,
                                           const int32_t* __restrict__ bw, const int64_t* __restrict__ boff,
                                           const int64_t* __restrict__ rsoff, const int32_t* __restrict__ rs,
                                           const V* __restrict__ val, const XT* __restrict__ x,
                                           double* __restrict__ y, int64_t ld, int nrhs, int groups, int64_t I,
                                           double* red) {
  const int t0 = ctb[I], nt = ctb[I + 1] - t0;
  const int rows_pad = blockDim.x / groups;
  const int g = threadIdx.x / rows_pad, r = threadIdx.x % rows_pad;
  for (int rh0 = 0; rh0 < nrhs; rh0 += NR) {
    const int nr = min(NR, nrhs - rh0);
    Acc acc[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) acc[k] = Acc(0);
    if (r < nt) {
      // block metadata of the next J is fetched while the current block is summed
      int W_n = 0, jl_n = 0;
      int64_t vo_n = 0, ro_n = 0;
      if (g < n_col) {
        const int64_t b = I * n_col + g;
        W_n = bw[b]; vo_n = boff[b]; ro_n = rsoff[b]; jl_n = ctb[g + 1] - 1;
      }
      for (int64_t J = g; J < n_col; J += groups) {
        const int W = W_n, jl = jl_n;
        const int64_t vo = vo_n, ro = ro_n;
        if (J + groups < n_col) {
          const int64_t b = I * n_col + J + groups;
          W_n = bw[b]; vo_n = boff[b]; ro_n = rsoff[b]; jl_n = ctb[J + groups + 1] - 1;
        }
        if (W == 0) continue;
        const int start = rs[ro + r];
        const V* v = val + vo + r;
        // the band values of a chunk are loaded together (more bytes in flight
        // per warp), then summed in order
        constexpr int CW = NR == 1 ? 16 : 8;
        for (int w0 = 0; w0 < W; w0 += CW) {
          Acc av[CW];
          int jv[CW];
#pragma unroll
          for (int u = 0; u < CW; ++u) {
            const int w = w0 + u;
            jv[u] = min(start + w, jl);
            av[u] = w < W ? (Acc)v[(int64_t)w * nt] : Acc(0);
          }
#pragma unroll
          for (int k = 0; k < NR; ++k) {
            if (k < nr) {
              const XT* xr = x + (int64_t)(rh0 + k) * ld;
#pragma unroll
              for (int u = 0; u < CW; ++u)
                if (w0 + u < W) acc[k] += av[u] * (Acc)xr[jv[u]];
            }
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < NR; ++k) red[(g * rows_pad + r) * NR + k] = (double)acc[k];
    __syncthreads();
    if (g == 0 && r < nt) {
      for (int k = 0; k < nr; ++k) {
        Acc sacc = Acc(0);
        for (int q = 0; q < groups; ++q) sacc += (Acc)red[(q * rows_pad + r) * NR + k];
        y[(int64_t)(rh0 + k) * ld + t0 + r] = (double)sacc;
      }
    }
    __syncthreads();
  }
}

// SpMV for one to a few right-hand sides (NR at a time, the matrix is read
// once per NR). One CTA per test column I; G groups of R_I threads split the
// trial columns J (g, g+G, ...), each thread owns one row.
template <typename V, typename Acc, typename XT, int NR>
__global__ void k_matvec(int64_t n_col, const int32_t* __restrict__ ctb, const int32_t* __restrict__ bw,
                         const int64_t* __restrict__ boff, const int64_t* __restrict__ rsoff,
                         const int32_t* __restrict__ rs, const V* __restrict__ val, const XT* __restrict__ x,
                         double* __restrict__ y, int64_t n_tet, int nrhs, int groups) {
  extern __shared__ double red[];
  matvec_col<V, Acc, XT, NR>(n_col, ctb, bw, boff, rsoff, rs, val, x, y, n_tet, nrhs, groups, blockIdx.x, red);
}

// The same over the block-diagonal operator of a batch: CTA k works on
// column cta_col[k] of segment cta_seg[k]; a segment's entries start at
// off within each of the nrhs vectors of length ld.
struct MvSeg {
  int64_t n_col, off;
  const int32_t* ctb;
  const int32_t* bw;
  const int64_t* boff;
  const int64_t* rsoff;
  const int32_t* rs;
  const void* val;
};

template <typename V, typename Acc, typename XT, int NR>
__global__ void k_matvec_batch(const MvSeg* __restrict__ segs, const int32_t* __restrict__ cta_seg,
                               const int32_t* __restrict__ cta_col, const XT* __restrict__ x, double* __restrict__ y,
                               int64_t ld, int nrhs, int groups) {
  extern __shared__ double red[];
  const MvSeg sg = segs[cta_seg[blockIdx.x]];
  matvec_col<V, Acc, XT, NR>(sg.n_col, sg.ctb, sg.bw, sg.boff, sg.rsoff, sg.rs, static_cast<const V*>(sg.val),
                             x + sg.off, y + sg.off, ld, nrhs, groups, cta_col[blockIdx.x], red);
}

__global__ void k_to_f32(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

template <typename V>
__global__ void k_to_bf16(const V* __restrict__ in, uint16_t* __restrict__ out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __bfloat16_as_ushort(__float2bfloat16_rn((float)in[i]));
}

// ---------------------------------------------------------------------------
// Tensor-core SpMM
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t to_tf32(float f) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Packed x for the B fragments: lane (g = lane/4) of an n-tile q needs
// x[k][8q + g]; the NT8 values of all n-tiles for one k sit together.
//   TF32: Xp[j][g * NT8 + q] = tf32(x[8q + g][j])
//   BF16: Xp[p][g * NT8 + q] = bf16(x[8q + g][2p]) | bf16(x[8q + g][2p + 1]) << 16
template <bool BF16>
__global__ void k_pack_x(const double* __restrict__ x, int64_t n_tet, int nrhs, int NT8, uint32_t* __restrict__ Xp,
                         int64_t n_rows) {
  const int NRp = NT8 * 8;
  const int64_t total = n_rows * NRp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / NRp;
    const int slot = (int)(i % NRp);
    const int g = slot / NT8, q = slot % NT8;
    const int rh = 8 * q + g;
    uint32_t v = 0;
    if (rh < nrhs) {
      if (BF16) {
        const int64_t j0 = 2 * row, j1 = 2 * row + 1;
        float f0 = j0 < n_tet ? (float)x[(int64_t)rh * n_tet + j0] : 0.f;
        float f1 = j1 < n_tet ? (float)x[(int64_t)rh * n_tet + j1] : 0.f;
        v = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(f0)) |
            ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(f1)) << 16);
      } else {
        v = to_tf32((float)x[(int64_t)rh * n_tet + row]);
      }
    }
    Xp[i] = v;
  }
}

__global__ void k_unpack_y(const float* __restrict__ Y, int NRp, int64_t n_tet, int nrhs, double* __restrict__ y) {
  const int64_t total = n_tet * nrhs;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t rh = i / n_tet, j = i % n_tet;
    y[i] = (double)Y[j * NRp + rh];
  }
}

struct SpmmArgs {
  int64_t n_col;
  const int32_t* ctb;
  const int32_t* bw;
  const int64_t* boff;
  const int64_t* rsoff;
  const int32_t* rs;
  const void* val;      // float (TF32 path) or BF16 bits
  const uint32_t* X;    // packed x
  float* Y;             // [n_tet][8 NT8]
  int strips;           // ceil(max rows per column / 16)
};

template <int NT8>
__device__ __forceinline__ void load_b(const uint32_t* p, uint32_t (&b)[NT8]) {
  if constexpr (NT8 % 4 == 0) {
#pragma unroll
    for (int q = 0; q < NT8; q += 4) {
      uint4 v = __ldg(reinterpret_cast<const uint4*>(p + q));
      b[q] = v.x; b[q + 1] = v.y; b[q + 2] = v.z; b[q + 3] = v.w;
    }
  } else if constexpr (NT8 == 2) {
    uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
    b[0] = v.x; b[1] = v.y;
  } else {
#pragma unroll
    for (int q = 0; q < NT8; ++q) b[q] = __ldg(p + q);
  }
}

// One CTA per test column I: warp (strip, ws) owns rows 16 strip .. +15 and
// the trial columns J = ws, ws + WS, ...; the WS partial tiles of a strip are
// summed in a fixed order at the end.
template <bool BF16, int NT8, int WS>
__global__ void __launch_bounds__(512) k_spmm(SpmmArgs a) {
  extern __shared__ float sred[];
  constexpr int NRp = NT8 * 8;
  const int64_t I = blockIdx.x;
  const int t0 = a.ctb[I], nt = a.ctb[I + 1] - t0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int strip = warp % a.strips, ws = warp / a.strips;
  const int g = lane >> 2, t = lane & 3;
  const int r0 = strip * 16 + g, r1 = r0 + 8;
  const bool v0 = r0 < nt, v1 = r1 < nt;
  const bool any_rows = strip * 16 < nt;
  float acc[NT8][4];
#pragma unroll
  for (int q = 0; q < NT8; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
  if (any_rows) {
    for (int64_t J = ws; J < a.n_col; J += WS) {
      const int64_t b = I * a.n_col + J;
      const int W = a.bw[b];
      if (W == 0) continue;
      const int64_t vo = a.boff[b], ro = a.rsoff[b];
      const int je = a.ctb[J + 1];
      const int s0 = v0 ? a.rs[ro + r0] : INT_MAX;
      const int s1 = v1 ? a.rs[ro + r1] : INT_MAX;
      int smin = min(s0, s1);
      int smax = max(v0 ? s0 : INT_MIN, v1 ? s1 : INT_MIN);
#pragma unroll
      for (int o = 16; o >= 4; o >>= 1) {
        smin = min(smin, __shfl_xor_sync(0xffffffffu, smin, o));
        smax = max(smax, __shfl_xor_sync(0xffffffffu, smax, o));
      }
      int c0 = smin;
      if (BF16) c0 &= ~1;
      const int K = smax + W - c0;
      if (!BF16) {
        const float* val = static_cast<const float*>(a.val) + vo;
        auto ld = [&](bool v, int r, int s, int c) -> uint32_t {
          const int w = c - s;
          return (v && w >= 0 && w < W && c < je) ? to_tf32(__ldg(val + (int64_t)w * nt + r)) : 0u;
        };
        for (int k0 = 0; k0 < K; k0 += 8) {
          const int ca = c0 + k0 + t, cb = ca + 4;
          const uint32_t A0 = ld(v0, r0, s0, ca), A1 = ld(v1, r1, s1, ca);
          const uint32_t A2 = ld(v0, r0, s0, cb), A3 = ld(v1, r1, s1, cb);
          uint32_t B0[NT8], B1[NT8];
          load_b<NT8>(a.X + (int64_t)min(ca, je - 1) * NRp + g * NT8, B0);
          load_b<NT8>(a.X + (int64_t)min(cb, je - 1) * NRp + g * NT8, B1);
#pragma unroll
          for (int q = 0; q < NT8; ++q) mma_tf32(acc[q], A0, A1, A2, A3, B0[q], B1[q]);
        }
      } else {
        const uint16_t* val = static_cast<const uint16_t*>(a.val) + vo;
        auto ld = [&](bool v, int r, int s, int c) -> uint32_t {
          const int w = c - s;
          return (v && w >= 0 && w < W && c < je) ? (uint32_t)__ldg(val + (int64_t)w * nt + r) : 0u;
        };
        const int plast = (je - 1) >> 1;
        for (int k0 = 0; k0 < K; k0 += 16) {
          const int pa = c0 + k0 + 2 * t, pb = pa + 8;
          const uint32_t A0 = ld(v0, r0, s0, pa) | (ld(v0, r0, s0, pa + 1) << 16);
          const uint32_t A1 = ld(v1, r1, s1, pa) | (ld(v1, r1, s1, pa + 1) << 16);
          const uint32_t A2 = ld(v0, r0, s0, pb) | (ld(v0, r0, s0, pb + 1) << 16);
          const uint32_t A3 = ld(v1, r1, s1, pb) | (ld(v1, r1, s1, pb + 1) << 16);
          uint32_t B0[NT8], B1[NT8];
          load_b<NT8>(a.X + (int64_t)min(pa >> 1, plast) * NRp + g * NT8, B0);
          load_b<NT8>(a.X + (int64_t)min(pb >> 1, plast) * NRp + g * NT8, B1);
#pragma unroll
          for (int q = 0; q < NT8; ++q) mma_bf16(acc[q], A0, A1, A2, A3, B0[q], B1[q]);
        }
      }
    }
  }
  if constexpr (WS > 1) {
    const int slab = NT8 * 4 * 32;
    if (ws > 0 && any_rows) {
      float* dst = sred + (int64_t)((ws - 1) * a.strips + strip) * slab;
#pragma unroll
      for (int q = 0; q < NT8; ++q)
#pragma unroll
        for (int e = 0; e < 4; ++e) dst[(q * 4 + e) * 32 + lane] = acc[q][e];
    }
    __syncthreads();
    if (ws == 0 && any_rows) {
      for (int u = 1; u < WS; ++u) {
        const float* src = sred + (int64_t)((u - 1) * a.strips + strip) * slab;
#pragma unroll
        for (int q = 0; q < NT8; ++q)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc[q][e] += src[(q * 4 + e) * 32 + lane];
      }
    }
  }
  if (ws == 0 && any_rows) {
#pragma unroll
    for (int q = 0; q < NT8; ++q) {
      const int col = 8 * q + 2 * t;
      if (v0) *reinterpret_cast<float2*>(a.Y + (int64_t)(t0 + r0) * NRp + col) = make_float2(acc[q][0], acc[q][1]);
      if (v1) *reinterpret_cast<float2*>(a.Y + (int64_t)(t0 + r1) * NRp + col) = make_float2(acc[q][2], acc[q][3]);
    }
  }
}

namespace {

unsigned grid_for(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16); }

bem_status ensure_ws(const bem_operator* op, int64_t floats) {
  if (op->ws_len >= floats) return BEM_OK;
  if (op->d_ws) cudaFree(op->d_ws);
  op->d_ws = nullptr;
  op->ws_len = 0;
  if (cudaMalloc(&op->d_ws, sizeof(float) * floats) != cudaSuccess) {
    cudaGetLastError();
    set_error("out of device memory (matvec workspace)");
    return BEM_ERR_OUT_OF_MEMORY;
  }
  op->ws_len = floats;
  return BEM_OK;
}

bem_status ensure_val16(const bem_operator* op, cudaStream_t s) {
  if (op->d_val16) return BEM_OK;
  const int64_t n = std::max<int64_t>(op->nstored, 1);
  if (cudaMalloc(&op->d_val16, sizeof(uint16_t) * n) != cudaSuccess) {
    cudaGetLastError();
    op->d_val16 = nullptr;
    set_error("out of device memory (BF16 values)");
    return BEM_ERR_OUT_OF_MEMORY;
  }
  if (op->nstored > 0) {
    if (op->d_val32) k_to_bf16<float><<<grid_for(op->nstored), 256, 0, s>>>(op->d_val32, op->d_val16, op->nstored);
    else k_to_bf16<double><<<grid_for(op->nstored), 256, 0, s>>>(op->d_val, op->d_val16, op->nstored);
    STBEM_CUDA(cudaGetLastError());
  }
  return BEM_OK;
}

// candidate warps per strip, the tuned choice per shape (process-wide, so
// that equal shapes always take the same summation order)
std::mutex g_tune_mu;
std::map<std::tuple<int64_t, int, int, int, int>, int> g_tuned;

template <bool BF16, int NT8, int WS>
bem_status launch_spmm_ws(const SpmmArgs& a, cudaStream_t s) {
  const int threads = a.strips * WS * 32;
  const size_t smem = WS > 1 ? sizeof(float) * (size_t)(WS - 1) * a.strips * NT8 * 4 * 32 : 0;
  if (smem > 48 * 1024)
  {
      bem_status sa = ensure_smem_attr((const void*)k_spmm<BF16, NT8, WS>, smem);
      if (sa != BEM_OK) return sa;
    }
  k_spmm<BF16, NT8, WS><<<(unsigned)a.n_col, threads, smem, s>>>(a);
  STBEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

template <bool BF16, int NT8>
bem_status launch_spmm(const SpmmArgs& a, int ws, cudaStream_t s) {
  switch (ws) {
    case 1: return launch_spmm_ws<BF16, NT8, 1>(a, s);
    case 2: return launch_spmm_ws<BF16, NT8, 2>(a, s);
    case 4: return launch_spmm_ws<BF16, NT8, 4>(a, s);
    default: return launch_spmm_ws<BF16, NT8, 8>(a, s);
  }
}

bool ws_ok(int strips, int nt8, int ws) {
  return strips * ws <= 16 && (ws == 1 || (size_t)(ws - 1) * strips * nt8 * 4 * 32 * 4 <= 100 * 1024);
}

template <bool BF16, int NT8>
bem_status run_spmm(const bem_operator* op, const SpmmArgs& a, cudaStream_t s) {
  const auto key = std::make_tuple(op->mesh->n_col, op->mesh->max_col_tets, NT8, (int)BF16, op->ctx->device);
  // candidates differ in summation order: the choice is kept per shape for the process
  int ws = 0;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) ws = it->second;
  }
  if (ws) return launch_spmm<BF16, NT8>(a, ws, s);
  // autotune: time every admissible candidate once (after one warm-up launch)
  cudaEvent_t e0, e1;
  STBEM_CUDA(cudaEventCreate(&e0));
  STBEM_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_ws = 1;
  bem_status st = BEM_OK;
  for (int c : {1, 2, 4, 8}) {
    if (!ws_ok(a.strips, NT8, c)) continue;
    if ((st = launch_spmm<BF16, NT8>(a, c, s)) != BEM_OK) break;
    cudaEventRecord(e0, s);
    if ((st = launch_spmm<BF16, NT8>(a, c, s)) != BEM_OK) break;
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) { best = ms; best_ws = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != BEM_OK) return st;
  if (best >= 1e30f) {
    set_error("tensor-core product: no launch shape fits this operator");
    return BEM_ERR_UNSUPPORTED;
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = best_ws;
  }
  // the result of the chosen variant (the candidates differ in summation order)
  return launch_spmm<BF16, NT8>(a, best_ws, s);
}

template <bool BF16>
bem_status spmm_nt8(const bem_operator* op, const SpmmArgs& a, int nt8, cudaStream_t s) {
  switch (nt8) {
    case 1: return run_spmm<BF16, 1>(op, a, s);
    case 2: return run_spmm<BF16, 2>(op, a, s);
    case 4: return run_spmm<BF16, 4>(op, a, s);
    default: return run_spmm<BF16, 8>(op, a, s);
  }
}

}  // namespace

// NR right-hand sides per pass over the values (1: the single-vector kernel,
// with fewer registers)
template <int NR>
static bem_status spmv_launch(const bem_operator* op, const double* x, double* y, int nrhs, int arith, int threads,
                              int groups, cudaStream_t s) {
  const bem_mesh* m = op->mesh;
  const int64_t n = m->n_tet;
  const size_t smem = sizeof(double) * threads * NR;
  if (arith == MV_FP32) {
    if (!op->d_val32) {
      set_error("operator has no FP32 values (store_fp32 = 0)");
      return BEM_ERR_INVALID_ARG;
    }
    bem_status st = ensure_ws(op, n * nrhs);
    if (st != BEM_OK) return st;
    k_to_f32<<<grid_for(n * nrhs), 256, 0, s>>>(x, op->d_ws, n * nrhs);
    k_matvec<float, float, float, NR><<<(unsigned)m->n_col, threads, smem, s>>>(
        m->n_col, m->d_col_tet_begin, op->d_bw, op->d_boff, op->d_rsoff, op->d_rs, op->d_val32, op->d_ws, y, n,
        nrhs, groups);
  } else if (op->d_val) {
    k_matvec<double, double, double, NR><<<(unsigned)m->n_col, threads, smem, s>>>(
        m->n_col, m->d_col_tet_begin, op->d_bw, op->d_boff, op->d_rsoff, op->d_rs, op->d_val, x, y, n, nrhs,
        groups);
  } else {
    // mixed-precision operators keep FP32 values only
    k_matvec<float, double, double, NR><<<(unsigned)m->n_col, threads, smem, s>>>(
        m->n_col, m->d_col_tet_begin, op->d_bw, op->d_boff, op->d_rsoff, op->d_rs, op->d_val32, x, y, n, nrhs,
        groups);
  }
  STBEM_CUDA(cudaGetLastError());
  return BEM_OK;
}


bem_status op_matvec(const bem_operator* op, const double* x, double* y, int nrhs, int arith, cudaStream_t s) {
  // matrix-free operators: the operator's own precision, whatever `arith` asks
  if (op->opts.matrix_free) return op_matvec_free(op, x, y, nrhs, s);
  const bem_mesh* m = op->mesh;
  const int64_t n = m->n_tet;
  if (arith == MV_TF32 || arith == MV_BF16) {
    // groups of up to 64 right-hand sides
    for (int r0 = 0; r0 < nrhs; r0 += 64) {
      const int nr = std::min(64, nrhs - r0);
      const int nt8 = nr <= 8 ? 1 : nr <= 16 ? 2 : nr <= 32 ? 4 : 8;
      const int NRp = nt8 * 8;
      const bool bf16 = arith == MV_BF16;
      const float* vals32 = op->d_val32;
      if (!bf16 && !vals32) {
        set_error("TF32 products need FP32 values (store_fp32 = 1)");
        return BEM_ERR_INVALID_ARG;
      }
      if (bf16) {
        bem_status st = ensure_val16(op, s);
        if (st != BEM_OK) return st;
      }
      const int64_t xrows = bf16 ? (n + 1) / 2 : n;
      bem_status st = ensure_ws(op, xrows * NRp + n * NRp);
      if (st != BEM_OK) return st;
      uint32_t* Xp = reinterpret_cast<uint32_t*>(op->d_ws);
      float* Yp = op->d_ws + xrows * NRp;
      const double* xr = x + (int64_t)r0 * n;
      if (bf16) k_pack_x<true><<<grid_for(xrows * NRp), 256, 0, s>>>(xr, n, nr, nt8, Xp, xrows);
      else k_pack_x<false><<<grid_for(xrows * NRp), 256, 0, s>>>(xr, n, nr, nt8, Xp, xrows);
      STBEM_CUDA(cudaGetLastError());
      SpmmArgs a;
      a.n_col = m->n_col;
      a.ctb = m->d_col_tet_begin;
      a.bw = op->d_bw;
      a.boff = op->d_boff;
      a.rsoff = op->d_rsoff;
      a.rs = op->d_rs;
      a.val = bf16 ? (const void*)op->d_val16 : (const void*)vals32;
      a.X = Xp;
      a.Y = Yp;
      a.strips = (m->max_col_tets + 15) / 16;
      st = bf16 ? spmm_nt8<true>(op, a, nt8, s) : spmm_nt8<false>(op, a, nt8, s);
      if (st != BEM_OK) return st;
      k_unpack_y<<<grid_for(n * nr), 256, 0, s>>>(Yp, NRp, n, nr, y + (int64_t)r0 * n);
      STBEM_CUDA(cudaGetLastError());
    }
    return BEM_OK;
  }
  const int rows_pad = ((m->max_col_tets + 31) / 32) * 32;
  const int groups = std::max(1, std::min(8, 512 / rows_pad));
  const int threads = rows_pad * groups;
  if (nrhs == 1) return spmv_launch<1>(op, x, y, nrhs, arith, threads, groups, s);
  return spmv_launch<4>(op, x, y, nrhs, arith, threads, groups, s);
}

bem_status BatchMatvec::init(const std::vector<bem_operator*>& o, cudaStream_t s) {
  ops = o;
  const int S = (int)ops.size();
  std::vector<MvSeg> segs(S);
  std::vector<int32_t> cseg, ccol;
  N = 0;
  int max_rows = 1;
  fp64_values = ops.empty() ? false : ops[0]->d_val != nullptr;
  for (int i = 0; i < S; ++i) {
    const bem_operator* op = ops[i];
    if ((op->d_val != nullptr) != fp64_values) {
      set_error("a batch takes one value precision");
      return BEM_ERR_INVALID_ARG;
    }
    segs[i].n_col = op->mesh->n_col;
    segs[i].off = N;
    segs[i].ctb = op->mesh->d_col_tet_begin;
    segs[i].bw = op->d_bw;
    segs[i].boff = op->d_boff;
    segs[i].rsoff = op->d_rsoff;
    segs[i].rs = op->d_rs;
    segs[i].val = fp64_values ? (const void*)op->d_val : (const void*)op->d_val32;
    for (int64_t I = 0; I < op->mesh->n_col; ++I) {
      cseg.push_back(i);
      ccol.push_back((int32_t)I);
    }
    max_rows = std::max(max_rows, op->mesh->max_col_tets);
    N += op->mesh->n_tet;
  }
  n_cta = (int64_t)cseg.size();
  rows_pad = ((max_rows + 31) / 32) * 32;
  groups = std::max(1, std::min(8, 512 / rows_pad));
  if (cudaMalloc(&d_segs, sizeof(MvSeg) * std::max(S, 1)) != cudaSuccess ||
      cudaMalloc(&d_cseg, sizeof(int32_t) * std::max<int64_t>(n_cta, 1)) != cudaSuccess ||
      cudaMalloc(&d_ccol, sizeof(int32_t) * std::max<int64_t>(n_cta, 1)) != cudaSuccess) {
    cudaGetLastError();
    set_error("out of device memory (batch matvec tables)");
    return BEM_ERR_OUT_OF_MEMORY;
  }
  STBEM_CUDA(cudaMemcpyAsync(d_segs, segs.data(), sizeof(MvSeg) * S, cudaMemcpyHostToDevice, s));
  STBEM_CUDA(cudaMemcpyAsync(d_cseg, cseg.data(), sizeof(int32_t) * n_cta, cudaMemcpyHostToDevice, s));
  STBEM_CUDA(cudaMemcpyAsync(d_ccol, ccol.data(), sizeof(int32_t) * n_cta, cudaMemcpyHostToDevice, s));
  STBEM_CUDA(cudaStreamSynchronize(s));
  return BEM_OK;
}

BatchMatvec::~BatchMatvec() {
  if (d_segs) cudaFree(d_segs);
  if (d_cseg) cudaFree(d_cseg);
  if (d_ccol) cudaFree(d_ccol);
  if (d_xf) cudaFree(d_xf);
}

bem_status BatchMatvec::apply(const double* x, double* y, int K, int arith, cudaStream_t s) {
  const int threads = rows_pad * groups;
  constexpr int NR = 4;
  const size_t smem = sizeof(double) * threads * NR;
  const MvSeg* sg = static_cast<const MvSeg*>(d_segs);
  if (arith == MV_FP32 && !fp64_values) {
    if (xf_len < N * K) {
      if (d_xf) cudaFree(d_xf);
      d_xf = nullptr;
      xf_len = 0;
      if (cudaMalloc(&d_xf, sizeof(float) * N * K) != cudaSuccess) {
        cudaGetLastError();
        set_error("out of device memory (batch matvec workspace)");
        return BEM_ERR_OUT_OF_MEMORY;
      }
      xf_len = N * K;
    }
    k_to_f32<<<grid_for(N * K), 256, 0, s>>>(x, d_xf, N * K);
    k_matvec_batch<float, float, float, NR><<<(unsigned)n_cta, threads, smem, s>>>(sg, d_cseg, d_ccol, d_xf, y, N,
                                                                                   K, groups);
  } else if (arith == MV_FP64 || arith == MV_FP32) {
    if (fp64_values)
      k_matvec_batch<double, double, double, NR><<<(unsigned)n_cta, threads, smem, s>>>(sg, d_cseg, d_ccol, x, y, N,
                                                                                        K, groups);
    else
      k_matvec_batch<float, double, double, NR><<<(unsigned)n_cta, threads, smem, s>>>(sg, d_cseg, d_ccol, x, y, N,
                                                                                       K, groups);
  } else {
    set_error("batched products support FP64 and FP32 arithmetic");
    return BEM_ERR_UNSUPPORTED;
  }
  STBEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

}  // namespace stbem
