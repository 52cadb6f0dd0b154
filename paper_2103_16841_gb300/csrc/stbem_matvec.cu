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
//   MV_TF32  tensor-core product (tcgen05, stbem_spmm_tc.cu): FP32 values
//            and x rounded to TF32 (10-bit mantissa), FP32 accumulation;
//   MV_BF16  the same on a BF16 copy of the values, x in BF16.
// The tensor-core path treats every block as a dense (rows of I) x K tile
// over the union of its rows' bands and multiplies it with the K x nrhs slab
// of x; each stored value is read from HBM once per 64 right-hand sides.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <type_traits>
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
    // passes of up to 64 right-hand sides
    for (int r0 = 0; r0 < nrhs; r0 += 64) {
      const int nr = std::min(64, nrhs - r0);
      const bem_status st = op_spmm_tc(op, x + (int64_t)r0 * n, y + (int64_t)r0 * n, nr, arith == MV_BF16, s);
      if (st != BEM_OK) return st;
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
