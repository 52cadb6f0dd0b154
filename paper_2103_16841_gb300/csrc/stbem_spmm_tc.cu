// Tensor-core block product Y = A X for up to 64 right-hand sides per pass
// (the multi-right-hand-side product of the GMRES solves; A in TF32 or BF16,
// FP32 accumulation in tensor memory).
//
// Storage of A (eq. int_bform assembled into column blocks): block (I, J)
// holds, for every panel row r of spatial column I, a band of W values
// starting at trial panel rs[r]. Within a block the union of the rows' bands
// is a contiguous range of trial panels [cmin, cend), so block (I, J) is a
// dense (rows of I) x (cend - cmin) tile with the band filled in and zeros
// elsewhere: a dense contraction with the matching rows of X.
//
// Operand layout in shared memory (no swizzle): 16-byte chunks along K; chunk
// kc of row m at kc * (rows * 16) + m * 16, i.e. core matrices of 8 rows x
// 16 bytes, K-adjacent core matrices rows * 16 bytes apart (leading byte
// offset), M/N-adjacent ones 128 bytes apart (stride byte offset).
//   X is packed per pass as Xc[chunk][rhs][16 bytes]; one chunk is N x 16
//   contiguous bytes, and a TMA box of {256-byte rows, N / 16 rows, 2
//   chunks} (one K step) lands in exactly this layout.
//   The values are kept, for this product, in the same chunks: row r's band
//   re-cut at the 16-byte chunk boundaries of the trial panel index (slot j
//   of row r = the chunk starting at panel E * (floor(rs[r] / E) + j), zeros
//   outside the band), stored per block as [slot][row] (made once from the
//   assembled values, BF16 or TF32-rounded, about 1.1-1.25 x their bytes).
//   Building a block's A tile is then a copy of whole chunks.
//
// One CTA per test column I, six warps:
//   warps 0-3  build the A tile of each block (thread = row: its slots to
//              their chunk positions, the previous band's other chunks
//              cleared) in shared memory (k_spmm_tc) or in tensor memory with
//              tcgen05.st (k_spmm_tm; the MMA then reads A from tensor
//              memory, and shared memory holds only B, slots and row starts,
//              so more stages fit), then read the accumulator rows out of
//              tensor memory (thread = row) into y;
//   warp 4     (one lane) loads, per block, the X rows (TMA tensor copies),
//              the value slots and the row starts (bulk copies) and the
//              block's record, into one of up to 6 pipeline stages;
//   warp 5     owns the tensor-memory allocation; one lane issues
//              tcgen05.mma (M = 128 rows, N = right-hand sides rounded up to
//              16, K = 16 BF16 or 8 TF32 per instruction) accumulating every
//              block of the column into one tensor-memory tile, and commits
//              each stage back to the builders and the loader.
// Which kernel and how many stages (1-6) run is timed once per shape.
// Every mbarrier wait is bounded (kWaitBudget); a wait that runs out flags
// the operator, stops the CTA's pipeline and writes NaN to its rows.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "stbem_internal.h"
#include "stbem_tc.cuh"

namespace stbem {

// One non-empty block of a test column, in the order of its trial columns.
struct TcBlk {
  int32_t je;          // end of trial column J (internal panel index)
  int32_t W;           // band width
  int32_t nt;          // rows (panels of column I)
  int32_t cmin;        // union of the rows' bands [cmin, cend), clipped to J
  int32_t cend;
  int32_t pad;
  int64_t vo;          // value offset in the assembled storage
  int64_t ro;          // row-start offset
  int64_t vc[2];       // offset of the block's chunk slots (16-byte units): BF16, TF32
  int64_t pad2;
};
static_assert(sizeof(TcBlk) == 64, "TcBlk layout");

#define TRY_STATUS(x)                 \
  do {                                \
    const bem_status st_ = (x);       \
    if (st_ != BEM_OK) return st_;    \
  } while (0)

namespace {

constexpr long long kWaitBudget = 4000000000LL;   // clock cycles (about 2 s) per wait
constexpr int kThreads = 192;
constexpr int kMaxStages = 6;
// after the stages: 3 mbarriers per stage and one more, the tensor-memory
// address and the abort flag
constexpr size_t kTailBytes = 256;
static_assert(8 * (3 * kMaxStages + 1) + 8 <= kTailBytes, "stage tail");
constexpr uint32_t kRsBytes = 1024;   // per stage: row starts (<= 784 bytes) and the block record
constexpr uint32_t kMetaOff = 896;

// chunk slots of a row's band of width W (E values per chunk)
__host__ __device__ constexpr int tc_slots(int W, int E) { return (W + 2 * E - 2) / E; }

__global__ void k_tc_meta(int64_t nb, const int32_t* __restrict__ bI, const int32_t* __restrict__ bJ,
                          const int64_t* __restrict__ vc16, const int64_t* __restrict__ vc32, int64_t n_col,
                          const int32_t* __restrict__ ctb, const int32_t* __restrict__ bw,
                          const int64_t* __restrict__ boff, const int64_t* __restrict__ rsoff,
                          const int32_t* __restrict__ rs, TcBlk* __restrict__ out, int* __restrict__ span) {
  const int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= nb) return;
  const int64_t I = bI[k], J = bJ[k], b = I * n_col + J;
  const int nt = ctb[I + 1] - ctb[I];
  const int W = bw[b];
  const int64_t ro = rsoff[b];
  int lo = INT_MAX, hi = INT_MIN;
  for (int r = lane; r < nt; r += 32) {
    const int s = rs[ro + r];
    lo = min(lo, s);
    hi = max(hi, s + W);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if (lane == 0) {
    const int je = ctb[J + 1];
    hi = min(hi, je);
    TcBlk t;
    t.je = je;
    t.W = W;
    t.nt = nt;
    t.cmin = lo;
    t.cend = hi;
    t.pad = 0;
    t.vo = boff[b];
    t.ro = ro;
    t.vc[0] = vc16[k];
    t.vc[1] = vc32[k];
    t.pad2 = 0;
    out[k] = t;
    atomicMax(&span[0], hi - (lo & ~7));   // BF16: chunks of 8
    atomicMax(&span[1], hi - (lo & ~3));   // TF32: chunks of 4
  }
}

// The chunk slots of every block (warp per block): slot j of row r holds the
// values of trial panels E * (floor(rs[r] / E) + j) + [0, E) that lie in the
// row's band (and in column J), zeros elsewhere; BF16 or TF32-rounded FP32.
template <bool TF32, typename V>
__global__ void k_tc_pack_vals(int64_t nb, const TcBlk* __restrict__ blk, const V* __restrict__ val,
                               const int32_t* __restrict__ rs, uint4* __restrict__ out) {
  constexpr int E = TF32 ? 4 : 8;
  const int lane = threadIdx.x & 31;
  for (int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; k < nb;
       k += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const TcBlk b = blk[k];
    const int S = tc_slots(b.W, E), nt = b.nt;
    for (int idx = lane; idx < S * nt; idx += 32) {
      const int j = idx / nt, r = idx - j * nt;
      const int st = rs[b.ro + r];
      const int base = (st / E) * E + j * E;
      uint32_t wv[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        if (TF32) {
          const int col = base + h, w = col - st;
          const float v = (w >= 0 && w < b.W && col < b.je) ? (float)val[b.vo + (int64_t)w * nt + r] : 0.f;
          uint32_t t;
          asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(v));
          wv[h] = t;
        } else {
          uint32_t p = 0;
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int col = base + 2 * h + e, w = col - st;
            const float v = (w >= 0 && w < b.W && col < b.je) ? (float)val[b.vo + (int64_t)w * nt + r] : 0.f;
            p |= (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v)) << (16 * e);
          }
          wv[h] = p;
        }
      }
      out[b.vc[TF32 ? 1 : 0] + (int64_t)j * nt + r] = make_uint4(wv[0], wv[1], wv[2], wv[3]);
    }
  }
}

// Xc[c][n][e] = x[n][c E + e] (zero outside), BF16 or TF32-rounded FP32.
template <bool TF32>
__global__ void k_pack_xc(const double* __restrict__ x, int64_t n_tet, int nr, int N, int64_t nchunks,
                          void* __restrict__ Xc) {
  constexpr int E = TF32 ? 4 : 8;
  const int64_t total = nchunks * N * E;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = i / (N * E);
    const int rem = (int)(i % (N * E));
    const int n = rem / E, e = rem % E;
    const int64_t j = c * E + e;
    const float v = (n < nr && j < n_tet) ? (float)x[(int64_t)n * n_tet + j] : 0.f;
    if (TF32) {
      uint32_t t;
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(v));
      static_cast<uint32_t*>(Xc)[i] = t;
    } else {
      static_cast<uint16_t*>(Xc)[i] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
  }
}

struct TcArgs {
  const int32_t* ctb;
  const int32_t* colptr;   // [n_col + 1] into blk
  const TcBlk* blk;
  const uint4* vals;       // chunk slots of the product's type
  const int32_t* rs;       // row starts (16 bytes of tail room)
  double* y;               // [nr][n_tet] (internal order)
  int64_t n_tet;
  int nr, N;               // right-hand sides of the pass, MMA N (multiple of 16)
  int nkc;                 // chunk capacity of a stage's A and B tiles (even)
  uint32_t v_bytes;        // capacity of a stage's value buffer (multiple of 1024)
  int stages;
  uint32_t tmem_cols;
  int* err;                // set to 1 when a wait ran out of budget
};

// Per stage in shared memory: the A tile, the B tile (X rows), the block's
// value slots, its row starts (bulk copy from the 16-byte granule holding
// the first one) and its record (written by the loader).
template <bool TF32, int MT>
__global__ void __launch_bounds__(kThreads, 1) k_spmm_tc(const TcArgs a, const __grid_constant__ CUtensorMap tmx) {
  using namespace tc;
  constexpr int E = TF32 ? 4 : 8;         // elements per 16-byte chunk
  constexpr int ROWS = MT * 128;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t I = blockIdx.x;
  const int t0 = a.ctb[I], nt = a.ctb[I + 1] - t0;
  const int b0 = a.colptr[I], nb = a.colptr[I + 1] - b0;
  const int ST = a.stages, N = a.N;
  const uint32_t a_bytes = (uint32_t)a.nkc * ROWS * 16, b_bytes = (uint32_t)a.nkc * N * 16;
  const uint32_t stage_bytes = a_bytes + b_bytes + a.v_bytes + kRsBytes;
  unsigned char* bar_base = smem + (size_t)ST * stage_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(bar_base);   // full_a[ST], full_b[ST], empty[ST], done
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar_base + 8 * (3 * ST + 1));
  volatile int* abort_flag = reinterpret_cast<int*>(bar_base + 8 * (3 * ST + 1) + 4);
  auto full_a = [&](int s) { return smem_u32(&bars[s]); };
  auto full_b = [&](int s) { return smem_u32(&bars[ST + s]); };
  auto empty = [&](int s) { return smem_u32(&bars[2 * ST + s]); };
  const uint32_t done = smem_u32(&bars[3 * ST]);
  auto stage_a = [&](int s) { return smem + (size_t)s * stage_bytes; };
  auto stage_b = [&](int s) { return smem + (size_t)s * stage_bytes + a_bytes; };
  auto stage_v = [&](int s) { return smem + (size_t)s * stage_bytes + a_bytes + b_bytes; };
  auto stage_r = [&](int s) { return smem + (size_t)s * stage_bytes + a_bytes + b_bytes + a.v_bytes; };
  auto meta = [&](int s) { return reinterpret_cast<TcBlk*>(stage_r(s) + kMetaOff); };
  auto fail = [&]() {
    *abort_flag = 1;
    atomicExch(a.err, 1);
  };

  if (tid == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(full_a(s), 128);
      mbar_init(full_b(s), 1);
      mbar_init(empty(s), 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    fence_proxy_async();
  }
  if (warp == 5) tmem_alloc(smem_u32(slot), a.tmem_cols);
  // the A tiles start zero; afterwards each row rewrites or clears only the
  // chunks its previous band touched
  if (warp < 4)
    for (int s = 0; s < ST; ++s)
      for (int kc = 0; kc < a.nkc; ++kc)
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
          *reinterpret_cast<uint4*>(stage_a(s) + (size_t)kc * ROWS * 16 + (tid + 128 * mt) * 16) = make_uint4(0, 0, 0, 0);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;

  if (warp < 4) {
    // ---------------------------------------------------------------- builders
    int dirty_lo[kMaxStages][MT], dirty_hi[kMaxStages][MT];   // chunks of each stage's row band
#pragma unroll
    for (int q = 0; q < kMaxStages; ++q)
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) dirty_lo[q][mt] = dirty_hi[q][mt] = 0;
    for (int k = 0; k < nb; ++k) {
      const int s = k % ST, u = k / ST;
      if (u > 0 && !mbar_wait(empty(s), (u - 1) & 1, kWaitBudget)) { fail(); break; }
      if (!mbar_wait(full_b(s), u & 1, kWaitBudget)) { fail(); break; }   // record, values, row starts landed
      if (*abort_flag) break;
      const TcBlk* bm = meta(s);
      const int c0c = bm->cmin / E;                      // first chunk of the tile (trial panel index / E)
      const int nkk = 2 * ((bm->cend - c0c * E + 2 * E - 1) / (2 * E));   // chunks the MMAs read
      const int S = tc_slots(bm->W, E);
      const int32_t* R = reinterpret_cast<const int32_t*>(stage_r(s)) + (int)((bm->ro & 3));
      const uint4* V = reinterpret_cast<const uint4*>(stage_v(s));
      unsigned char* A = stage_a(s);
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        const int r = tid + 128 * mt;
        unsigned char* row = A + r * 16;
        int lo_old = 0, hi_old = 0;
#pragma unroll
        for (int q = 0; q < kMaxStages; ++q)
          if (q == s) { lo_old = dirty_lo[q][mt]; hi_old = dirty_hi[q][mt]; }
        int lo_new = 0, hi_new = 0;
        if (r < nt) {
          lo_new = R[r] / E - c0c;
          hi_new = min(lo_new + S, nkk);
          for (int kc = lo_new; kc < hi_new; ++kc)
            *reinterpret_cast<uint4*>(row + (size_t)kc * ROWS * 16) = V[(kc - lo_new) * nt + r];
        }
        for (int kc = lo_old; kc < hi_old; ++kc)
          if (kc < lo_new || kc >= hi_new)
            *reinterpret_cast<uint4*>(row + (size_t)kc * ROWS * 16) = make_uint4(0, 0, 0, 0);
#pragma unroll
        for (int q = 0; q < kMaxStages; ++q)
          if (q == s) { dirty_lo[q][mt] = lo_new; dirty_hi[q][mt] = hi_new; }
      }
      fence_proxy_async();
      mbar_arrive(full_a(s));
    }
    // ---------------------------------------------------------------- epilogue
    __syncwarp();
    const bool ok = mbar_wait(done, 0, kWaitBudget);
    if (!ok) fail();
    tc_fence_after();
    const bool bad = !ok || *abort_flag;
    __syncwarp();
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      const int r = mt * 128 + warp * 32 + lane;
      for (int c = 0; c < N; c += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(mt * N + c), v);
        if (r < nt) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int n = c + j;
            if (n < a.nr) {
              const double o = nb == 0 ? 0.0 : bad ? __longlong_as_double(0x7ff8000000000000LL) : (double)v[j];
              a.y[(int64_t)n * a.n_tet + t0 + r] = o;
            }
          }
        }
      }
    }
  } else if (warp == 4) {
    // ---------------------------------------------------------------- loader
    if (lane == 0) {
      prefetch_tensormap(&tmx);
      int issued = 0;
      TcBlk nxt = nb > 0 ? a.blk[b0] : TcBlk{};
      for (int k = 0; k < nb; ++k) {
        const int s = k % ST, u = k / ST;
        const TcBlk b = nxt;
        if (k + 1 < nb) nxt = a.blk[b0 + k + 1];          // the next record in flight meanwhile
        if (u > 0 && !mbar_wait(empty(s), (u - 1) & 1, kWaitBudget)) { fail(); break; }
        if (*abort_flag) break;
        *meta(s) = b;
        const int c0c = b.cmin / E;
        const int nk = (b.cend - c0c * E + 2 * E - 1) / (2 * E);
        const uint32_t v_bytes = (uint32_t)tc_slots(b.W, E) * nt * 16;
        const uint64_t rs_src = reinterpret_cast<uint64_t>(a.rs + (b.ro & ~(int64_t)3));
        const uint32_t rs_bytes = (uint32_t)(((b.ro & 3) + nt + 3) & ~3) * 4;
        mbar_arrive_expect_tx(full_b(s), (uint32_t)nk * 2 * N * 16 + v_bytes + rs_bytes);
        const uint32_t B = smem_u32(stage_b(s));
        for (int ks = 0; ks < nk; ++ks) tma_load_3d(B + (uint32_t)ks * 2 * N * 16, &tmx, 0, 0, c0c + 2 * ks, full_b(s));
        bulk_load(smem_u32(stage_v(s)), reinterpret_cast<uint64_t>(a.vals + b.vc[TF32 ? 1 : 0]), v_bytes, full_b(s));
        bulk_load(smem_u32(stage_r(s)), rs_src, rs_bytes, full_b(s));
        issued = k + 1;
      }
      // copies still in flight land before the CTA's shared memory is released
      for (int k = max(0, issued - ST); k < issued; ++k)
        if (!mbar_wait(full_b(k % ST), (k / ST) & 1, kWaitBudget)) fail();
    }
  } else {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = instr_desc(TF32 ? 2u : 1u, 128, N);
      for (int k = 0; k < nb; ++k) {
        const int s = k % ST, u = k / ST;
        if (!mbar_wait(full_a(s), u & 1, kWaitBudget) || !mbar_wait(full_b(s), u & 1, kWaitBudget)) {
          fail();
          break;
        }
        if (*abort_flag) break;
        tc_fence_after();
        const TcBlk* bm = meta(s);
        const int c0c = bm->cmin / E;
        const int nk = (bm->cend - c0c * E + 2 * E - 1) / (2 * E);
        const uint32_t A = smem_u32(stage_a(s)), B = smem_u32(stage_b(s));
        for (int ks = 0; ks < nk; ++ks) {
          const uint64_t bd = smem_desc(B + (uint32_t)ks * 2 * N * 16, (uint32_t)N * 16, 128);
#pragma unroll
          for (int mt = 0; mt < MT; ++mt) {
            const uint64_t ad = smem_desc(A + (uint32_t)ks * 2 * ROWS * 16 + mt * 128 * 16, ROWS * 16, 128);
            mma<TF32>(tmem + (uint32_t)(mt * N), ad, bd, idesc, (k > 0 || ks > 0) ? 1u : 0u);
          }
        }
        mma_commit(empty(s));
      }
      mma_commit(done);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 5) {
    tc_fence_after();
    tmem_dealloc(tmem, a.tmem_cols);
  }
}

// The same product with the A tiles in tensor memory: per stage MT x nkc
// chunks of 4 columns each (row m = lane m), written by the builder warps
// with tcgen05.st (warp w owns lanes 32w..32w+31, i.e. rows 32w + lane) and
// read by the MMA straight from tensor memory; shared memory then holds only
// the B tiles, value slots and row starts, so more stages fit.
template <bool TF32, int MT>
__global__ void __launch_bounds__(kThreads, 1) k_spmm_tm(const TcArgs a, const __grid_constant__ CUtensorMap tmx) {
  using namespace tc;
  constexpr int E = TF32 ? 4 : 8;         // elements per 16-byte chunk
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t I = blockIdx.x;
  const int t0 = a.ctb[I], nt = a.ctb[I + 1] - t0;
  const int b0 = a.colptr[I], nb = a.colptr[I + 1] - b0;
  const int ST = a.stages, N = a.N, NKC = a.nkc;
  const uint32_t b_bytes = (uint32_t)NKC * N * 16;
  const uint32_t stage_bytes = b_bytes + a.v_bytes + kRsBytes;
  unsigned char* bar_base = smem + (size_t)ST * stage_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(bar_base);   // full_a[ST], full_b[ST], empty[ST], done
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar_base + 8 * (3 * ST + 1));
  volatile int* abort_flag = reinterpret_cast<int*>(bar_base + 8 * (3 * ST + 1) + 4);
  auto full_a = [&](int s) { return smem_u32(&bars[s]); };
  auto full_b = [&](int s) { return smem_u32(&bars[ST + s]); };
  auto empty = [&](int s) { return smem_u32(&bars[2 * ST + s]); };
  const uint32_t done = smem_u32(&bars[3 * ST]);
  auto stage_b = [&](int s) { return smem + (size_t)s * stage_bytes; };
  auto stage_v = [&](int s) { return smem + (size_t)s * stage_bytes + b_bytes; };
  auto stage_r = [&](int s) { return smem + (size_t)s * stage_bytes + b_bytes + a.v_bytes; };
  auto meta = [&](int s) { return reinterpret_cast<TcBlk*>(stage_r(s) + kMetaOff); };
  auto fail = [&]() {
    *abort_flag = 1;
    atomicExch(a.err, 1);
  };

  if (tid == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(full_a(s), 128);
      mbar_init(full_b(s), 1);
      mbar_init(empty(s), 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    fence_proxy_async();
  }
  if (warp == 5) tmem_alloc(smem_u32(slot), a.tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;
  // column of chunk kc of M-tile mt in stage s (after the MT x N accumulator columns)
  auto a_col = [&](int s, int mt, int kc) { return (uint32_t)(MT * N + ((s * MT + mt) * NKC + kc) * 4); };

  if (warp < 4) {
    const uint32_t lanes = (uint32_t)(warp * 32) << 16;
    // the A tiles start zero
    for (int s = 0; s < ST; ++s)
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
        for (int kc = 0; kc < NKC; ++kc) tmem_st4(tmem + lanes + a_col(s, mt, kc), make_uint4(0, 0, 0, 0));
    tmem_st_wait();
    // ---------------------------------------------------------------- builders
    int dlo[kMaxStages][MT], dhi[kMaxStages][MT];   // chunks of each stage this warp left non-zero
#pragma unroll
    for (int q = 0; q < kMaxStages; ++q)
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) dlo[q][mt] = dhi[q][mt] = 0;
    for (int k = 0; k < nb; ++k) {
      const int s = k % ST, u = k / ST;
      if (u > 0 && !mbar_wait(empty(s), (u - 1) & 1, kWaitBudget)) { fail(); break; }
      if (!mbar_wait(full_b(s), u & 1, kWaitBudget)) { fail(); break; }   // record, values, row starts landed
      if (*abort_flag) break;
      const TcBlk* bm = meta(s);
      const int c0c = bm->cmin / E;
      const int nkk = 2 * ((bm->cend - c0c * E + 2 * E - 1) / (2 * E));   // chunks the MMAs read
      const int S = tc_slots(bm->W, E);
      const int32_t* R = reinterpret_cast<const int32_t*>(stage_r(s)) + (int)(bm->ro & 3);
      const uint4* V = reinterpret_cast<const uint4*>(stage_v(s));
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        const int r = mt * 128 + warp * 32 + lane;
        int lo = 0, hi = 0;
        if (r < nt) {
          lo = R[r] / E - c0c;
          hi = min(lo + S, nkk);
        }
        // the warp's range: its rows' bands and what it left non-zero in this stage
        int wlo = hi > lo ? lo : INT_MAX, whi = hi > lo ? hi : 0;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
          wlo = min(wlo, __shfl_xor_sync(0xffffffffu, wlo, o));
          whi = max(whi, __shfl_xor_sync(0xffffffffu, whi, o));
        }
        int olo = 0, ohi = 0;
#pragma unroll
        for (int q = 0; q < kMaxStages; ++q)
          if (q == s) { olo = dlo[q][mt]; ohi = dhi[q][mt]; }
        const int from = whi > 0 ? min(wlo, ohi > olo ? olo : wlo) : olo;
        const int to = max(whi, ohi);
        for (int kc = from; kc < to; ++kc) {
          const uint4 v = (kc >= lo && kc < hi) ? V[(kc - lo) * nt + r] : make_uint4(0, 0, 0, 0);
          tmem_st4(tmem + lanes + a_col(s, mt, kc), v);
        }
#pragma unroll
        for (int q = 0; q < kMaxStages; ++q)
          if (q == s) { dlo[q][mt] = whi > 0 ? wlo : 0; dhi[q][mt] = whi; }
      }
      tmem_st_wait();
      tc_fence_before();
      mbar_arrive(full_a(s));
    }
    // ---------------------------------------------------------------- epilogue
    __syncwarp();
    const bool ok = mbar_wait(done, 0, kWaitBudget);
    if (!ok) fail();
    tc_fence_after();
    const bool bad = !ok || *abort_flag;
    __syncwarp();
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      const int r = mt * 128 + warp * 32 + lane;
      for (int c = 0; c < N; c += 16) {
        float v[16];
        tmem_ld16(tmem + lanes + (uint32_t)(mt * N + c), v);
        if (r < nt) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int n = c + j;
            if (n < a.nr) {
              const double o = nb == 0 ? 0.0 : bad ? __longlong_as_double(0x7ff8000000000000LL) : (double)v[j];
              a.y[(int64_t)n * a.n_tet + t0 + r] = o;
            }
          }
        }
      }
    }
  } else if (warp == 4) {
    // ---------------------------------------------------------------- loader
    if (lane == 0) {
      prefetch_tensormap(&tmx);
      int issued = 0;
      TcBlk nxt = nb > 0 ? a.blk[b0] : TcBlk{};
      for (int k = 0; k < nb; ++k) {
        const int s = k % ST, u = k / ST;
        const TcBlk b = nxt;
        if (k + 1 < nb) nxt = a.blk[b0 + k + 1];          // the next record in flight meanwhile
        if (u > 0 && !mbar_wait(empty(s), (u - 1) & 1, kWaitBudget)) { fail(); break; }
        if (*abort_flag) break;
        *meta(s) = b;
        const int c0c = b.cmin / E;
        const int nk = (b.cend - c0c * E + 2 * E - 1) / (2 * E);
        const uint32_t v_bytes = (uint32_t)tc_slots(b.W, E) * nt * 16;
        const uint64_t rs_src = reinterpret_cast<uint64_t>(a.rs + (b.ro & ~(int64_t)3));
        const uint32_t rs_bytes = (uint32_t)(((b.ro & 3) + nt + 3) & ~3) * 4;
        mbar_arrive_expect_tx(full_b(s), (uint32_t)nk * 2 * N * 16 + v_bytes + rs_bytes);
        const uint32_t B = smem_u32(stage_b(s));
        for (int ks = 0; ks < nk; ++ks)
          tma_load_3d(B + (uint32_t)ks * 2 * N * 16, &tmx, 0, 0, c0c + 2 * ks, full_b(s));
        bulk_load(smem_u32(stage_v(s)), reinterpret_cast<uint64_t>(a.vals + b.vc[TF32 ? 1 : 0]), v_bytes, full_b(s));
        bulk_load(smem_u32(stage_r(s)), rs_src, rs_bytes, full_b(s));
        issued = k + 1;
      }
      // copies still in flight land before the CTA's shared memory is released
      for (int k = max(0, issued - ST); k < issued; ++k)
        if (!mbar_wait(full_b(k % ST), (k / ST) & 1, kWaitBudget)) fail();
    }
  } else {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = instr_desc(TF32 ? 2u : 1u, 128, N);
      for (int k = 0; k < nb; ++k) {
        const int s = k % ST, u = k / ST;
        if (!mbar_wait(full_a(s), u & 1, kWaitBudget) || !mbar_wait(full_b(s), u & 1, kWaitBudget)) {
          fail();
          break;
        }
        if (*abort_flag) break;
        tc_fence_after();
        const TcBlk* bm = meta(s);
        const int c0c = bm->cmin / E;
        const int nk = (bm->cend - c0c * E + 2 * E - 1) / (2 * E);
        const uint32_t B = smem_u32(stage_b(s));
        for (int ks = 0; ks < nk; ++ks) {
          const uint64_t bd = smem_desc(B + (uint32_t)ks * 2 * N * 16, (uint32_t)N * 16, 128);
#pragma unroll
          for (int mt = 0; mt < MT; ++mt)
            mma_ts<TF32>(tmem + (uint32_t)(mt * N), tmem + a_col(s, mt, 2 * ks), bd, idesc, (k > 0 || ks > 0) ? 1u : 0u);
        }
        mma_commit(empty(s));
      }
      mma_commit(done);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 5) {
    tc_fence_after();
    tmem_dealloc(tmem, a.tmem_cols);
  }
}

std::mutex g_tc_mu;
std::map<std::tuple<int64_t, int, int, int64_t, int, int, int>, std::pair<int, int>> g_tc_shape;   // shape -> (kind, stages)

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Block records of the operator (made once; an operator's sparsity
// structure never changes): the non-empty blocks of each test column, their
// band unions and the offsets of their chunk slots in both types.
bem_status ensure_tc_meta(const bem_operator* op, cudaStream_t s) {
  if (op->d_tc_blk) return BEM_OK;
  const bem_mesh* m = op->mesh;
  const int64_t nc = m->n_col;
  std::vector<int32_t> hbw(nc * nc);
  STBEM_CUDA(cudaMemcpyAsync(hbw.data(), op->d_bw, sizeof(int32_t) * nc * nc, cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaStreamSynchronize(s));
  std::vector<int32_t> colptr(nc + 1, 0), bI, bJ;
  std::vector<int64_t> vc16, vc32;
  int64_t o16 = 0, o32 = 0, cap16 = 0, cap32 = 0;
  for (int64_t I = 0; I < nc; ++I) {
    const int64_t nt = m->col_tet_begin[I + 1] - m->col_tet_begin[I];
    for (int64_t J = 0; J < nc; ++J) {
      const int W = hbw[I * nc + J];
      if (W <= 0) continue;
      bI.push_back((int32_t)I);
      bJ.push_back((int32_t)J);
      vc16.push_back(o16);
      vc32.push_back(o32);
      o16 += tc_slots(W, 8) * nt;
      o32 += tc_slots(W, 4) * nt;
      cap16 = std::max<int64_t>(cap16, tc_slots(W, 8) * nt * 16);
      cap32 = std::max<int64_t>(cap32, tc_slots(W, 4) * nt * 16);
    }
    colptr[I + 1] = (int32_t)bI.size();
  }
  const int64_t nb = (int64_t)bI.size();
  int32_t *d_ptr = nullptr, *d_I = nullptr, *d_J = nullptr;
  int64_t *d_v16 = nullptr, *d_v32 = nullptr;
  int* d_span = nullptr;
  void* d_blk = nullptr;
  auto cleanup = [&]() {
    cudaFree(d_I); cudaFree(d_J); cudaFree(d_v16); cudaFree(d_v32); cudaFree(d_span);
  };
  const size_t nb1 = (size_t)std::max<int64_t>(nb, 1);
  if (cudaMalloc(&d_ptr, sizeof(int32_t) * (nc + 1)) != cudaSuccess ||
      cudaMalloc(&d_blk, sizeof(TcBlk) * nb1) != cudaSuccess || cudaMalloc(&d_I, sizeof(int32_t) * nb1) != cudaSuccess ||
      cudaMalloc(&d_J, sizeof(int32_t) * nb1) != cudaSuccess || cudaMalloc(&d_v16, sizeof(int64_t) * nb1) != cudaSuccess ||
      cudaMalloc(&d_v32, sizeof(int64_t) * nb1) != cudaSuccess || cudaMalloc(&d_span, sizeof(int) * 2) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(d_ptr); cudaFree(d_blk);
    cleanup();
    set_error("out of device memory (tensor-core product tables)");
    return BEM_ERR_OUT_OF_MEMORY;
  }
  int hspan[2] = {0, 0};
  cudaMemcpyAsync(d_ptr, colptr.data(), sizeof(int32_t) * (nc + 1), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d_span, hspan, sizeof(hspan), cudaMemcpyHostToDevice, s);
  if (nb > 0) {
    cudaMemcpyAsync(d_I, bI.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_J, bJ.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_v16, vc16.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d_v32, vc32.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice, s);
    const int64_t threads = nb * 32;
    k_tc_meta<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(nb, d_I, d_J, d_v16, d_v32, nc, m->d_col_tet_begin,
                                                                op->d_bw, op->d_boff, op->d_rsoff, op->d_rs,
                                                                static_cast<TcBlk*>(d_blk), d_span);
  }
  cudaMemcpyAsync(hspan, d_span, sizeof(hspan), cudaMemcpyDeviceToHost, s);
  const cudaError_t e = cudaStreamSynchronize(s);
  cleanup();
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    cudaFree(d_ptr); cudaFree(d_blk);
    set_error(std::string("tensor-core product tables: ") + cudaGetErrorString(e));
    return BEM_ERR_CUDA;
  }
  if (!op->d_tc_err) {
    if (cudaMalloc(&op->d_tc_err, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(d_ptr); cudaFree(d_blk);
      set_error("out of device memory (tensor-core product flag)");
      return BEM_ERR_OUT_OF_MEMORY;
    }
    cudaMemsetAsync(op->d_tc_err, 0, sizeof(int), s);
  }
  op->d_tc_colptr = d_ptr;
  op->d_tc_blk = d_blk;
  op->tc_nblk = nb;
  op->tc_span[0] = hspan[0];
  op->tc_span[1] = hspan[1];
  op->tcv_len[0] = o16;
  op->tcv_len[1] = o32;
  op->tcv_cap[0] = cap16;
  op->tcv_cap[1] = cap32;
  return BEM_OK;
}

// the chunk slots of the product's type, made on first use and after a reassembly
bem_status ensure_tc_vals(const bem_operator* op, bool tf32, cudaStream_t s) {
  const int t = tf32 ? 1 : 0;
  if (op->d_tcv[t] && !op->tcv_stale[t]) return BEM_OK;
  if (!op->d_tcv[t] &&
      cudaMalloc(&op->d_tcv[t], sizeof(uint4) * (size_t)std::max<int64_t>(op->tcv_len[t], 1)) != cudaSuccess) {
    cudaGetLastError();
    op->d_tcv[t] = nullptr;
    set_error("out of device memory (tensor-core product values)");
    return BEM_ERR_OUT_OF_MEMORY;
  }
  op->tcv_stale[t] = false;
  if (op->tc_nblk == 0) return BEM_OK;
  const TcBlk* blk = static_cast<const TcBlk*>(op->d_tc_blk);
  uint4* out = static_cast<uint4*>(op->d_tcv[t]);
  const unsigned grid = (unsigned)std::min<int64_t>((op->tc_nblk * 32 + 255) / 256, 152 * 32);
  if (tf32) k_tc_pack_vals<true, float><<<grid, 256, 0, s>>>(op->tc_nblk, blk, op->d_val32, op->d_rs, out);
  else if (op->d_val32) k_tc_pack_vals<false, float><<<grid, 256, 0, s>>>(op->tc_nblk, blk, op->d_val32, op->d_rs, out);
  else k_tc_pack_vals<false, double><<<grid, 256, 0, s>>>(op->tc_nblk, blk, op->d_val, op->d_rs, out);
  STBEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

// kind 0: A tiles in shared memory (k_spmm_tc); kind 1: in tensor memory (k_spmm_tm)
template <bool TF32, int MT>
bem_status launch_tc(int kind, const TcArgs& a, const CUtensorMap& map, size_t smem, int64_t n_col, cudaStream_t s) {
  const void* kern = kind ? (const void*)k_spmm_tm<TF32, MT> : (const void*)k_spmm_tc<TF32, MT>;
  TRY_STATUS(ensure_smem_attr(kern, smem));
  if (kind) k_spmm_tm<TF32, MT><<<(unsigned)n_col, kThreads, smem, s>>>(a, map);
  else k_spmm_tc<TF32, MT><<<(unsigned)n_col, kThreads, smem, s>>>(a, map);
  STBEM_CUDA(cudaGetLastError());
  return BEM_OK;
}

}  // namespace

int64_t tc_table_bytes(const bem_operator* op) {
  int64_t b = op->d_tc_blk ? op->tc_nblk * (int64_t)sizeof(TcBlk) + (op->mesh->n_col + 1) * 4 : 0;
  for (int t = 0; t < 2; ++t)
    if (op->d_tcv[t]) b += op->tcv_len[t] * 16;
  return b;
}

bem_status op_spmm_tc(const bem_operator* op, const double* x, double* y, int nrhs, bool bf16, cudaStream_t s) {
  const bem_mesh* m = op->mesh;
  const int64_t n = m->n_tet;
  if (nrhs < 1 || nrhs > 64) {
    set_error("tensor-core product: 1..64 right-hand sides per pass");
    return BEM_ERR_INVALID_ARG;
  }
  if (!bf16 && !op->d_val32) {
    set_error("TF32 products need FP32 values (store_fp32 = 1)");
    return BEM_ERR_INVALID_ARG;
  }
  TRY_STATUS(ensure_tc_meta(op, s));
  TRY_STATUS(ensure_tc_vals(op, !bf16, s));
  auto enc = encode_fn();
  if (!enc) {
    set_error("tensor-core product: cuTensorMapEncodeTiled is not available");
    return BEM_ERR_UNSUPPORTED;
  }
  const int E = bf16 ? 8 : 4;
  const int N = std::max(16, (nrhs + 15) / 16 * 16);
  const int64_t nchunks = (n + E - 1) / E;
  TRY_STATUS(ensure_ws(op, nchunks * N * 4));   // 16 bytes per (chunk, rhs)
  void* Xc = op->d_ws;
  if (bf16) k_pack_xc<false><<<grid_for(nchunks * N * E), 256, 0, s>>>(x, n, nrhs, N, nchunks, Xc);
  else k_pack_xc<true><<<grid_for(nchunks * N * E), 256, 0, s>>>(x, n, nrhs, N, nchunks, Xc);
  STBEM_CUDA(cudaGetLastError());

  // Xc as rows of 256 bytes: {256-byte row, N / 16 rows per chunk, chunks};
  // a box of {256 bytes, N / 16, 2 chunks} is one K step of the B tile
  CUtensorMap map;
  const int inner = 256 / (bf16 ? 2 : 4);
  cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)(N / 16), (cuuint64_t)nchunks};
  cuuint64_t strides[2] = {256, (cuuint64_t)N * 16};
  cuuint32_t box[3] = {(cuuint32_t)inner, (cuuint32_t)(N / 16), 2};
  cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = enc(&map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, Xc, dims,
                         strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("tensor-core product: tensor map rejected (" + std::to_string((int)r) + ")");
    return BEM_ERR_CUDA;
  }
  const int MT = m->max_col_tets > 128 ? 2 : 1;
  const int span = std::max(op->tc_span[bf16 ? 0 : 1], 1);
  const int nkc = 2 * ((span + 2 * E - 1) / (2 * E));
  // value slots of the largest block; a multiple of 1024 bytes keeps every
  // stage's TMA tiles aligned
  const size_t v_bytes = ((size_t)op->tcv_cap[bf16 ? 0 : 1] + 1023) & ~(size_t)1023;
  // shared memory per stage: A tile (kind 0 only), B tile, value slots, row starts
  const size_t stage_b = (size_t)nkc * N * 16 + v_bytes + kRsBytes;
  const size_t stage_a = (size_t)nkc * MT * 128 * 16;
  const size_t tail = kTailBytes;
  size_t smem_max = 0;
  {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    smem_max = (size_t)v;
  }
  TcArgs a;
  a.ctb = m->d_col_tet_begin;
  a.colptr = op->d_tc_colptr;
  a.blk = static_cast<const TcBlk*>(op->d_tc_blk);
  a.vals = static_cast<const uint4*>(op->d_tcv[bf16 ? 0 : 1]);
  a.rs = op->d_rs;
  a.y = y;
  a.n_tet = n;
  a.nr = nrhs;
  a.N = N;
  a.nkc = nkc;
  a.v_bytes = (uint32_t)v_bytes;
  a.err = op->d_tc_err;
  auto pow2 = [](int c) {
    uint32_t v = 32;
    while (v < (uint32_t)c) v <<= 1;
    return v;
  };
  // tensor-memory columns: the accumulator, and for kind 1 the A tiles of every stage
  auto cols_of = [&](int kind, int st) { return kind ? MT * N + st * MT * nkc * 4 : MT * N; };
  auto fits = [&](int kind, int st) {
    const size_t smem = st * (stage_b + (kind ? 0 : stage_a)) + tail;
    return smem <= smem_max && cols_of(kind, st) <= 512;
  };
  auto launch = [&](int kind, int st) -> bem_status {
    a.stages = st;
    a.tmem_cols = pow2(cols_of(kind, st));
    const size_t smem = st * (stage_b + (kind ? 0 : stage_a)) + tail;
    if (bf16)
      return MT == 1 ? launch_tc<false, 1>(kind, a, map, smem, m->n_col, s)
                     : launch_tc<false, 2>(kind, a, map, smem, m->n_col, s);
    return MT == 1 ? launch_tc<true, 1>(kind, a, map, smem, m->n_col, s)
                   : launch_tc<true, 2>(kind, a, map, smem, m->n_col, s);
  };
  // launch shape: where the A tiles live and the pipeline depth (1 to 6
  // stages; with the stage size they fix the CTAs per SM), timed once per
  // shape in the process, then kept. Neither changes the arithmetic (every
  // CTA sums its blocks in order), so the candidates give the same bits.
  std::vector<std::pair<int, int>> cand;
  for (int kind = 0; kind < 2; ++kind)
    for (int st = 1; st <= kMaxStages; ++st)
      if (fits(kind, st)) cand.emplace_back(kind, st);
  if (cand.empty()) {
    set_error("tensor-core product: the widest block does not fit in shared or tensor memory");
    return BEM_ERR_UNSUPPORTED;
  }
  const auto key = std::make_tuple(m->n_col, m->max_col_tets, op->tc_span[bf16 ? 0 : 1], op->tcv_cap[bf16 ? 0 : 1], N,
                                   (int)bf16, op->ctx->device);
  {
    std::lock_guard<std::mutex> lk(g_tc_mu);
    auto it = g_tc_shape.find(key);
    if (it != g_tc_shape.end()) return launch(it->second.first, it->second.second);
  }
  cudaEvent_t e0, e1;
  STBEM_CUDA(cudaEventCreate(&e0));
  STBEM_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  std::pair<int, int> best_c = cand.back();
  bem_status st = BEM_OK;
  for (const auto& c : cand) {
    if ((st = launch(c.first, c.second)) != BEM_OK) break;   // warm-up
    cudaEventRecord(e0, s);
    if ((st = launch(c.first, c.second)) != BEM_OK) break;
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = BEM_ERR_CUDA;
      set_error("tensor-core product: tuning launch failed");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      best_c = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != BEM_OK) return st;
  {
    std::lock_guard<std::mutex> lk(g_tc_mu);
    g_tc_shape[key] = best_c;
  }
  return launch(best_c.first, best_c.second);
}

namespace {
// One thread waits, with the product's bounded wait, on an mbarrier that
// nothing arrives on; it records whether the wait gave up and after how many
// cycles.
__global__ void k_wait_selftest(long long budget, int* gave_up, long long* cycles) {
  __shared__ uint64_t bar;
  const uint32_t b = tc::smem_u32(&bar);
  tc::mbar_init(b, 1);
  tc::fence_proxy_async();
  const long long t0 = clock64();
  const bool ok = tc::mbar_wait(b, 0, budget);
  *cycles = clock64() - t0;
  *gave_up = ok ? 0 : 1;
}
}  // namespace

bem_status op_tc_error(const bem_operator* op, int* flag) {
  *flag = 0;
  if (!op->d_tc_err) return BEM_OK;
  STBEM_CUDA(cudaMemcpy(flag, op->d_tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  return BEM_OK;
}

}  // namespace stbem

using namespace stbem;

extern "C" bem_status bem_selftest_bounded_wait(bem_context* ctx, double* waited_ms) {
  if (!ctx) {
    set_error("bem_selftest_bounded_wait: null context");
    return BEM_ERR_INVALID_ARG;
  }
  STBEM_CUDA(cudaSetDevice(ctx->device));
  int* d_flag = nullptr;
  long long* d_cyc = nullptr;
  if (cudaMalloc(&d_flag, sizeof(int)) != cudaSuccess || cudaMalloc(&d_cyc, sizeof(long long)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(d_flag);
    set_error("out of device memory");
    return BEM_ERR_OUT_OF_MEMORY;
  }
  int dev_clock_khz = 0;
  cudaDeviceGetAttribute(&dev_clock_khz, cudaDevAttrClockRate, ctx->device);
  const long long budget = 2000000;   // clock cycles: about a millisecond
  k_wait_selftest<<<1, 1, 0, ctx->stream>>>(budget, d_flag, d_cyc);
  int flag = 0;
  long long cyc = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&cyc, d_cyc, sizeof(long long), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(d_flag);
  cudaFree(d_cyc);
  if (e != cudaSuccess) {
    set_error(std::string("bem_selftest_bounded_wait: ") + cudaGetErrorString(e));
    return BEM_ERR_CUDA;
  }
  if (waited_ms) *waited_ms = dev_clock_khz > 0 ? (double)cyc / dev_clock_khz : 0.0;
  if (flag) {
    set_error("bounded wait gave up (expected: nothing arrives on the self-test barrier)");
    return BEM_ERR_DEVICE_TIMEOUT;
  }
  return BEM_OK;
}
