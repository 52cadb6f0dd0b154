// Internal host-side structures of the library (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <functional>
#include <memory>
#include <string>
#include <vector>

#include "../../include/stbem.h"
#include "stbem_quad.cuh"

namespace stbem {

void set_error(const std::string& msg);

#define STBEM_CUDA(call)                                                                   \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      ::stbem::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));             \
      return BEM_ERR_CUDA;                                                                 \
    }                                                                                      \
  } while (0)

constexpr int MAX_COL_TETS = 192;   // panels sharing one spatial triangle
constexpr int MAX_COL_SURF = 193;   // nu_t != 0 faces over one spatial triangle
constexpr int MAX_NQ = 64;          // m_Q^2 outer points per face
#ifndef STBEM_QUAD_MIN_CTAS
#define STBEM_QUAD_MIN_CTAS 4           // CTAs per SM the quadrature's default register budget is cut for
#endif
constexpr int STBEM_QUAD_BUDGET_CTAS = STBEM_QUAD_MIN_CTAS;

// Per panel data on the device (internal panel order: by column, then time).
struct TetDev {
  int32_t lo, hi;      // global surface ids of the lower / upper face
  int32_t col;         // column (spatial triangle)
  int32_t dup;         // corner index (0..2) of the vertical edge
  double tmin, tmax;   // min / max vertex time
  double pmax;         // running max of tmax within the column (window search)
  double vt[4];        // vertex times: corner 0,1,2 lower times, then the upper time at `dup`
  double ball[5];      // 4D ball of the vertices in input order: centre (t,x,y,z), radius
};

struct SurfDev {
  int32_t col;
  int32_t pad;
  FaceGeom f;          // corner times and in-frame gradient
};

}  // namespace stbem

struct bem_context {
  int device = 0;
  cudaStream_t stream = nullptr;
  double sm_count = 0;
  int tune_mode = 0;          // 1: launch shapes timed per shape class (bem_context_set_tuning)
  std::string tune_path;      // text cache of the tuned shapes ("" = process only)
};

struct bem_mesh {
  bem_context* ctx = nullptr;
  int64_t n_tet = 0, n_col = 0, n_surf = 0;
  int max_col_tets = 0, max_col_surf = 0;
  std::vector<int32_t> perm;    // internal -> caller panel id
  std::vector<int32_t> iperm;   // caller -> internal
  std::vector<int32_t> col_tet_begin, col_surf_begin;  // [n_col+1]
  double coord_scale = 1.0;     // max |coordinate| over all vertices (FP32 filter margins)
  // device
  stbem::ColGeom* d_col = nullptr;
  int32_t* d_col_tet_begin = nullptr;
  int32_t* d_col_surf_begin = nullptr;
  stbem::SurfDev* d_surf = nullptr;
  stbem::TetDev* d_tet = nullptr;
  int32_t* d_perm = nullptr;    // internal -> caller
};

struct bem_operator {
  bem_context* ctx = nullptr;
  const bem_mesh* mesh = nullptr;
  bem_op_opts opts{};
  int mq = 3, nq = 9, n_theta = 12;
  double* d_pts = nullptr;       // [n_surf][nq][4] outer points
  float* d_ptsf = nullptr;       // the same rounded to FP32 (the sparsity filter's inputs)
  double* d_pts_trange = nullptr;// [n_surf][2] min / max time of the outer points
  int32_t* d_bw = nullptr;       // [n_col*n_col] band width per column block
  int64_t* d_bnnz = nullptr;     // [n_col*n_col] pattern entries per block
  int64_t* d_boff = nullptr;     // [n_col*n_col] value offset
  int64_t* d_rsoff = nullptr;    // [n_col*n_col] row-start offset
  int32_t* d_rs = nullptr;       // row starts (internal trial index)
  double* d_val = nullptr;       // values, per block column-major [W][R_I]
  float* d_val32 = nullptr;
  int64_t nnz = 0, nstored = 0, nblocks = 0, nrows_stored = 0;
  int64_t n_inner = 0;           // inner integrals per assembly (m_Q^2 x (test face, trial panel) pattern pairs)
  int max_bw = 0;                // widest band of any block
  double assemble_ms = 0.0;
  double phase_ms[4] = {0, 0, 0, 0};
  int quad_per_sm = 0;           // CTAs per SM of the persistent quadrature (0: not chosen yet)
  int quad_variant = 0;          // its register budget (0: 4 CTAs per SM, 1: 2 CTAs per SM)
  int quad_tuned = 0;            // 0 default shape, 1 timed here, 2 from the tuning cache
  double tune_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // sample time per candidate: index = 4 variant + CTAs per SM - 1
  unsigned long long* d_counter = nullptr;  // work counter of the persistent kernels
  // quadrature scratch
  double* d_tmp = nullptr;
  int64_t tmp_len = 0;
  // made on first use by the products (an operator is used by one host thread at a time)
  mutable float* d_ws = nullptr;        // packed operands of the FP32 / tensor-core products
  mutable int64_t ws_len = 0;
  mutable double* d_pv = nullptr;       // caller-order <-> internal-order vectors of the products
  mutable int64_t pv_len = 0;           // (stream-ordered allocation, grown on demand)
  mutable int32_t* d_tc_colptr = nullptr;  // tensor-core product: non-empty blocks per test column
  mutable void* d_tc_blk = nullptr;        // (TcBlk records, trial columns ascending)
  mutable int64_t tc_nblk = 0;
  mutable int tc_span[2] = {0, 0};         // widest band union of a block from a BF16 / TF32 chunk boundary
  mutable void* d_tcv[2] = {nullptr, nullptr};  // values as chunk slots (BF16, TF32) of the tensor-core product
  mutable int64_t tcv_len[2] = {0, 0};     // 16-byte slots of each
  mutable int64_t tcv_cap[2] = {0, 0};     // bytes of the largest block's slots
  mutable bool tcv_stale[2] = {false, false};   // the values were reassembled since the slots were made
  mutable int* d_tc_err = nullptr;         // set when a tensor-core product gave up on a wait
  // optional admission hook, called once the sparsity structure is known
  // (nstored, nrows_stored, tmp_len set) and before the value arrays are allocated
  std::function<bem_status(const bem_operator*)> admit;
};

namespace stbem {
// kernels wrappers (stbem_core.cu)
bem_status upload_gauss_tables();
bem_status mesh_device_geometry(bem_mesh* m, const double* d_sv_xyz, const int32_t* d_col_corner_sv,
                                const double* d_tet_vx, const int32_t* d_tet_info, const double* d_surf_p);
bem_status op_outer_points(bem_operator* op, cudaStream_t s);
bem_status op_pattern(bem_operator* op, cudaStream_t s);
bem_status op_quadrature(bem_operator* op, cudaStream_t s);
// register-budget variants of the quadrature kernel (1 for FP64 operators;
// 2 for mixed ones: the 4-CTA budget, and the 2-CTA budget of 255 registers)
int quad_variants(const bem_operator* op);
// most CTAs of a variant of the quadrature kernel resident per SM (shared memory and registers)
int quad_max_per_sm(const bem_operator* op, int variant);
// one persistent quadrature launch of a variant with per_sm CTAs per SM over
// the blocks [0, end) of the dense (I, J) order (assembled, or summed against mf_x)
bem_status quad_launch(const bem_operator* op, int per_sm, int64_t end, const double* mf_x, double* mf_y, int nrhs,
                       cudaStream_t s, int variant);
// the untuned shape: the 2-CTA budget where shared memory admits no more than
// 2 CTAs per SM anyway, else the 4-CTA budget; its occupancy
void default_quad_shape(const bem_operator* op, int* per_sm, int* variant);
// sets op->quad_per_sm: the context's tuning cache, a timed choice, or the default (stbem_tune.cu)
bem_status choose_quad_shape(bem_operator* op, cudaStream_t s);
// the tuner behind it: the fastest of the candidate launch codes of launch(code, end)
// over a sample [0, end) of a block queue (the code's meaning is the caller's)
bem_status tune_launch_shape(const bem_context* ctx, const std::string& key, const std::vector<int>& codes,
                             int64_t end, const std::function<bem_status(int, int64_t)>& launch, cudaStream_t s,
                             int* best_code, int* how, double* ms_out);
std::string batch_shape_class(const bem_context* ctx, int prec, int nq, int n_theta, int max_tet, int max_surf,
                              int64_t n_ops, int64_t n_blocks);
// raise a kernel's dynamic shared-memory limit to at least `bytes` (never lowers it)
bem_status ensure_smem_attr(const void* kern, size_t bytes);
// matrix-free product (internal order): the quadrature pass summed against x
bem_status op_matvec_free(const bem_operator* op, const double* x, double* y, int nrhs, cudaStream_t s);
// Layout of the vectors of a batched GMRES: K vectors of length N ([K][N]);
// entries [seg_off[s], seg_off[s+1]) of a vector belong to segment s (one
// operator of a block-diagonal batch). Each (vector, segment) is a column
// with its own Krylov process.
struct SegLayout {
  int64_t N = 0;
  int K = 1, S = 1;
  std::vector<int64_t> seg_off;   // [S+1]
};
// y = A x for all K vectors (device arrays in the [K][N] layout), enqueued on s
using MatvecFn = std::function<bem_status(const double* x, double* y, cudaStream_t s)>;
bem_status gmres_device(const SegLayout& L, const MatvecFn& mv, const double* d_b, double* d_x, double tol, int m,
                        int maxit, std::vector<int>& iters, std::vector<double>& relres, std::vector<int>& conv,
                        cudaStream_t s);
// block-diagonal product over the operators of a batch ([K][N] vectors,
// operator i owning entries [off_i, off_i + n_tet_i) of every vector)
struct BatchMatvec {
  std::vector<bem_operator*> ops;
  void* d_segs = nullptr;
  int32_t* d_cseg = nullptr;
  int32_t* d_ccol = nullptr;
  int64_t n_cta = 0, N = 0;
  int rows_pad = 32, groups = 1;
  bool fp64_values = false;
  float* d_xf = nullptr;
  int64_t xf_len = 0;
  bem_status init(const std::vector<bem_operator*>& o, cudaStream_t s);
  bem_status apply(const double* x, double* y, int K, int arith, cudaStream_t s);
  ~BatchMatvec();
};
// Cancellation of a solve run by a worker thread (bem_solve_async): the
// thread installs its request's flag; the GMRES host loops poll it between
// blocks of Arnoldi steps and return BEM_ERR_CANCELLED once it is set.
void set_thread_cancel_flag(const std::atomic<int>* flag);
bool cancel_requested();
// per-column 2-norms of a [K][N] vector (host result)
bem_status seg_norms(const SegLayout& L, const double* v, std::vector<double>& out, cudaStream_t s);
// refined solve over a layout: FP64 GMRES with mv_hi, or inner GMRES with
// mv_lo inside FP64 refinement (o->inner_dtype != FP64); info per column
bem_status gmres_solve_layout(const SegLayout& L, const MatvecFn& mv_hi, const MatvecFn& mv_lo, const double* d_b,
                              double* d_x, const bem_solve_opts* o, bem_solve_info* info, cudaStream_t s);
// operator creation with an admission hook (see bem_operator::admit)
bem_status operator_create(bem_context* ctx, const bem_mesh* mesh, const bem_op_opts* opts,
                           std::function<bem_status(const bem_operator*)> admit, bem_operator** out);
// operator object with its structure arrays allocated (nothing assembled yet)
bem_status op_structure_alloc(bem_context* ctx, const bem_mesh* mesh, const bem_op_opts* opts,
                              std::unique_ptr<bem_operator>& op);
// block offsets from the per-block band widths and counts (host arrays);
// first: set the storage sizes, call the admission hook, allocate the values
// (and the quadrature scratch when own_scratch)
bem_status op_layout(bem_operator* op, const int32_t* bw, const int64_t* bnnz, bool first, bool own_scratch,
                     cudaStream_t s);
// batched pattern and quadrature passes over several operators (one
// persistent launch each); the operators share `uscratch` for the quadrature
struct BatchDev {
  void* d_ctx = nullptr;                 // BlockCtx[S]
  int64_t* d_prefix = nullptr;           // [S+1] block prefix
  unsigned long long* d_counter = nullptr;
  double* d_uscratch = nullptr;
  int64_t uscratch_len = 0;
};
bem_status op_outer_points_all(const std::vector<bem_operator*>& ops, cudaStream_t s);
bem_status op_pattern_batch(const std::vector<bem_operator*>& ops, BatchDev& dev, cudaStream_t s);
bem_status op_quadrature_batch(const std::vector<bem_operator*>& ops, BatchDev& dev, cudaStream_t s);
int64_t quad_batch_scratch(const std::vector<bem_operator*>& ops);
size_t block_ctx_size();
// bytes held by an operator's value arrays, row starts and quadrature scratch
int64_t operator_value_bytes(const bem_operator* op);
// arithmetic of a product (values equal to BEM_DTYPE_*)
enum { MV_FP64 = 0, MV_FP32 = 1, MV_TF32 = 2, MV_BF16 = 3 };
bem_status op_matvec(const bem_operator* op, const double* x, double* y, int nrhs, int arith, cudaStream_t s);
// product workspaces of an operator (made on first use)
bem_status ensure_ws(const bem_operator* op, int64_t floats);
// grid of a grid-stride elementwise kernel over n items (256 threads per CTA)
unsigned grid_for(int64_t n);
// tensor-core product of up to 64 right-hand sides (internal order, [nrhs][n_tet])
bem_status op_spmm_tc(const bem_operator* op, const double* x, double* y, int nrhs, bool bf16, cudaStream_t s);
// 1 when a tensor-core product of the operator gave up on a wait (its output is NaN)
bem_status op_tc_error(const bem_operator* op, int* flag);
int64_t tc_table_bytes(const bem_operator* op);
bem_status op_rhs(const bem_operator* op, int kind, int nrhs, const double* d_params, double* d_b, cudaStream_t s);
// right-hand side rule for arbitrary data (points [n_surf * 4^level * ng^2][4], weights)
bem_status op_rhs_points(const bem_operator* op, int level, int ng, double* d_pts, double* d_wts, cudaStream_t s);
// b (internal order, [nrhs][n_tet]) from samples g [nrhs][n_pts]; d_S scratch [nrhs][n_surf]
bem_status op_rhs_samples(const bem_operator* op, int level, int ng, const double* d_wts, const double* d_g, int nrhs,
                          double* d_S, double* d_b, cudaStream_t s);
bem_status op_value_scan(const bem_operator* op, int64_t* nbad, double* maxabs, cudaStream_t s);
bem_status op_entries(const bem_operator* op, int64_t n, const int32_t* d_ij, double* d_out, cudaStream_t s);
bem_status op_pattern_csr(const bem_operator* op, int64_t* d_rowcount, int64_t* d_rowptr, int32_t* d_cols,
                          bool fill, cudaStream_t s, int64_t I_only = -1);
bem_status inner_potentials(int64_t n, const double* d_x4, const double* d_tets, const int32_t* d_sv, int prec,
                            int n_theta, double* d_out, cudaStream_t s);
bem_status permute(const int32_t* d_perm, const double* in, double* out, int64_t n, int nrhs, bool to_internal,
                   cudaStream_t s);
// solver (stbem_solver.cu)
bem_status gmres_solve(bem_operator* op, const double* d_b, double* d_x, int nrhs, const bem_solve_opts* o,
                       bem_solve_info* info, cudaStream_t s);
// refinement with the residual of hi_op (FP64 accumulation) and inner solves on lo_op
bem_status gmres_solve_two(const bem_operator* hi_op, bem_operator* lo_op, const double* d_b, double* d_x,
                           int nrhs, const bem_solve_opts* o, bem_solve_info* info, cudaStream_t s);
}  // namespace stbem
