/*
 * stbem.h - C ABI of the GB300 space-time Galerkin BEM library for the
 * retarded single layer of the 3D wave equation (Poelz & Schanz, "On the
 * space-time discretization of variational retarded potential boundary
 * integral equations").
 *
 * Problem (Sec. 2, eq. pde/ic/bc and Table bie, indirect method): given the
 * lateral boundary Sigma = (0,T) x Gamma, meshed by flat space-time
 * tetrahedra ("panels", Sec. 3), and Dirichlet data g, find the density
 * w_h in S_h^0 (one value per panel, Def. st_be) with
 *     b_V(w_h, v_h) = b_I(g, v_h)   for all v_h in S_h^0      (eq. df_ind),
 * where b_A(w, v_h) = -sum_sigma int_{d sigma} nu_{d sigma,t} v_h A w dS
 * (eq. int_bform), V is the retarded single layer operator (eq. slp) and the
 * face integrals use the composite midpoint rule of Fig. int_tri_mid.
 *
 * Conventions for every call:
 *   - Every call returns a bem_status; no C++ exception crosses the ABI.
 *     bem_last_error() gives a thread-local description of the last failure.
 *   - Pointers are host pointers unless a name says "dev" or the call takes a
 *     stream; device pointers must be on the context's device.
 *   - Inputs are copied; the caller keeps ownership of its arrays. Outputs are
 *     caller-allocated. Handles are opaque and released by their destroy call.
 *   - Panels, matrix rows/columns and vector entries use the caller's panel
 *     numbering (the order of `tets`); multi-vector arrays are column-major
 *     [n_tet x nrhs] (entry (i, r) at i + n_tet * r).
 *   - All computation runs in CUDA kernels on the GPU; there is no CPU path.
 *     A call made without a usable GPU returns BEM_ERR_CUDA.
 */
#ifndef STBEM_H
#define STBEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BEM_OK = 0,
  BEM_ERR_INVALID_ARG = 1,   /* null pointer, negative size, unknown enum */
  BEM_ERR_OUT_OF_MEMORY = 2, /* device or host allocation failed */
  BEM_ERR_CUDA = 3,          /* a CUDA runtime call failed (no GPU, launch error) */
  BEM_ERR_NOT_CONVERGED = 4, /* solver stopped at maxit; best iterate returned */
  BEM_ERR_DEVICE_TIMEOUT = 5,/* a bounded device wait gave up */
  BEM_ERR_UNSUPPORTED = 6,   /* option or mesh shape outside what is built */
  BEM_ERR_BAD_MESH = 7,      /* mesh fails validation (see bem_mesh_create) */
  BEM_ERR_INTERNAL = 8,
  BEM_ERR_CANCELLED = 9      /* an asynchronous solve was cancelled (bem_request_cancel) */
} bem_status;

typedef struct bem_context bem_context;
typedef struct bem_mesh bem_mesh;
typedef struct bem_operator bem_operator;

/* Precision of the panel-pair quadrature.
 *  FP64 : every step in double precision.
 *  MIXED: light-cone / panel intersection geometry (distances, cone-function
 *         values at vertices, crossing points) in double; the conic-arc
 *         quadrature and the closed-form edge terms in single precision. */
enum { BEM_PREC_FP64 = 0, BEM_PREC_MIXED = 1 };

/* Arithmetic of products with the assembled operator:
 * FP64  FP64 accumulation (of FP64 values, or of FP32 values for MIXED operators);
 * FP32  FP32 values, x rounded to FP32, FP32 accumulation;
 * TF32  tensor cores: FP32 values and x rounded to TF32, FP32 accumulation;
 * BF16  tensor cores: values and x rounded to BF16, FP32 accumulation. */
enum { BEM_DTYPE_FP64 = 0, BEM_DTYPE_FP32 = 1, BEM_DTYPE_TF32 = 2, BEM_DTYPE_BF16 = 3 };

/* Trial space of the density (Def. st_be, Sec. 3): P0 = S_h^0, piecewise
 * constant per panel (the space of eq. df_ind, built); P1 = V_h^1, continuous
 * piecewise linear in space-time (not built: BEM_ERR_UNSUPPORTED). */
enum { BEM_TRIAL_P0 = 0, BEM_TRIAL_P1 = 1 };

/* Dirichlet data families (evaluated at space-time points (t, x)):
 *  BEM_DATA_SIN2_UNIFORM: g = sin^2(pi t / 2) for 0 < t < 2, else 0
 *                         (params ignored);
 *  BEM_DATA_PULSE       : g = exp(-((t - <x, d> - c) / w)^2), params per
 *                         right-hand side: (d0, d1, d2, c, w). */
enum { BEM_DATA_SIN2_UNIFORM = 0, BEM_DATA_PULSE = 1 };

/* ------------------------------------------------------------------ */
/* Context                                                              */
/* ------------------------------------------------------------------ */

/* Binds CUDA device `device` (usually 0) and creates the streams the library
 * uses. Fails with BEM_ERR_CUDA when no device is usable. */
bem_status bem_context_create(int device, bem_context** out);
void bem_context_destroy(bem_context* ctx);
/* Thread-local text of the last failure in this thread ("" if none). */
const char* bem_last_error(void);
const char* bem_version(void);

/* Measured FMA throughput of the context's device at its present clocks, in
 * TFLOP/s (2 flops per FMA lane): FP32 (the larger of scalar and paired
 * FMAs) and FP64. Diagnostics with no counterpart in the paper: the
 * light-cone quadrature is bound by these two pipes, and these rates are the
 * denominators of its roofline. Register-resident FMA chains on every SM,
 * each kernel timed with CUDA events at >= 50 ms per launch (about 1 s in
 * all); synchronizes the context stream. */
bem_status bem_alu_peaks(bem_context* ctx, double* fp32_tflops, double* fp64_tflops);

/* Launch-shape autotuning of the persistent quadrature (no counterpart in the
 * paper): the number of CTAs per SM it runs with. mode 0 (default): the
 * occupancy limit of the build. mode 1: the first assembly of every shape
 * class (device, precision, m_Q^2, rule order, largest column sizes, number
 * of columns to within a factor 2) on this context times each candidate on
 * 1/32 of the block queue and keeps the fastest; choices are kept for the
 * process and, when cache_path is not NULL, read from and appended to that
 * text file. Values do not depend on the shape (bit-identical either way).
 * Matrix-free operators keep the default. Operators take the context's mode
 * when they are assembled. */
bem_status bem_context_set_tuning(bem_context* ctx, int mode, const char* cache_path);

/* Self-test of the bounded device waits (no counterpart in the paper): one
 * thread waits, with the clock budget of the tensor-core product's mbarrier
 * waits cut to about 2e6 cycles, on a barrier that nothing completes. Returns
 * BEM_ERR_DEVICE_TIMEOUT with waited_ms (may be NULL) = the time waited, and
 * the context stays usable; any other status is a failure of the mechanism. */
bem_status bem_selftest_bounded_wait(bem_context* ctx, double* waited_ms);

/* ------------------------------------------------------------------ */
/* Space-time mesh of Sigma (Sec. 3: Sigma_N of open tetrahedra)        */
/* ------------------------------------------------------------------ */

/* General space-time tetrahedral mesh.
 *   sv_xyz [n_sv][3]  spatial vertices (points of Gamma's triangulation)
 *   stv_sv [n_stv]    spatial vertex of each space-time vertex
 *   stv_t  [n_stv]    time of each space-time vertex
 *   tets   [n_tet][4] space-time vertex ids of each panel
 * Each panel must be flat in Gamma_K x R for a flat spatial triangle K: its
 * four vertices lie over the three corners of K, two of them over the same
 * spatial vertex (a vertical edge) with different times; K must be
 * non-degenerate. The two faces containing the vertical edge have
 * nu_{F,t} = 0 (decided on vertex ids, never on floating point) and drop out
 * of eq. int_bform; the other two faces are graphs tau = P(y) over K.
 * Violations return BEM_ERR_BAD_MESH. At most 192 panels may share one
 * spatial triangle (BEM_ERR_UNSUPPORTED beyond). */
bem_status bem_mesh_create(bem_context* ctx, int64_t n_sv, const double* sv_xyz, int64_t n_stv,
                           const int32_t* stv_sv, const double* stv_t, int64_t n_tet, const int32_t* tets,
                           bem_mesh** out);

/* Prism mesh convenience builder: triangles tri [n_tri][3] of Gamma, per
 * spatial vertex the time nodes time_nodes [n_sv][n_slabs+1] (increasing).
 * Each prism K x [t_n, t_{n+1}] is split into three panels by the sorted
 * vertex-id rule (vertices a<b<c): {a_n,b_n,c_n,a_{n+1}}, {b_n,c_n,a_{n+1},b_{n+1}},
 * {c_n,a_{n+1},b_{n+1},c_{n+1}}; panel (k, n, s) gets number (k*n_slabs+n)*3+s. */
bem_status bem_mesh_create_prisms(bem_context* ctx, int64_t n_sv, const double* sv_xyz, int64_t n_tri,
                                  const int32_t* tri, int32_t n_slabs, const double* time_nodes,
                                  bem_mesh** out);

/* Sizes: panels, spatial triangles ("columns"), distinct nu_t != 0 faces. */
bem_status bem_mesh_info(const bem_mesh* mesh, int64_t* n_tet, int64_t* n_columns, int64_t* n_surfaces);
void bem_mesh_destroy(bem_mesh* mesh);

/* ------------------------------------------------------------------ */
/* Operator: the Galerkin matrix A_ij = b_V(1_{sigma_j}, 1_{sigma_i})    */
/* ------------------------------------------------------------------ */

typedef struct {
  int32_t precision; /* BEM_PREC_FP64 or BEM_PREC_MIXED */
  int32_t m_q;       /* midpoint-rule subdivision m_Q (Fig. int_tri_mid); 1..8, paper uses 3 */
  int32_t n_theta;   /* cap on Gauss nodes per conic-arc piece (4..32); 0 = default (32 FP64, 16 MIXED).
                        The count per piece is chosen from the distance of the integrand's nearest
                        complex pole to reach 1e-15 (FP64) or 1e-7 (MIXED) relative accuracy. */
  int32_t store_fp32;/* FP64 operators: 1 also keeps an FP32 copy of the values for low-precision
                        matvecs. MIXED operators always store FP32 values only (their accuracy). */
  int32_t matrix_free;/* 1: no values are stored; every product re-runs the quadrature with the
                        entries summed against x on the fly (the dot product fused into the
                        quadrature pass); export_dense / entries are then unsupported. */
  int32_t trial_space;/* BEM_TRIAL_P0 (0, the default); BEM_TRIAL_P1 returns BEM_ERR_UNSUPPORTED */
} bem_op_opts;

/* Assembles the sparse Galerkin matrix on the device.
 *   A_ij = -sum_{F in faces(sigma_i), nu_{F,t} != 0} nu_{F,t} |F|/m_Q^2
 *          * sum_q V 1_{sigma_j}(x_{F,q})                 (eq. int_bform, Fig. int_tri_mid)
 * with the inner value V 1_sigma(x) of eq. tk_para (exact up to the conic-arc
 * rule). Entry (i,j) is in the sparsity pattern when some outer point x_{F,q}
 * of panel i can see panel j on its backward light cone: causality
 * (Def. choice_r), the strong Huygens principle (the panel is not strictly
 * inside the cone) and the ball bound of Theorem phi_xi_sphere; entries
 * outside the pattern are exactly 0.0. The pattern decisions are made in
 * FP64 with the operation order of the published contract (bit-exact).
 * Returns BEM_ERR_INTERNAL if any assembled value is not finite. */
bem_status bem_operator_create(bem_context* ctx, const bem_mesh* mesh, const bem_op_opts* opts,
                               bem_operator** out);

/* nnz_pattern: pattern entries; stored_values: values kept (band padding
 * included); n_blocks: stored (column, column) blocks; assemble_ms: device
 * time of the last assembly. Any pointer may be NULL. */
bem_status bem_operator_stats(const bem_operator* op, int64_t* nnz_pattern, int64_t* stored_values,
                              int64_t* n_blocks, double* assemble_ms);

/* Algorithmic work of one assembly: inner_integrals = m_Q^2 x the number of
 * (test face with nu_t != 0, trial panel) pairs in the sparsity pattern, i.e.
 * the values V 1_{sigma_j}(x_{F,q}) of eq. int_bform the quadrature evaluates
 * (a face shared by two test panels counted once). Counted by the pattern pass. */
bem_status bem_operator_work(const bem_operator* op, int64_t* inner_integrals);

/* The quadrature's launch shape: CTAs per SM, the CTAs per SM its register
 * budget was compiled for (4: 128 registers; 2: 255, mixed precision only),
 * how it was chosen (0 default, 1 timed in this assembly, 2 taken from the
 * tuning cache) and, when timed, the sample time in ms of each candidate
 * (index = 4 x (budget == 2) + CTAs per SM - 1; 0 where not timed). Untuned,
 * the 2-CTA budget is taken where shared memory admits no more than 2 CTAs
 * per SM anyway. Any pointer may be NULL; sample_ms has 8 entries. */
bem_status bem_operator_tuning(const bem_operator* op, int* ctas_per_sm, int* budget_ctas, int* tuned,
                               double* sample_ms);

/* Scans the stored values on the device: number of non-finite values (NaN,
 * Inf) and the largest magnitude. A healthy operator has n_nonfinite = 0.
 * Returns BEM_ERR_DEVICE_TIMEOUT (outputs still set) when a TF32 / BF16
 * product of the operator gave up waiting for its own pipeline (every wait
 * in that kernel is bounded); that product's output was set to NaN. */
bem_status bem_operator_check(const bem_operator* op, int64_t* n_nonfinite, double* max_abs);

/* Device time of the last assembly by phase (CUDA events on the assembly
 * stream): ms[0] outer points, ms[1] sparsity pattern pass, ms[2] block
 * offsets (host scan), ms[3] quadrature + assembly pass. */
bem_status bem_operator_timings(const bem_operator* op, double* ms);

/* Re-runs pattern + quadrature + assembly on the existing operator (same
 * mesh and options) on `stream` (NULL: the context stream). Used to time
 * assembly passes; the values are overwritten with identical results. */
bem_status bem_operator_reassemble(bem_operator* op, void* stream);

/* Pattern rows in the caller's numbering, CSR with ascending columns.
 * rowptr [n_tet+1] (int64), cols [nnz_pattern]. */
bem_status bem_operator_export_pattern(const bem_operator* op, int64_t* rowptr, int32_t* cols);

/* Pattern of selected rows (caller numbering): counts[k] = entries of row
 * rows[k]; cols[k*cap ...] its first min(counts[k], cap) columns, ascending.
 * Cost scales with the number of distinct spatial triangles of the rows, not
 * with the mesh: meant for checks on large meshes. */
bem_status bem_operator_pattern_rows(const bem_operator* op, int64_t n, const int32_t* rows, int64_t cap,
                                     int64_t* counts, int32_t* cols);

/* Dense matrix (row-major [n_tet][n_tet]); for small meshes (n_tet <= 20000). */
bem_status bem_operator_export_dense(const bem_operator* op, double* A);

/* Values A_ij for a list of pairs ij [n][2] (caller numbering). Pairs
 * outside the pattern give exactly 0.0. */
bem_status bem_operator_entries(const bem_operator* op, int64_t n, const int32_t* ij, double* out);

void bem_operator_destroy(bem_operator* op);

/* ------------------------------------------------------------------ */
/* Right-hand side b_i = b_I(g, 1_{sigma_i}) = -sum_F nu_{F,t} int_F g dS */
/* (eq. int_bform with A = Id, the problem statement of Sec. 2).        */
/* A face F of panel i with nu_{F,t} != 0 is a graph tau = P(y) over the  */
/* panel's spatial triangle K, and nu_{F,t} |F| dS = -+ dA(y) on the     */
/* lower / upper face, so b_i = int_K g(P_lo(y), y) - g(P_hi(y), y) dA.  */
/* ------------------------------------------------------------------ */

/* Built-in data families: params [nrhs][5] for BEM_DATA_PULSE (NULL for
 * SIN2_UNIFORM); b host [n_tet x nrhs] column-major. Rule per face: K split
 * into 4^k congruent triangles (k from the data's length scale), each with a
 * Duffy-collapsed 8 x 8 Gauss-Legendre rule. */
bem_status bem_rhs(const bem_operator* op, int32_t kind, int32_t nrhs, const double* params, double* b);

/* Quadrature points of the right-hand side for arbitrary Dirichlet data g:
 * the caller evaluates g at the points and passes the samples to
 * bem_rhs_from_samples. Points belong to the distinct nu_t != 0 faces of the
 * mesh ("surfaces", bem_mesh_info's n_surfaces); each face's spatial triangle
 * K is split into 4^level congruent triangles (level 0..4), each carrying a
 * Duffy-collapsed n_gauss x n_gauss Gauss-Legendre rule (n_gauss 1..16), so
 * n_pts = n_surfaces * 4^level * n_gauss^2. pts_txyz [n_pts][4] receives the
 * space-time points (t, x, y, z) = (P(y), y) and w [n_pts] the weights of
 * the projected measure dA(y) (their sum over one face is |K|; the sign
 * -nu_{F,t} is applied per panel by bem_rhs_from_samples). Call with
 * pts_txyz = w = NULL to get n_pts only. Host arrays. */
bem_status bem_rhs_points(const bem_operator* op, int32_t level, int32_t n_gauss, int64_t* n_pts, double* pts_txyz,
                          double* w);

/* b [n_tet x nrhs] (column-major, caller panel order) from samples g
 * [nrhs][n_pts] of the data at the points of bem_rhs_points with the same
 * level and n_gauss: per face S_F = sum_q w_q g(x_q) in a fixed order (FP64),
 * then b_i = S_{F_lo(i)} - S_{F_hi(i)}. Host arrays; computed on the GPU. */
bem_status bem_rhs_from_samples(const bem_operator* op, int32_t level, int32_t n_gauss, const double* g,
                                int32_t nrhs, double* b);

/* ------------------------------------------------------------------ */
/* Matrix-vector products                                               */
/* ------------------------------------------------------------------ */

/* y_dev = A x_dev for nrhs column-major vectors in FP64 (device pointers),
 * enqueued on `stream` (a cudaStream_t; NULL = context stream); returns
 * without synchronizing. The caller/internal reordering uses a per-operator
 * workspace, allocated stream-ordered (cudaMallocAsync) on the first call that
 * needs more room and kept until the operator is destroyed: products of one
 * operator must not overlap on the GPU (one stream, or ordered streams). */
bem_status bem_matvec(const bem_operator* op, const double* x_dev, double* y_dev, int32_t nrhs, void* stream);

/* y_dev = A x_dev in the arithmetic `dtype` (BEM_DTYPE_*), same layout as
 * bem_matvec. TF32 and BF16 run the block matvec on the 5th-generation tensor
 * cores (tcgen05.mma, FP32 accumulation in tensor memory) for up to 64
 * right-hand sides per pass (the values are read once per pass); FP32 and
 * TF32 need the FP32 values (MIXED operators, or store_fp32 = 1). On first
 * use the TF32 / BF16 products make the operator's block records and a copy
 * of its values cut into 16-byte chunk slots in their type (1.1-1.25 x the
 * value bytes, kept with the operator and remade after a reassembly); the
 * products keep packed operands in a per-operator workspace; the first
 * TF32 / BF16 product of a mesh shape times the candidate launch shapes once
 * and keeps the fastest for the process (so these first calls synchronize
 * the stream). Otherwise stream-ordered like bem_matvec: no allocation once
 * the workspaces have grown to the call's size, no synchronization. */
bem_status bem_matvec_dtype(const bem_operator* op, const double* x_dev, double* y_dev, int32_t nrhs,
                            int32_t dtype, void* stream);

/* Allocation-free y_dev = A x_dev (no counterpart in the paper: it exists for
 * callers that cannot let a library allocate device memory while they run,
 * such as a serving loop or runtime that reserves all device memory up front,
 * or code on a latency budget where cudaMalloc/cudaFree cost time and
 * cudaFree synchronizes the device). Same arguments and result as bem_matvec,
 * but the two temporary vectors of the caller/internal reordering come from a
 * fixed array compiled into the library (2 x 2^20 doubles, 16 MiB, held on
 * every GPU that loads the library until exit), so n_tet * nrhs must not
 * exceed 1,048,576 (BEM_ERR_INVALID_ARG otherwise). It calls no allocator.
 * The first call on a device looks up the array's device address (once per
 * device); make that first call before any stream capture. The call is
 * enqueued on `stream` and returns without synchronizing; the calling thread's
 * current device is the same after the call as before it. All calls share the
 * array: calls whose work overlaps on the GPU (other streams, other threads)
 * race on it and must be ordered by the caller. Matrix-free operators run
 * their quadrature pass with the operator's own scratch, allocated when the
 * operator was created. */
bem_status bem_matvec_noalloc(const bem_operator* op, const double* x_dev, double* y_dev, int32_t nrhs, void* stream);

/* ------------------------------------------------------------------ */
/* Solve eq. df_ind (the paper names no linear solver: restarted GMRES)  */
/* ------------------------------------------------------------------ */

typedef struct {
  double tol;          /* relative residual ||b - A w|| / ||b|| target */
  int32_t restart;     /* GMRES restart length m (1..200) */
  int32_t maxit;       /* max total inner iterations per right-hand side */
  int32_t inner_dtype; /* BEM_DTYPE_FP64, or FP32 / TF32 / BF16 inner solves with FP64 refinement */
  int32_t max_refine;  /* outer refinement steps when inner_dtype != FP64 */
} bem_solve_opts;

typedef struct {
  int32_t iterations;  /* total GMRES iterations (all refinement steps) */
  int32_t refinements; /* outer refinement steps taken */
  int32_t converged;   /* 1 if tol was met */
  int32_t reserved;
  double rel_residual; /* final FP64 relative residual */
  double solve_ms;     /* wall time of the solve on the device */
} bem_solve_info;

/* Host arrays b, w [n_tet x nrhs]; info [nrhs] may be NULL. Zero initial
 * guess. Returns BEM_ERR_NOT_CONVERGED (with the best iterate in w) when a
 * right-hand side misses tol. */
bem_status bem_solve(bem_operator* op, const double* b, double* w, int32_t nrhs, const bem_solve_opts* opts,
                     bem_solve_info* info);

/* Iterative refinement with an FP64-accurate residual (precision pattern of
 * the reduced-precision form): solves op_hi w = b, where the outer residual
 * r = b - A_hi w is formed with op_hi's values in FP64 (an FP64 operator, or
 * a matrix-free FP64 one) and the corrections come from GMRES on op_lo (a
 * MIXED operator) in opts->inner_dtype (FP32, TF32 or BF16). The refinement
 * converges to op_hi's solution, so the FP32 quadrature error of op_lo limits
 * only the speed of convergence, not the accuracy. Both operators must be
 * built on the same mesh handle. Host arrays as bem_solve; info [nrhs]. */
bem_status bem_solve_refined(const bem_operator* op_hi, bem_operator* op_lo, const double* b, double* w,
                             int32_t nrhs, const bem_solve_opts* opts, bem_solve_info* info);

/* Same on device arrays, enqueued on `stream`; blocks until done. */
bem_status bem_solve_device(bem_operator* op, const double* b_dev, double* w_dev, int32_t nrhs,
                            const bem_solve_opts* opts, bem_solve_info* info, void* stream);

/* Asynchronous solve: bem_solve_device run by a worker thread of the library
 * on `stream` (NULL = context stream), returned as a request handle at once.
 * The GMRES host loop polls a cancellation flag between its blocks of Arnoldi
 * steps (each block one CUDA-graph launch) and between refinement steps. Until
 * the request has completed, the caller must not use `op`, b_dev or w_dev. */
typedef struct bem_request bem_request;
bem_status bem_solve_async(bem_operator* op, const double* b_dev, double* w_dev, int32_t nrhs,
                           const bem_solve_opts* opts, void* stream, bem_request** out);
/* Waits at most timeout_ns (>= 0; 0 polls) for the request. Returns
 * BEM_ERR_DEVICE_TIMEOUT while it is still running (the request stays valid:
 * wait again, cancel or destroy it), else the solve's own status, with info
 * [nrhs] (may be NULL) filled. Never blocks longer than timeout_ns plus
 * scheduling delay. */
bem_status bem_request_wait(bem_request* req, int64_t timeout_ns, bem_solve_info* info);
/* Asks a running solve to stop at its next poll; it then completes with
 * BEM_ERR_CANCELLED and w_dev holds the iterate reached. */
bem_status bem_request_cancel(bem_request* req);
/* Cancels the solve if it is still running, waits for the worker to stop
 * (at most one block of Arnoldi steps) and frees the request. */
void bem_request_destroy(bem_request* req);

/* ------------------------------------------------------------------ */
/* Kernel-level entry: inner integral for arbitrary (point, panel) pairs */
/* ------------------------------------------------------------------ */

/* out[k] = V 1_{sigma_k}(x_k) = (1/4pi) int_{K_k} 1[(t - |x-y|, y) in sigma_k] / |x-y| dA
 * (eq. slp with the delta integrated, i.e. T_{k_1} of eq. tk_para), for host
 * arrays x4 [n][4] = (t,x,y,z), tets [n][4][4] vertex coordinates (t,x,y,z),
 * tet_sv [n][4] spatial-vertex ids (equal ids mark the vertical edge).
 * precision and n_theta as in bem_op_opts. */
bem_status bem_inner_potentials(bem_context* ctx, int64_t n, const double* x4, const double* tets,
                                const int32_t* tet_sv, int32_t precision, int32_t n_theta, double* out);

/* ------------------------------------------------------------------ */
/* Batches of small scatterers (no counterpart in the paper: many         */
/* independent problems of eq. df_ind solved together)                  */
/* ------------------------------------------------------------------ */

/* Assembles the operators of n meshes (all on ctx's device, opts as for
 * bem_operator_create, one precision for all) with one persistent launch per
 * pass over the blocks of every operator. The meshes must outlive the batch. */
typedef struct bem_batch bem_batch;
bem_status bem_batch_create(bem_context* ctx, int32_t n, const bem_mesh* const* meshes, const bem_op_opts* opts,
                            bem_batch** out);
bem_status bem_batch_stats(const bem_batch* batch, int32_t* n_ops, int64_t* n_tet_total, int64_t* nnz,
                           double* assemble_ms);
/* Solves every operator's problem for its own right-hand sides: nrhs[i]
 * pulses for operator i (params: the [nrhs[i]][5] rows of all operators
 * concatenated; NULL for SIN2_UNIFORM). The block-diagonal system runs as one
 * set of GMRES launches (each (scatterer, right-hand side) an independent
 * Krylov column; blocks of Arnoldi steps captured as CUDA graphs, the active
 * columns checked between graph launches); opts->inner_dtype FP64 or FP32
 * (then FP64 refinement). w (host): the [nrhs[i]][n_tet_i] densities of the
 * operators concatenated, caller panel order; info: one per right-hand side
 * in the same order (may be NULL). */
bem_status bem_batch_solve(bem_batch* batch, int32_t data_kind, const int32_t* nrhs, const double* params,
                           const bem_solve_opts* opts, double* w, bem_solve_info* info);
void bem_batch_destroy(bem_batch* batch);

/* ------------------------------------------------------------------ */
/* Serving: continuous batching of Dirichlet solves (no counterpart in    */
/* the paper; each request is the problem of eq. df_ind on its own mesh) */
/* ------------------------------------------------------------------ */

/* A server owns max_slots worker slots, each with its own CUDA stream on the
 * context's device. Requests queue in arrival order; a free slot takes the
 * next request, uploads its mesh, builds the sparsity structure, and is then
 * admitted by HBM footprint: the bytes of the operator's values, row starts,
 * quadrature scratch and solver workspace are reserved against a pool of
 * hbm_budget minus the slots' shares (max(hbm_budget / (10 max_slots),
 * 64 MiB) each, for a request's mesh and sparsity structure); reservations
 * are granted in arrival order, a request waits in its slot until its
 * reservation fits, and a request that can never fit (in the pool or in its
 * slot's share) completes with BEM_ERR_OUT_OF_MEMORY. Slots run
 * concurrently, so the kernels of different requests overlap on the device;
 * every request's arithmetic is the same alone and in a mix (its reductions
 * have a fixed order), so its result does not depend on the other requests.
 * Device memory of a request (right-hand side, solution, GMRES workspace) is
 * allocated and released stream-ordered on its slot's stream, so one
 * request's release does not stall the others. With cache_operators = 1 the
 * assembled operators stay resident (see bem_server_opts). */
typedef struct bem_server bem_server;

typedef struct {
  int64_t hbm_budget;    /* bytes the server may hold on the device (0: 90% of free memory) */
  int32_t max_slots;     /* concurrent requests (1..16) */
  int32_t precision;     /* BEM_PREC_FP64 or BEM_PREC_MIXED */
  int32_t inner_dtype;   /* bem_solve_opts.inner_dtype (BEM_DTYPE_FP64 for the plain FP64 path) */
  int32_t restart, maxit, max_refine;
  double tol;            /* relative residual target of every solve */
  int32_t cache_operators;/* 1: keep each assembled operator (mesh, sparsity, values) resident after its
                            request, keyed by the request's mesh arrays; a later request on the same mesh
                            reuses it and reserves only its solver workspace. Cached operators hold pool
                            bytes and are evicted least recently used when an admission needs the room. */
  int32_t reserved0;
} bem_server_opts;

typedef struct {         /* one request: a space-time mesh (as bem_mesh_create) and its data */
  int64_t n_sv;
  const double* sv_xyz;
  int64_t n_stv;
  const int32_t* stv_sv;
  const double* stv_t;
  int64_t n_tet;
  const int32_t* tets;
  int32_t data_kind;     /* BEM_DATA_* */
  int32_t nrhs;
  const double* params;  /* [nrhs][5] for BEM_DATA_PULSE, else NULL */
} bem_job;

typedef struct {
  uint64_t ticket;
  int32_t status;        /* bem_status of the request */
  int32_t nrhs;
  int64_t n_tet;
  const double* w;       /* [nrhs][n_tet] densities (caller order), owned by the server
                            until bem_server_release(ticket); NULL on failure */
  int32_t iterations;    /* largest GMRES iteration count over the right-hand sides */
  int32_t refinements;
  double rel_residual;   /* largest final relative residual */
  double queue_ms;       /* submit -> taken by a slot */
  double latency_ms;     /* submit -> completed */
  int64_t reserved_bytes;/* HBM reserved at admission */
  int32_t cache_hit;     /* 1: the request reused a resident operator (no assembly) */
  int32_t reserved0;
} bem_completion;

typedef struct {
  int64_t submitted, completed, failed, queued, running;
  int32_t peak_running;  /* most requests admitted at once */
  int32_t reserved;
  int64_t peak_reserved_bytes;
  double solves_per_s;   /* completed / (last completion - first submission) */
  double p50_ms, p99_ms, mean_ms, max_ms;  /* latency over completed requests */
  int64_t cache_hits;    /* requests served by a resident operator */
  int64_t cached_operators, cached_bytes;  /* operators resident now and the pool bytes they hold */
} bem_server_stats;

/* Inputs of bem_server_submit are copied; the call never blocks on the GPU. */
bem_status bem_server_create(bem_context* ctx, const bem_server_opts* opts, bem_server** out);
bem_status bem_server_submit(bem_server* srv, const bem_job* job, uint64_t* ticket);
/* Up to max completions not returned before; waits up to timeout_ms (0: no
 * wait) for at least one. */
bem_status bem_server_poll(bem_server* srv, bem_completion* out, int32_t max, int32_t* n_out, int64_t timeout_ms);
bem_status bem_server_release(bem_server* srv, uint64_t ticket);
bem_status bem_server_stats_get(const bem_server* srv, bem_server_stats* out);
/* Finishes the queued and running requests, then frees everything. */
void bem_server_destroy(bem_server* srv);

/* ------------------------------------------------------------------ */
/* Lit-panel search of Sec. 3.3 (host only, no device or context): a    */
/* binary cluster tree over the panels (Def. bct) with a bounding ball  */
/* per cluster, and the search ApproximateLitLeaves (Algorithm          */
/* lit_leaves) with the ball test of Theorem phi_xi_sphere. It returns  */
/* X_N(x), a superset of the panels whose support the backward light    */
/* cone of x meets. The GPU path does not use it (it searches column    */
/* windows with the same ball test per panel); it serves the            */
/* cardinality study of Sec. 4.1.                                      */
/* ------------------------------------------------------------------ */
typedef struct bem_cluster_tree bem_cluster_tree;

/* Panels as in bem_mesh_create_tets: vertices vert_txyz [n_vert][4]
 * (t, x, y, z), panels tets [n_tet][4] (vertex ids). Leaves hold at most
 * n_min >= 1 panels. Clusters split at the median of the panel centroids
 * along the coordinate of largest extent; balls by Ritter's approximate
 * bounding sphere in R^4 over the cluster's panel vertices. */
bem_status bem_cluster_tree_create(int64_t n_vert, const double* vert_txyz, int64_t n_tet, const int32_t* tets,
                                   int32_t n_min, bem_cluster_tree** out);
/* Nodes, leaves and depth of the tree. Any pointer may be NULL. */
bem_status bem_cluster_tree_info(const bem_cluster_tree* tree, int64_t* n_nodes, int64_t* n_leaves, int32_t* depth);
/* X_N(x) for the point x_txyz [4]: the panels of the leaves the search
 * keeps, in tree order, into panels [cap]; n_panels = their number (also
 * when it exceeds cap, which returns BEM_ERR_INVALID_ARG), n_visited (may
 * be NULL) = clusters whose ball was tested. */
bem_status bem_cluster_tree_query(const bem_cluster_tree* tree, const double* x_txyz, int64_t cap, int32_t* panels,
                                  int64_t* n_panels, int64_t* n_visited);
void bem_cluster_tree_destroy(bem_cluster_tree* tree);

#ifdef __cplusplus
}
#endif

#endif /* STBEM_H */
