// Launch-shape autotuning of the persistent quadrature (no counterpart in the
// paper). The quadrature kernel is a persistent block queue; its free launch
// parameters are the number of CTAs per SM it runs with (up to the occupancy
// limit of its register and shared-memory budget) and, in mixed precision,
// the register budget it was compiled for (128 registers for 4 CTAs per SM,
// with spills; or 255 for 2, without). Fewer CTAs give each more L1 and issue
// slots, more CTAs hide more latency; which wins depends on the device and
// on the mesh's column sizes (the shared memory a CTA needs grows with them).
//
// With tuning on (bem_context_set_tuning), the first assembly of a shape
// class times every candidate on a sample of the block queue (the first
// blocks of the dense (I, J) order; their values are rewritten by the full
// pass that follows) and keeps the fastest. A shape class is the device
// (name, SM count), the precision, m_Q^2, the rule order, the largest column
// sizes and the number of columns to within a factor of two. Choices are
// kept for the process and, with a cache path, in a text file, one line per
// class: "stbem-tune-v2 <class> <code>", code = 4 x budget variant + CTAs per
// SM - 1 (variant 0: the 4-CTA budget, 1: the 2-CTA budget; a batch's code
// is its CTAs per SM with the 4-CTA budget). The values do not depend on
// the launch shape (every block is computed by one CTA alone), so tuned and
// untuned assemblies give the same bits.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>
#include <cmath>
#include <fstream>
#include <functional>
#include <map>
#include <mutex>
#include <set>
#include <sstream>
#include <string>

#include "stbem_internal.h"

namespace stbem {
namespace {

std::mutex g_mu;
std::map<std::string, int> g_shape;      // class -> CTAs per SM
std::set<std::string> g_read;            // cache files already read

std::string shape_class(const bem_operator* op) {
  cudaDeviceProp p;
  std::string name = "device";
  if (cudaGetDeviceProperties(&p, op->ctx->device) == cudaSuccess) name = p.name;
  for (char& c : name)
    if (c == ' ' || c == '|') c = '_';
  const bem_mesh* m = op->mesh;
  const int cols_log2 = (int)std::floor(std::log2((double)std::max<int64_t>(m->n_col, 1)));
  std::ostringstream k;
  k << name << "|sm" << (int)op->ctx->sm_count << "|p" << op->opts.precision << "|q" << op->nq << "|t"
    << op->n_theta << "|r" << m->max_col_tets << "|f" << m->max_col_surf << "|c" << cols_log2;
  return k.str();
}

}  // namespace

std::string batch_shape_class(const bem_context* ctx, int prec, int nq, int n_theta, int max_tet, int max_surf,
                              int64_t n_ops, int64_t n_blocks) {
  cudaDeviceProp p;
  std::string name = "device";
  if (cudaGetDeviceProperties(&p, ctx->device) == cudaSuccess) name = p.name;
  for (char& c : name)
    if (c == ' ' || c == '|') c = '_';
  std::ostringstream k;
  k << name << "|sm" << (int)ctx->sm_count << "|batch|p" << prec << "|q" << nq << "|t" << n_theta << "|r" << max_tet
    << "|f" << max_surf << "|o" << (int)std::floor(std::log2((double)std::max<int64_t>(n_ops, 1))) << "|b"
    << (int)std::floor(std::log2((double)std::max<int64_t>(n_blocks, 1)));
  return k.str();
}

namespace {

void read_cache(const std::string& path) {
  if (path.empty() || g_read.count(path)) return;
  g_read.insert(path);
  std::ifstream f(path);
  std::string tag, key;
  int per = 0;
  std::string line;
  while (std::getline(f, line)) {
    std::istringstream ls(line);
    if (ls >> tag >> key >> per && tag == "stbem-tune-v2" && per >= 0 && per < 64) g_shape[key] = per;
  }
}

void append_cache(const std::string& path, const std::string& key, int per) {
  if (path.empty()) return;
  std::ofstream f(path, std::ios::app);
  f << "stbem-tune-v2 " << key << " " << per << "\n";
}

}  // namespace

// Times launch(code, end) for every candidate code on the sample [0, end)
// after one warm-up launch of the first; *best = the fastest code,
// ms_out[code] its sample time (how = 1), or the class's cached code (how = 2).
bem_status tune_launch_shape(const bem_context* ctx, const std::string& key, const std::vector<int>& codes,
                             int64_t end, const std::function<bem_status(int, int64_t)>& launch, cudaStream_t s,
                             int* best_code, int* how, double* ms_out) {
  std::lock_guard<std::mutex> lk(g_mu);   // one tuning at a time (and a quiet device for it)
  read_cache(ctx->tune_path);
  auto it = g_shape.find(key);
  if (it != g_shape.end() && std::find(codes.begin(), codes.end(), it->second) != codes.end()) {
    *best_code = it->second;
    *how = 2;
    return BEM_OK;
  }
  cudaEvent_t e0, e1;
  STBEM_CUDA(cudaEventCreate(&e0));
  STBEM_CUDA(cudaEventCreate(&e1));
  bem_status st = launch(codes.back(), end);   // warm-up
  int best = codes.back();
  float best_ms = 1e30f;
  for (int c : codes) {
    if (st != BEM_OK) break;
    cudaEventRecord(e0, s);
    st = launch(c, end);
    cudaEventRecord(e1, s);
    if (st != BEM_OK) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      set_error("quadrature tuning launch failed");
      st = BEM_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms_out && c >= 0 && c < 8) ms_out[c] = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != BEM_OK) return st;
  g_shape[key] = best;
  append_cache(ctx->tune_path, key, best);
  *best_code = best;
  *how = 1;
  return BEM_OK;
}

void default_quad_shape(const bem_operator* op, int* per_sm, int* variant) {
  const int occ0 = quad_max_per_sm(op, 0);
  if (quad_variants(op) > 1 && occ0 <= 2) {
    *variant = 1;
    *per_sm = quad_max_per_sm(op, 1);
  } else {
    *variant = 0;
    *per_sm = occ0;
  }
}

// Candidates: each register-budget variant at its occupancy and the one or
// two CTA counts below it; code = 4 variant + CTAs per SM - 1.
bem_status choose_quad_shape(bem_operator* op, cudaStream_t s) {
  if (op->quad_per_sm > 0) return BEM_OK;
  if (op->ctx->tune_mode == 0 || op->opts.matrix_free) {
    default_quad_shape(op, &op->quad_per_sm, &op->quad_variant);
    op->quad_tuned = 0;
    return BEM_OK;
  }
  std::vector<int> codes;
  for (int v = 0; v < quad_variants(op); ++v) {
    const int occ = std::min(quad_max_per_sm(op, v), 4);
    for (int per = std::max(1, occ - 2); per <= occ; ++per) codes.push_back(4 * v + per - 1);
  }
  // sample: 1/32 of the dense block order, at least 16 test columns
  const int64_t nblk = op->mesh->n_col * op->mesh->n_col;
  const int64_t end = std::min(nblk, std::max(nblk / 32, 16 * op->mesh->n_col));
  auto launch = [&](int code, int64_t e) { return quad_launch(op, code % 4 + 1, e, nullptr, nullptr, 0, s, code / 4); };
  int best = 0;
  const bem_status st = tune_launch_shape(op->ctx, shape_class(op), codes, end, launch, s, &best, &op->quad_tuned,
                                          op->tune_ms);
  if (st != BEM_OK) return st;
  op->quad_per_sm = best % 4 + 1;
  op->quad_variant = best / 4;
  return BEM_OK;
}

}  // namespace stbem

using namespace stbem;

extern "C" bem_status bem_context_set_tuning(bem_context* ctx, int mode, const char* cache_path) {
  if (!ctx || (mode != 0 && mode != 1)) {
    set_error("bem_context_set_tuning: invalid argument");
    return BEM_ERR_INVALID_ARG;
  }
  ctx->tune_mode = mode;
  ctx->tune_path = cache_path ? cache_path : "";
  return BEM_OK;
}

extern "C" bem_status bem_operator_tuning(const bem_operator* op, int* ctas_per_sm, int* budget_ctas, int* tuned,
                                          double* sample_ms) {
  if (!op) {
    set_error("bem_operator_tuning: null operator");
    return BEM_ERR_INVALID_ARG;
  }
  if (ctas_per_sm) *ctas_per_sm = op->quad_per_sm;
  if (budget_ctas) *budget_ctas = op->quad_variant ? 2 : STBEM_QUAD_BUDGET_CTAS;
  if (tuned) *tuned = op->quad_tuned;
  if (sample_ms)
    for (int k = 0; k < 8; ++k) sample_ms[k] = op->tune_ms[k];
  return BEM_OK;
}
