// Launch-shape autotuning of the persistent quadrature (no counterpart in the
// paper). The quadrature kernel is a persistent block queue; its one free
// launch parameter is the number of CTAs per SM it runs with (up to the
// occupancy limit of its register and shared-memory budget). Fewer CTAs give
// each more L1 and issue slots, more CTAs hide more latency; which wins
// depends on the device and on the mesh's column sizes.
//
// With tuning on (bem_context_set_tuning), the first assembly of a shape
// class times every candidate on a sample of the block queue (the first
// blocks of the dense (I, J) order; their values are rewritten by the full
// pass that follows) and keeps the fastest. A shape class is the device
// (name, SM count), the precision, m_Q^2, the rule order, the largest column
// sizes and the number of columns to within a factor of two. Choices are
// kept for the process and, with a cache path, in a text file, one line per
// class: "stbem-tune-v1 <class> <CTAs per SM>". The values do not depend on
// the launch shape (every block is computed by one CTA alone), so tuned and
// untuned assemblies give the same bits.
#include <cuda_runtime.h>

#include <algorithm>
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
    if (ls >> tag >> key >> per && tag == "stbem-tune-v1" && per >= 1 && per <= 32) g_shape[key] = per;
  }
}

void append_cache(const std::string& path, const std::string& key, int per) {
  if (path.empty()) return;
  std::ofstream f(path, std::ios::app);
  f << "stbem-tune-v1 " << key << " " << per << "\n";
}

}  // namespace

// Times launch(per_sm, end) for per_sm = occ - 2 .. occ on the sample
// [0, end) after one warm-up launch; *per = the fastest, ms[per - 1] its
// sample times (how = 1), or the class's cached choice (how = 2).
bem_status tune_launch_shape(const bem_context* ctx, const std::string& key, int occ, int64_t end,
                             const std::function<bem_status(int, int64_t)>& launch, cudaStream_t s, int* per,
                             int* how, double* ms_out) {
  std::lock_guard<std::mutex> lk(g_mu);   // one tuning at a time (and a quiet device for it)
  read_cache(ctx->tune_path);
  auto it = g_shape.find(key);
  if (it != g_shape.end()) {
    *per = std::min(it->second, occ);
    *how = 2;
    return BEM_OK;
  }
  cudaEvent_t e0, e1;
  STBEM_CUDA(cudaEventCreate(&e0));
  STBEM_CUDA(cudaEventCreate(&e1));
  bem_status st = launch(occ, end);   // warm-up
  int best = occ;
  float best_ms = 1e30f;
  for (int p = std::max(1, occ - 2); p <= occ && st == BEM_OK; ++p) {
    cudaEventRecord(e0, s);
    st = launch(p, end);
    cudaEventRecord(e1, s);
    if (st != BEM_OK) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      set_error("quadrature tuning launch failed");
      st = BEM_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms_out && p - 1 < 8) ms_out[p - 1] = ms;
    if (ms < best_ms) {
      best_ms = ms;
      best = p;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != BEM_OK) return st;
  g_shape[key] = best;
  append_cache(ctx->tune_path, key, best);
  *per = best;
  *how = 1;
  return BEM_OK;
}

bem_status choose_quad_shape(bem_operator* op, cudaStream_t s) {
  if (op->quad_per_sm > 0) return BEM_OK;
  const int occ = quad_max_per_sm(op);
  if (op->ctx->tune_mode == 0 || op->opts.matrix_free) {
    op->quad_per_sm = occ;
    op->quad_tuned = 0;
    return BEM_OK;
  }
  // sample: 1/32 of the dense block order, at least 16 test columns
  const int64_t nblk = op->mesh->n_col * op->mesh->n_col;
  const int64_t end = std::min(nblk, std::max(nblk / 32, 16 * op->mesh->n_col));
  auto launch = [&](int per, int64_t e) { return quad_launch(op, per, e, nullptr, nullptr, 0, s); };
  return tune_launch_shape(op->ctx, shape_class(op), occ, end, launch, s, &op->quad_per_sm, &op->quad_tuned,
                           op->tune_ms);
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

extern "C" bem_status bem_operator_tuning(const bem_operator* op, int* ctas_per_sm, int* tuned, double* sample_ms) {
  if (!op) {
    set_error("bem_operator_tuning: null operator");
    return BEM_ERR_INVALID_ARG;
  }
  if (ctas_per_sm) *ctas_per_sm = op->quad_per_sm;
  if (tuned) *tuned = op->quad_tuned;
  if (sample_ms)
    for (int k = 0; k < 8; ++k) sample_ms[k] = op->tune_ms[k];
  return BEM_OK;
}
