// Continuous batching of Dirichlet solves (eq. df_ind on each request's own
// mesh). Host-side runtime: a FIFO of requests, max_slots worker threads each
// owning a CUDA stream, and an HBM reservation pool that admits a request once
// its operator's footprint is known (after the sparsity pattern, before the
// values are allocated). A request's kernels run on its slot's stream, so the
// assembly and solver kernels of different requests overlap on the device;
// no kernel depends on another request's data, and every reduction has a
// fixed order, so a request's result is the same alone and in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <set>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "stbem_internal.h"

using namespace stbem;
using Clock = std::chrono::steady_clock;


#define SRV_TRY(x)                    \
  do {                                \
    bem_status st_ = (x);             \
    if (st_ != BEM_OK) return st_;    \
  } while (0)

namespace {

struct Job {
  uint64_t ticket = 0;
  int64_t n_sv = 0, n_stv = 0, n_tet = 0;
  std::vector<double> sv, stv_t, params;
  std::vector<int32_t> stv_sv, tets;
  int32_t kind = 0, nrhs = 1;
  Clock::time_point t_submit, t_start;
};

struct Done {
  bem_completion c{};
  std::vector<double> w;
};

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

// per-request device vectors, allocated and released on the slot's stream
template <typename T>
struct DBuf {
  T* p = nullptr;
  cudaStream_t st = nullptr;
  ~DBuf() { if (p) cudaFreeAsync(p, st); }
  bem_status alloc(int64_t n, cudaStream_t s) {
    st = s;
    if (cudaMallocAsync((void**)&p, sizeof(T) * std::max<int64_t>(n, 1), s) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      set_error("out of device memory");
      return BEM_ERR_OUT_OF_MEMORY;
    }
    return BEM_OK;
  }
};

// A resident operator, keyed by its request's mesh arrays.
struct CacheEntry {
  uint64_t key = 0;
  std::vector<double> sv, stv_t;
  std::vector<int32_t> stv_sv, tets;
  bem_mesh* mesh = nullptr;
  bem_operator* op = nullptr;
  int64_t bytes = 0;     // pool bytes it holds (values, row starts, scratch, mesh and structure)
  bool busy = false;     // in use by a request (operators are used by one stream at a time)
  uint64_t last = 0;     // LRU clock
};

uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) { h ^= c[i]; h *= 1099511628211ull; }
  return h;
}

uint64_t job_key(const Job& J) {
  uint64_t h = 1469598103934665603ull;
  h = fnv1a(h, J.sv.data(), J.sv.size() * sizeof(double));
  h = fnv1a(h, J.stv_sv.data(), J.stv_sv.size() * sizeof(int32_t));
  h = fnv1a(h, J.stv_t.data(), J.stv_t.size() * sizeof(double));
  return fnv1a(h, J.tets.data(), J.tets.size() * sizeof(int32_t));
}

bool same_mesh(const CacheEntry& e, const Job& J) {
  return e.sv == J.sv && e.stv_sv == J.stv_sv && e.stv_t == J.stv_t && e.tets == J.tets;
}

}  // namespace

struct bem_server {
  bem_context* ctx = nullptr;
  bem_server_opts o{};
  std::vector<bem_context*> slot_ctx;
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv_work, cv_mem, cv_done, cv_cache;
  std::deque<std::unique_ptr<Job>> queue;
  std::deque<uint64_t> mem_fifo;              // requests waiting for a reservation, in order
  std::deque<std::unique_ptr<Done>> ready;    // completed, not yet polled
  std::map<uint64_t, std::unique_ptr<Done>> held;  // polled, not yet released
  int64_t pool = 0, slot_share = 0, in_use = 0, peak_in_use = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  int64_t submitted = 0, completed = 0, failed = 0, running = 0;
  int peak_running = 0;
  bool any_submit = false;
  Clock::time_point t_first, t_last;
  std::vector<double> lat;
  // resident operators (cache_operators = 1)
  std::vector<std::unique_ptr<CacheEntry>> cache;
  std::set<uint64_t> building;   // meshes whose operator a slot is assembling now
  uint64_t use_clock = 0;
  int64_t cache_hits = 0, cached_bytes = 0;
};

namespace {

void destroy_entry(std::unique_ptr<CacheEntry> e) {
  if (!e) return;
  if (e->op) bem_operator_destroy(e->op);
  if (e->mesh) bem_mesh_destroy(e->mesh);
}

// HBM reservation in arrival order; a request that can never fit fails. The
// request at the head of the queue evicts idle resident operators (least
// recently used first) when they hold the room it needs.
bem_status acquire(bem_server* S, uint64_t ticket, int64_t bytes) {
  std::unique_lock<std::mutex> lk(S->mu);
  if (bytes > S->pool) {
    set_error("request needs " + std::to_string(bytes) + " bytes of HBM, more than the server's pool of " +
              std::to_string(S->pool));
    return BEM_ERR_OUT_OF_MEMORY;
  }
  S->mem_fifo.push_back(ticket);
  for (;;) {
    if (S->mem_fifo.front() == ticket && S->in_use + bytes <= S->pool) break;
    if (S->mem_fifo.front() == ticket) {
      int victim = -1;
      for (int k = 0; k < (int)S->cache.size(); ++k)
        if (!S->cache[k]->busy && (victim < 0 || S->cache[k]->last < S->cache[victim]->last)) victim = k;
      if (victim >= 0) {
        std::unique_ptr<CacheEntry> e = std::move(S->cache[victim]);
        S->cache.erase(S->cache.begin() + victim);
        S->in_use -= e->bytes;
        S->cached_bytes -= e->bytes;
        lk.unlock();
        destroy_entry(std::move(e));
        lk.lock();
        continue;
      }
    }
    S->cv_mem.wait(lk);
  }
  S->mem_fifo.pop_front();
  S->in_use += bytes;
  S->peak_in_use = std::max(S->peak_in_use, S->in_use);
  ++S->running;
  S->peak_running = std::max<int>(S->peak_running, (int)S->running);
  S->cv_mem.notify_all();
  return BEM_OK;
}

// device bytes of a mesh and of an operator's sparsity structure (the slot's share)
int64_t structure_bytes(const bem_mesh* m) {
  const int64_t nb = m->n_col * m->n_col;
  return m->n_tet * (int64_t)(sizeof(TetDev) + 4 + 16 * 8) + m->n_col * (int64_t)(sizeof(ColGeom) + 8) +
         m->n_surf * (int64_t)(sizeof(SurfDev) + (MAX_NQ * 4 + 2) * 8 + MAX_NQ * 4 * 4) + nb * (4 + 8 + 8 + 8);
}

// operator values + solver workspace for nrhs right-hand sides
int64_t admission_bytes(const bem_operator* op, const bem_server_opts& o, int nrhs) {
  const int64_t n = op->mesh->n_tet;
  int64_t b = operator_value_bytes(op);
  b += n * (int64_t)nrhs * 8 * (o.restart + 1 + 8);  // Krylov basis, b, x, r, w, dx, Ax, permutations
  if (o.inner_dtype == BEM_DTYPE_TF32 || o.inner_dtype == BEM_DTYPE_BF16)
    b += (n + 1) * (int64_t)std::min(nrhs, 64) * 8 * 2;
  if (o.inner_dtype == BEM_DTYPE_FP32) b += n * (int64_t)nrhs * 4;
  // chunk slots of the tensor-core product: at most two 16-byte slots per block row beyond the values
  if (o.inner_dtype == BEM_DTYPE_TF32) b += op->nstored * 4 + op->nrows_stored * 32;
  if (o.inner_dtype == BEM_DTYPE_BF16) b += op->nstored * 2 + op->nrows_stored * 32;
  return b;
}

// Right-hand side, solve and density of a request on an assembled operator
// (device vectors stream-ordered on the slot's stream s).
bem_status solve_job(bem_server* S, cudaStream_t s, bem_operator* op, const Job& J, Done& D) {
  const bem_mesh* mesh = op->mesh;
  const int nrhs = J.nrhs;
  const int64_t n = mesh->n_tet, nn = n * nrhs;
  DBuf<double> dp, db, dx, dw;
  SRV_TRY(db.alloc(nn, s));
  SRV_TRY(dx.alloc(nn, s));
  SRV_TRY(dw.alloc(nn, s));
  if (J.kind == BEM_DATA_PULSE) {
    SRV_TRY(dp.alloc(5 * nrhs, s));
    STBEM_CUDA(cudaMemcpyAsync(dp.p, J.params.data(), sizeof(double) * 5 * nrhs, cudaMemcpyHostToDevice, s));
  }
  SRV_TRY(op_rhs(op, J.kind, nrhs, dp.p, db.p, s));
  bem_solve_opts so{S->o.tol, S->o.restart, S->o.maxit, S->o.inner_dtype, S->o.max_refine};
  std::vector<bem_solve_info> info(nrhs);
  bem_status st = gmres_solve(op, db.p, dx.p, nrhs, &so, info.data(), s);
  if (st != BEM_OK && st != BEM_ERR_NOT_CONVERGED) return st;
  SRV_TRY(permute(mesh->d_perm, dx.p, dw.p, n, nrhs, false, s));
  D.w.resize(nn);
  STBEM_CUDA(cudaMemcpyAsync(D.w.data(), dw.p, sizeof(double) * nn, cudaMemcpyDeviceToHost, s));
  STBEM_CUDA(cudaStreamSynchronize(s));
  int it = 0;
  double rr = 0.0;
  for (auto& i : info) {
    it = std::max(it, i.iterations);
    rr = std::max(rr, i.rel_residual);
  }
  D.c.iterations = it;
  D.c.refinements = info.empty() ? 0 : info[0].refinements;
  D.c.rel_residual = rr;
  return st;
}

// returns the request's reservation to the pool (moving `keep` bytes of it,
// plus `extra` bytes from the slot's share, into the operator cache)
void release(bem_server* S, int64_t reserved, int64_t keep_in_pool) {
  std::lock_guard<std::mutex> lk(S->mu);
  if (reserved > 0) --S->running;
  S->in_use += keep_in_pool - reserved;
}

bem_status run_job(bem_server* S, bem_context* cx, const Job& J, Done& D, int64_t& reserved) {
  cudaStream_t s = cx->stream;
  const int nrhs = J.nrhs;
  const bool caching = S->o.cache_operators != 0;
  const uint64_t key = caching ? job_key(J) : 0;
  // a resident operator on the same mesh; a request whose mesh is in use by
  // another request, or being assembled by one, waits for it instead of
  // assembling a second copy
  CacheEntry* hit = nullptr;
  bool builder = false;
  if (caching) {
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
      bool present = false;
      for (auto& e : S->cache)
        if (e->key == key && same_mesh(*e, J)) {
          present = true;
          if (!e->busy) {
            e->busy = true;
            e->last = ++S->use_clock;
            hit = e.get();
          }
          break;
        }
      if (hit) break;
      if (!present && !S->building.count(key)) {
        S->building.insert(key);
        builder = true;
        break;
      }
      S->cv_cache.wait(lk);
    }
  }
  // the assembling request clears its mark on every way out (after keeping the operator)
  struct BuildMark {
    bem_server* S;
    uint64_t key;
    bool on;
    ~BuildMark() {
      if (!on) return;
      {
        std::lock_guard<std::mutex> lk(S->mu);
        S->building.erase(key);
      }
      S->cv_cache.notify_all();
    }
  } mark{S, key, builder};
  if (hit) {
    const int64_t need = admission_bytes(hit->op, S->o, nrhs) - operator_value_bytes(hit->op);
    bem_status st = acquire(S, J.ticket, need);
    if (st == BEM_OK) {
      reserved = need;
      st = solve_job(S, s, hit->op, J, D);
      release(S, reserved, 0);
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      hit->busy = false;
      if (st == BEM_OK || st == BEM_ERR_NOT_CONVERGED) ++S->cache_hits;
    }
    S->cv_mem.notify_all();
    S->cv_cache.notify_all();
    D.c.cache_hit = 1;
    return st;
  }
  bem_mesh* mesh = nullptr;
  bem_status st = bem_mesh_create(cx, J.n_sv, J.sv.data(), J.n_stv, J.stv_sv.data(), J.stv_t.data(), J.n_tet,
                                  J.tets.data(), &mesh);
  if (st != BEM_OK) return st;
  std::unique_ptr<bem_mesh, void (*)(bem_mesh*)> mesh_guard(mesh, bem_mesh_destroy);
  const int64_t sbytes = structure_bytes(mesh);
  if (sbytes > S->slot_share) {
    set_error("mesh and sparsity structure exceed the slot's share of the HBM budget");
    return BEM_ERR_OUT_OF_MEMORY;
  }
  bem_op_opts oo{};
  oo.precision = S->o.precision;
  oo.m_q = 3;
  oo.n_theta = 0;
  oo.store_fp32 = (S->o.inner_dtype == BEM_DTYPE_FP32 || S->o.inner_dtype == BEM_DTYPE_TF32) ? 1 : 0;
  bem_operator* op = nullptr;
  const uint64_t ticket = J.ticket;
  bem_server_opts so_srv = S->o;
  st = operator_create(cx, mesh, &oo, [&, ticket, nrhs](const bem_operator* o2) -> bem_status {
        const int64_t need = admission_bytes(o2, so_srv, nrhs);
        bem_status a = acquire(S, ticket, need);
        if (a == BEM_OK) reserved = need;
        return a;
      }, &op);
  if (st != BEM_OK) {
    if (reserved > 0) release(S, reserved, 0);
    return st;
  }
  std::unique_ptr<bem_operator, void (*)(bem_operator*)> op_guard(op, bem_operator_destroy);
  st = solve_job(S, s, op, J, D);
  if (!caching || (st != BEM_OK && st != BEM_ERR_NOT_CONVERGED)) {
    release(S, reserved, 0);
    return st;
  }
  // keep the operator resident if the pool has room for it beside the others
  const int64_t keep = operator_value_bytes(op) + sbytes + op->ws_len * (int64_t)sizeof(float) +
                       op->pv_len * (int64_t)sizeof(double) + tc_table_bytes(op);
  bool kept = false;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    bool have = false;   // another request on this mesh built and kept it meanwhile
    for (auto& e : S->cache) have = have || (e->key == key && same_mesh(*e, J));
    if (!have && S->in_use - reserved + keep <= S->pool) {
      std::unique_ptr<CacheEntry> e(new CacheEntry());
      e->key = key;
      e->sv = J.sv; e->stv_sv = J.stv_sv; e->stv_t = J.stv_t; e->tets = J.tets;
      e->mesh = mesh; e->op = op;
      e->bytes = keep;
      e->last = ++S->use_clock;
      S->cache.push_back(std::move(e));
      S->cached_bytes += keep;
      kept = true;
    }
  }
  if (kept) {
    op_guard.release();
    mesh_guard.release();
  }
  release(S, reserved, kept ? keep : 0);
  S->cv_mem.notify_all();
  return st;
}

void worker(bem_server* S, int slot) {
  bem_context* cx = S->slot_ctx[slot];
  cudaSetDevice(cx->device);
  for (;;) {
    std::unique_ptr<Job> J;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
      if (S->queue.empty()) return;
      J = std::move(S->queue.front());
      S->queue.pop_front();
    }
    J->t_start = Clock::now();
    std::unique_ptr<Done> D(new Done());
    D->c.ticket = J->ticket;
    D->c.nrhs = J->nrhs;
    D->c.n_tet = J->n_tet;
    int64_t reserved = 0;
    bem_status st = run_job(S, cx, *J, *D, reserved);
    const Clock::time_point t_end = Clock::now();
    D->c.status = st;
    D->c.queue_ms = ms_between(J->t_submit, J->t_start);
    D->c.latency_ms = ms_between(J->t_submit, t_end);
    D->c.reserved_bytes = reserved;
    if (st != BEM_OK && st != BEM_ERR_NOT_CONVERGED) D->w.clear();
    D->c.w = D->w.empty() ? nullptr : D->w.data();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      if (st == BEM_OK) {
        ++S->completed;
        S->lat.push_back(D->c.latency_ms);
        S->t_last = t_end;
      } else {
        ++S->failed;
      }
      S->ready.push_back(std::move(D));
    }
    S->cv_mem.notify_all();
    S->cv_done.notify_all();
  }
}

}  // namespace

extern "C" {

bem_status bem_server_create(bem_context* ctx, const bem_server_opts* opts, bem_server** out) {
  if (!ctx || !opts || !out) { set_error("bem_server_create: invalid argument"); return BEM_ERR_INVALID_ARG; }
  *out = nullptr;
  const bem_server_opts& o = *opts;
  if (o.max_slots < 1 || o.max_slots > 16 || (o.precision != BEM_PREC_FP64 && o.precision != BEM_PREC_MIXED) ||
      o.inner_dtype < BEM_DTYPE_FP64 || o.inner_dtype > BEM_DTYPE_BF16 || o.restart < 1 || o.restart > 200 ||
      o.maxit < 1 || !(o.tol > 0) || o.hbm_budget < 0 || (o.cache_operators != 0 && o.cache_operators != 1)) {
    set_error("bem_server_create: bad options");
    return BEM_ERR_INVALID_ARG;
  }
  STBEM_CUDA(cudaSetDevice(ctx->device));
  std::unique_ptr<bem_server> S(new bem_server());
  S->ctx = ctx;
  S->o = o;
  int64_t budget = o.hbm_budget;
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    STBEM_CUDA(cudaMemGetInfo(&fr, &tot));
    budget = (int64_t)(0.9 * (double)fr);
  }
  S->slot_share = std::max<int64_t>(budget / (10 * (int64_t)o.max_slots), (int64_t)64 << 20);
  S->pool = budget - S->slot_share * o.max_slots;
  if (S->pool <= 0) {
    set_error("bem_server_create: hbm_budget leaves no room beyond the slots' shares (64 MiB each at least)");
    return BEM_ERR_INVALID_ARG;
  }
  for (int k = 0; k < o.max_slots; ++k) {
    bem_context* c = nullptr;
    bem_status st = bem_context_create(ctx->device, &c);
    if (st != BEM_OK) {
      for (auto* q : S->slot_ctx) bem_context_destroy(q);
      return st;
    }
    c->tune_mode = ctx->tune_mode;   // slots assemble with the server context's tuning
    c->tune_path = ctx->tune_path;
    S->slot_ctx.push_back(c);
  }
  for (int k = 0; k < o.max_slots; ++k) S->workers.emplace_back(worker, S.get(), k);
  *out = S.release();
  return BEM_OK;
}

bem_status bem_server_submit(bem_server* S, const bem_job* j, uint64_t* ticket) {
  if (!S || !j || !ticket || !j->sv_xyz || !j->stv_sv || !j->stv_t || !j->tets || j->n_sv <= 0 || j->n_stv <= 0 ||
      j->n_tet <= 0 || j->nrhs <= 0 || (j->data_kind != BEM_DATA_SIN2_UNIFORM && j->data_kind != BEM_DATA_PULSE) ||
      (j->data_kind == BEM_DATA_PULSE && !j->params)) {
    set_error("bem_server_submit: invalid argument");
    return BEM_ERR_INVALID_ARG;
  }
  std::unique_ptr<Job> J(new Job());
  J->n_sv = j->n_sv; J->n_stv = j->n_stv; J->n_tet = j->n_tet;
  J->sv.assign(j->sv_xyz, j->sv_xyz + 3 * j->n_sv);
  J->stv_sv.assign(j->stv_sv, j->stv_sv + j->n_stv);
  J->stv_t.assign(j->stv_t, j->stv_t + j->n_stv);
  J->tets.assign(j->tets, j->tets + 4 * j->n_tet);
  J->kind = j->data_kind;
  J->nrhs = j->nrhs;
  if (j->params) J->params.assign(j->params, j->params + 5 * j->nrhs);
  J->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    J->ticket = S->next_ticket++;
    *ticket = J->ticket;
    if (!S->any_submit) { S->any_submit = true; S->t_first = J->t_submit; }
    ++S->submitted;
    S->queue.push_back(std::move(J));
  }
  S->cv_work.notify_one();
  return BEM_OK;
}

bem_status bem_server_poll(bem_server* S, bem_completion* out, int32_t max, int32_t* n_out, int64_t timeout_ms) {
  if (!S || !n_out || max < 0 || (max > 0 && !out)) { set_error("bem_server_poll: invalid argument"); return BEM_ERR_INVALID_ARG; }
  std::unique_lock<std::mutex> lk(S->mu);
  if (S->ready.empty() && timeout_ms > 0)
    S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return !S->ready.empty(); });
  int k = 0;
  while (k < max && !S->ready.empty()) {
    std::unique_ptr<Done> D = std::move(S->ready.front());
    S->ready.pop_front();
    out[k++] = D->c;
    const uint64_t t = D->c.ticket;
    S->held[t] = std::move(D);
  }
  *n_out = k;
  return BEM_OK;
}

bem_status bem_server_release(bem_server* S, uint64_t ticket) {
  if (!S) { set_error("null server"); return BEM_ERR_INVALID_ARG; }
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->held.find(ticket);
  if (it == S->held.end()) { set_error("unknown or unpolled ticket"); return BEM_ERR_INVALID_ARG; }
  S->held.erase(it);
  return BEM_OK;
}

bem_status bem_server_stats_get(const bem_server* Sc, bem_server_stats* out) {
  if (!Sc || !out) { set_error("bem_server_stats_get: invalid argument"); return BEM_ERR_INVALID_ARG; }
  bem_server* S = const_cast<bem_server*>(Sc);
  std::lock_guard<std::mutex> lk(S->mu);
  bem_server_stats r{};
  r.submitted = S->submitted;
  r.completed = S->completed;
  r.failed = S->failed;
  r.queued = (int64_t)S->queue.size();
  r.running = S->running;
  r.peak_running = S->peak_running;
  r.peak_reserved_bytes = S->peak_in_use;
  r.cache_hits = S->cache_hits;
  r.cached_operators = (int64_t)S->cache.size();
  r.cached_bytes = S->cached_bytes;
  if (!S->lat.empty()) {
    std::vector<double> v = S->lat;
    std::sort(v.begin(), v.end());
    auto rank = [&](double p) {
      size_t k = (size_t)std::ceil(p * v.size());
      return v[std::min(v.size() - 1, k > 0 ? k - 1 : 0)];
    };
    r.p50_ms = rank(0.50);
    r.p99_ms = rank(0.99);
    double sum = 0.0;
    for (double x : v) sum += x;
    r.mean_ms = sum / v.size();
    r.max_ms = v.back();
    const double span = ms_between(S->t_first, S->t_last) / 1e3;
    r.solves_per_s = span > 0 ? S->completed / span : 0.0;
  }
  *out = r;
  return BEM_OK;
}

void bem_server_destroy(bem_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto& e : S->cache) destroy_entry(std::move(e));
  S->cache.clear();
  for (auto* c : S->slot_ctx) bem_context_destroy(c);
  delete S;
}

}  // extern "C"
