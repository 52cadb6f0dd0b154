// Allocation-free matrix-vector product.
//
// bem_matvec moves x and y between the caller's panel numbering and the
// library's internal order through two temporary device vectors that it
// allocates per call. Some callers cannot let a library allocate device
// memory while they run: a serving loop or a runtime that reserves all device
// memory up front and forbids allocations afterwards, and code on a latency
// budget, where cudaMalloc/cudaFree cost time and cudaFree synchronizes the
// device. For them, bem_matvec_noalloc takes the two temporary vectors from a
// fixed array in device memory that is part of this library (file-scope
// static __device__), so the call allocates nothing.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "stbem_internal.h"

namespace {

// entries per temporary vector: n_tet * nrhs must not exceed this
constexpr int64_t kNoAllocMaxEntries = int64_t(1) << 20;

// Two vectors of kNoAllocMaxEntries doubles (16 MiB). Every GPU that loads the
// library holds this array until the process exits.
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocMaxEntries];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_dev_ptr[kMaxDevices] = {};

}  // namespace

extern "C" bem_status bem_matvec_noalloc(const bem_operator* op, const double* x_dev, double* y_dev, int32_t nrhs,
                                         void* stream) {
  using namespace stbem;
  if (!op || !x_dev || !y_dev || nrhs <= 0) {
    set_error("bem_matvec_noalloc: invalid argument");
    return BEM_ERR_INVALID_ARG;
  }
  const bem_mesh* m = op->mesh;
  const int64_t nn = m->n_tet * (int64_t)nrhs;
  if (nn > kNoAllocMaxEntries) {
    set_error("bem_matvec_noalloc: n_tet * nrhs = " + std::to_string(nn) + " exceeds the fixed scratch of " +
              std::to_string(kNoAllocMaxEntries) + " entries per vector");
    return BEM_ERR_INVALID_ARG;
  }
  const int dev = op->ctx->device;
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("bem_matvec_noalloc: device index out of range");
    return BEM_ERR_INVALID_ARG;
  }
  // the caller's current device is put back before returning
  int prev = -1;
  STBEM_CUDA(cudaGetDevice(&prev));
  if (prev != dev) STBEM_CUDA(cudaSetDevice(dev));
  struct Restore {
    int to, from;
    ~Restore() { if (to != from) cudaSetDevice(to); }
  } restore{prev, dev};
  double* base = nullptr;
  {
    // once per device, with that device current: the array's device address
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_dev_ptr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) {
        set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return BEM_ERR_CUDA;
      }
      g_dev_ptr[dev] = static_cast<double*>(p);
    }
    base = g_dev_ptr[dev];
  }
  cudaStream_t s = stream ? (cudaStream_t)stream : op->ctx->stream;
  double* xi = base;
  double* yi = base + kNoAllocMaxEntries;
  // every element of both temporaries is written before it is read: no clearing needed
  bem_status st = permute(m->d_perm, x_dev, xi, m->n_tet, nrhs, true, s);
  if (st != BEM_OK) return st;
  st = op_matvec(op, xi, yi, nrhs, false, s);
  if (st != BEM_OK) return st;
  return permute(m->d_perm, yi, y_dev, m->n_tet, nrhs, false, s);
}
