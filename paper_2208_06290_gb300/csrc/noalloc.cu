// Allocation-free FP64 HODLR matvec.
//
// Some callers cannot call cudaMalloc or any other allocator at the point
// where they need A x: code running inside a CUDA-graph capture that must not
// add allocation nodes, plugin hooks of host applications that own all device
// memory, or real-time loops where allocation latency or failure is not
// acceptable. hodlr_matvec_noalloc gives them the FP64 product of
// hodlr_matvec with the same kernels, taking its scratch (the per-node
// projection partials) from a fixed array in device global memory that this
// library defines at file scope.
//
// The array is a module-scope __device__ variable: every GPU on which the
// library's module is loaded holds it (kNoAllocScratchBytes) until the
// process exits. In host code its name is only a host-side stand-in, so the
// device address is obtained once per device with cudaGetSymbolAddress while
// that device is current, at the first call on the device (do that first call
// before any stream capture). All calls share the one array and it keeps the
// last call's contents; nothing in it needs to start at zero (every partial is
// written before it is read), but calls that overlap on the GPU (other
// streams, other threads) race on it and must be serialized by the caller.
#include <mutex>

#include "hodlr_internal.cuh"

namespace hodlr {

hodlr_status matvec_core_ext(const hodlr_desc& d, const double* D, const double* U, const double* V, const double* X,
                             int64_t ldx, double* Y, int64_t ldy, int k, void* work, cudaStream_t s,
                             size_t work_bytes);
size_t matvec_scratch_bytes(const hodlr_desc& d, int k);

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchBytes / sizeof(double)];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

}  // namespace
}  // namespace hodlr

using namespace hodlr;

extern "C" hodlr_status hodlr_matvec_noalloc(const hodlr_desc* desc, const double* D, const double* U,
                                             const double* V, const double* X, int64_t ldx, double* Y, int64_t ldy,
                                             int32_t k, hodlr_stream_t stream) {
  const hodlr_status st = check_desc_ext(desc);  // the descriptor rules of every other entry point
  if (st != HODLR_OK) return st;
  if (!D || !U || !V || !X || !Y || k < 1 || ldx < desc->N || ldy < desc->N || X == Y) return HODLR_ERR_ARG;
  if (matvec_scratch_bytes(*desc, k) > kNoAllocScratchBytes) return HODLR_ERR_SCRATCH_LIMIT;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HODLR_ERR_CUDA;
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return HODLR_ERR_CUDA;
      g_noalloc_addr[dev] = p;
    }
    scratch = g_noalloc_addr[dev];
  }
  return matvec_core_ext(*desc, D, U, V, X, ldx, Y, ldy, k, scratch, reinterpret_cast<cudaStream_t>(stream),
                         kNoAllocScratchBytes);
}
