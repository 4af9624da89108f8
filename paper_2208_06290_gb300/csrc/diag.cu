// Diagnostics that are not part of the method: a register-only FP64 FMA
// probe, so that benchmarks can measure the FP64 pipe rate of the GPU they run
// on (the roofline denominator of FP64-bound kernels) instead of assuming it.
#include "hodlr_internal.cuh"

namespace hodlr {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;  // independent FMA chains per thread (covers the pipe latency)

__global__ void __launch_bounds__(kProbeThreads) fp64_fma_probe_kernel(int64_t iters, double* out) {
  double a[kProbeChains];
  const double x = 1.0 + 1e-9 * threadIdx.x, y = 1.0 - 1e-9 * blockIdx.x;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) a[c] = 1e-3 * (c + 1);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) a[c] = fma(a[c], x, y);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s += a[c];
  if (s == -1.0) out[0] = s;  // never true for these inputs; keeps the chains live
}

}  // namespace
}  // namespace hodlr

using namespace hodlr;

extern "C" hodlr_status hodlr_probe_fp64_fma(int64_t iters, int32_t blocks_per_sm, double* out,
                                             hodlr_stream_t stream, int64_t* fmas) {
  if (iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 64 || !out || !fmas) return HODLR_ERR_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HODLR_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HODLR_ERR_CUDA;
  const int64_t grid = (int64_t)sms * blocks_per_sm;
  fp64_fma_probe_kernel<<<(unsigned)grid, kProbeThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(iters, out);
  note_launches(1);
  if (cudaGetLastError() != cudaSuccess) return HODLR_ERR_CUDA;
  *fmas = grid * kProbeThreads * kProbeChains * iters;
  return HODLR_OK;
}
