// Column-vector kernels for the solves and the refined solvers: copies with
// precision change, axpby, and deterministic FP64 dot products (fixed-order
// two-stage reductions, so results do not depend on scheduling).
#include <type_traits>

#include "hodlr_internal.cuh"

namespace hodlr {

template <typename TD, typename TS>
__global__ void copy_cols_kernel(int64_t N, int k, const TS* __restrict__ src, int64_t lds, TD* __restrict__ dst,
                                 int64_t ldd) {
  const int j = blockIdx.y;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    dst[(int64_t)j * ldd + i] = conv<TD>(src[(int64_t)j * lds + i]);
}

static unsigned grid_for(int64_t N) {
  int64_t b = (N + 255) / 256;
  return (unsigned)(b < 4096 ? b : 4096);
}

// FP64 -> BF16 column copy, eight elements per thread: four 16-byte loads,
// one 16-byte store (N, lds, ldd multiples of 8; 16-byte aligned bases).
__global__ void copy_cols_bf16_vec_kernel(int64_t N, int k, const double* __restrict__ src, int64_t lds,
                                          __nv_bfloat16* __restrict__ dst, int64_t ldd) {
  const int64_t per_col = N / 8;
  const int64_t total = per_col * k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / per_col, i = (e % per_col) * 8;
    const double2* p = reinterpret_cast<const double2*>(src + j * lds + i);
    const double2 a = p[0], b = p[1], c = p[2], d = p[3];
    auto pack = [](double x, double y) {
      return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn((float)x)) |
             ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn((float)y)) << 16);
    };
    *reinterpret_cast<uint4*>(dst + j * ldd + i) = make_uint4(pack(a.x, a.y), pack(b.x, b.y), pack(c.x, c.y),
                                                              pack(d.x, d.y));
  }
}

template <typename TD, typename TS>
cudaError_t launch_copy_cols(int64_t N, int k, const TS* src, int64_t lds, TD* dst, int64_t ldd, cudaStream_t s) {
  ProfScope prof_(KC_VECTOR, s);
  if (k <= 0) return cudaSuccess;
  note_work((sizeof(TS) + sizeof(TD)) * (double)N * k, 0.0);
  if constexpr (std::is_same<TD, __nv_bfloat16>::value && std::is_same<TS, double>::value) {
    if (N % 8 == 0 && lds % 8 == 0 && ldd % 8 == 0 && reinterpret_cast<uintptr_t>(src) % 16 == 0 &&
        reinterpret_cast<uintptr_t>(dst) % 16 == 0) {
      const int64_t total = N / 8 * k;
      int64_t grid = (total + 255) / 256;
      if (grid > 152 * 32) grid = 152 * 32;
      { copy_cols_bf16_vec_kernel<<<(unsigned)grid, 256, 0, s>>>(N, k, src, lds, dst, ldd); note_launches(1); }
      return cudaGetLastError();
    }
  }
  { copy_cols_kernel<TD, TS><<<dim3(grid_for(N), k), 256, 0, s>>>(N, k, src, lds, dst, ldd); note_launches(1); }
  return cudaGetLastError();
}
template cudaError_t launch_copy_cols<float, double>(int64_t, int, const double*, int64_t, float*, int64_t,
                                                     cudaStream_t);
template cudaError_t launch_copy_cols<double, float>(int64_t, int, const float*, int64_t, double*, int64_t,
                                                     cudaStream_t);
template cudaError_t launch_copy_cols<double, double>(int64_t, int, const double*, int64_t, double*, int64_t,
                                                      cudaStream_t);
template cudaError_t launch_copy_cols<float, float>(int64_t, int, const float*, int64_t, float*, int64_t,
                                                    cudaStream_t);
template cudaError_t launch_copy_cols<__nv_bfloat16, double>(int64_t, int, const double*, int64_t, __nv_bfloat16*,
                                                             int64_t, cudaStream_t);

__global__ void axpby_kernel(int64_t N, double a, const double* __restrict__ x, int64_t ldx, double b,
                             double* __restrict__ y, int64_t ldy) {
  const int j = blockIdx.y;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    y[(int64_t)j * ldy + i] = a * x[(int64_t)j * ldx + i] + b * y[(int64_t)j * ldy + i];
}

cudaError_t launch_axpby_cols(int64_t N, int k, double a, const double* x, int64_t ldx, double b, double* y,
                              int64_t ldy, cudaStream_t s) {
  ProfScope prof_(KC_VECTOR, s);
  if (k <= 0) return cudaSuccess;
  note_work(24.0 * N * k, 3.0 * N * k);
  { axpby_kernel<<<dim3(grid_for(N), k), 256, 0, s>>>(N, a, x, ldx, b, y, ldy); note_launches(1); }
  return cudaGetLastError();
}

// Stage 1: block b of column j sums x(i,j)*y(i,j) over its grid-stride rows,
// tree-reduced in shared memory -> scratch[j * nb + b]. Stage 2: one block per
// column sums the nb partials in index order.
constexpr int kDotBlocks = 512;

size_t dot_scratch_elems(int64_t N, int k) {
  (void)N;
  return (size_t)k * kDotBlocks;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int tid = threadIdx.x;
  sh[tid] = v;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) sh[tid] += sh[tid + w];
    __syncthreads();
  }
  return sh[0];
}

// mode 0: x(:,j) . y(:,j); mode 1: X(:,j) . w (y is one vector)
__global__ void dot_stage1(int64_t N, const double* __restrict__ x, int64_t ldx, const double* __restrict__ y,
                           int64_t ldy, int mode, double* __restrict__ scratch) {
  __shared__ double sh[256];
  const int j = blockIdx.y;
  const double* xj = x + (int64_t)j * ldx;
  const double* yj = mode == 0 ? y + (int64_t)j * ldy : y;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    acc += xj[i] * yj[i];
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) scratch[(size_t)j * gridDim.x + blockIdx.x] = t;
}

__global__ void dot_stage2(const double* __restrict__ scratch, int nb, double* __restrict__ out) {
  __shared__ double sh[256];
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += scratch[(size_t)j * nb + b];
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) out[j] = t;
}

static cudaError_t dots_impl(int64_t N, int k, const double* x, int64_t ldx, const double* y, int64_t ldy, int mode,
                             double* out, double* scratch, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  int64_t nb = (N + 255) / 256;
  if (nb > kDotBlocks) nb = kDotBlocks;
  note_work(mode == 0 ? 16.0 * N * k : 8.0 * N * (k + 1.0), 2.0 * N * k);
  { dot_stage1<<<dim3((unsigned)nb, k), 256, 0, s>>>(N, x, ldx, y, ldy, mode, scratch); note_launches(1); }
  { dot_stage2<<<k, 256, 0, s>>>(scratch, (int)nb, out); note_launches(1); }
  return cudaGetLastError();
}

cudaError_t launch_dots(int64_t N, int k, const double* x, int64_t ldx, const double* y, int64_t ldy, double* out,
                        double* scratch, cudaStream_t s) {
  ProfScope prof_(KC_VECTOR, s);
  return dots_impl(N, k, x, ldx, y, ldy, 0, out, scratch, s);
}

cudaError_t launch_multidot(int64_t N, int k, const double* X, int64_t ldx, const double* w, double* out,
                            double* scratch, cudaStream_t s) {
  ProfScope prof_(KC_VECTOR, s);
  return dots_impl(N, k, X, ldx, w, 0, 1, out, scratch, s);
}

// w -= X h, X N x k (ld ldx), h a device vector of length k.
__global__ void gemv_sub_kernel(int64_t N, int k, const double* __restrict__ X, int64_t ldx,
                                const double* __restrict__ h, double* __restrict__ w) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < k; ++j) acc += X[(int64_t)j * ldx + i] * h[j];
    w[i] -= acc;
  }
}

cudaError_t launch_gemv_sub(int64_t N, int k, const double* X, int64_t ldx, const double* h, double* w,
                            cudaStream_t s) {
  ProfScope prof_(KC_VECTOR, s);
  if (k <= 0) return cudaSuccess;
  note_work(8.0 * N * (k + 2.0), 2.0 * N * k);
  { gemv_sub_kernel<<<grid_for(N), 256, 0, s>>>(N, k, X, ldx, h, w); note_launches(1); }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched Krylov-basis kernels of the lockstep multi-column FGMRES: basis
// vector q of right-hand side j is column q * k + j of a column-major block
// (ld N), so the q-th vectors of all k columns form one N x k matrix.

// out[q * k + j] = V(:, q * k + j) . w(:, j) for q < nq, fixed-order two-stage
// sums (stage 2 is dot_stage2 over the nb partials of each (q, j)).
__global__ void bdot_stage1(int64_t N, int k, const double* __restrict__ V, const double* __restrict__ w,
                            double* __restrict__ scratch) {
  __shared__ double sh[256];
  const int qj = blockIdx.y;
  const int j = qj % k;
  const double* v = V + (int64_t)qj * N;
  const double* x = w + (int64_t)j * N;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    acc += v[i] * x[i];
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) scratch[(size_t)qj * gridDim.x + blockIdx.x] = t;
}

cudaError_t launch_bdots(int64_t N, int k, int nq, const double* V, const double* w, double* out, double* scratch,
                         cudaStream_t s) {
  ProfScope prof_(KC_VECTOR, s);
  if (k <= 0 || nq <= 0) return cudaSuccess;
  int64_t nb = (N + 255) / 256;
  if (nb > kDotBlocks) nb = kDotBlocks;
  note_work(8.0 * N * k * (nq + 1.0), 2.0 * N * k * nq);
  { bdot_stage1<<<dim3((unsigned)nb, nq * k), 256, 0, s>>>(N, k, V, w, scratch); note_launches(1); }
  { dot_stage2<<<nq * k, 256, 0, s>>>(scratch, (int)nb, out); note_launches(1); }
  return cudaGetLastError();
}

// y(:, j) += alpha * sum_{q < nq} coef[q * k + j] V(:, q * k + j)   (coef on the device)
__global__ void bgemv_kernel(int64_t N, int k, int nq, const double* __restrict__ V, const double* __restrict__ coef,
                             double alpha, double* __restrict__ y, int64_t ldy) {
  const int j = blockIdx.y;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int q = 0; q < nq; ++q) acc += V[(int64_t)(q * k + j) * N + i] * coef[q * k + j];
    y[(int64_t)j * ldy + i] += alpha * acc;
  }
}

cudaError_t launch_bgemv(int64_t N, int k, int nq, const double* V, const double* coef, double alpha, double* y,
                         int64_t ldy, cudaStream_t s) {
  ProfScope prof_(KC_VECTOR, s);
  if (k <= 0 || nq <= 0) return cudaSuccess;
  note_work(8.0 * N * k * (nq + 2.0), 2.0 * N * k * nq);
  { bgemv_kernel<<<dim3(grid_for(N), k), 256, 0, s>>>(N, k, nq, V, coef, alpha, y, ldy); note_launches(1); }
  return cudaGetLastError();
}

// out(:, j) = w(:, j) / sqrt(nrm2[j]) (0 where nrm2[j] is 0): the next Arnoldi
// vectors, scaled on the device from the device norms.
__global__ void scale_inv_norm_kernel(int64_t N, const double* __restrict__ w, const double* __restrict__ nrm2,
                                      double* __restrict__ out) {
  const int j = blockIdx.y;
  const double nn = nrm2[j];
  const double sc = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    out[(int64_t)j * N + i] = w[(int64_t)j * N + i] * sc;
}

cudaError_t launch_scale_inv_norm(int64_t N, int k, const double* w, const double* nrm2, double* out,
                                  cudaStream_t s) {
  ProfScope prof_(KC_VECTOR, s);
  if (k <= 0) return cudaSuccess;
  note_work(16.0 * N * k, 1.0 * N * k);
  { scale_inv_norm_kernel<<<dim3(grid_for(N), k), 256, 0, s>>>(N, w, nrm2, out); note_launches(1); }
  return cudaGetLastError();
}

}  // namespace hodlr
