// Small kernels of the gradient of  loss = sum_j b_j^T A^{-1} b_j + log|det A|
// with respect to b, the leaf blocks D_b and the bases U_big, V_big
// (the sequencing is in api.cu, hodlr_grad).
#include "hodlr_internal.cuh"

namespace hodlr {

// Identity blocks: E(b*m + i, j) = delta_ij for every leaf b (N x m, ld N).
__global__ void leaf_identity_kernel(int64_t N, int m, double* E) {
  const int j = blockIdx.y;
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < N; row += (int64_t)gridDim.x * blockDim.x)
    E[(int64_t)j * N + row] = (row % m) == j ? 1.0 : 0.0;
}

cudaError_t launch_leaf_identity(int64_t N, int m, double* E, cudaStream_t s) {
  ProfScope prof_(KC_VECTOR, s);
  note_work(8.0 * N * m, 0.0);
  int64_t b = (N + 255) / 256;
  dim3 grid((unsigned)(b < 4096 ? b : 4096), m);
  { leaf_identity_kernel<<<grid, 256, 0, s>>>(N, m, E); note_launches(1); }
  return cudaGetLastError();
}

// out_b(i, j) = beta * out_b(i, j) + alpha * sum_t A(b m + i, t) B(b m + j, t)
//               + (Tadd ? Tadd(b m + j, i) : 0)          for every leaf b,
// out in the leaf-block layout of D (column-major m x m blocks), A and B
// N x K column-major, Tadd N x m column-major (ld N). CTA = one leaf x a
// 64 x 64 output tile; K streamed 32 at a time; 4 x 4 outputs per thread.
template <typename TB>
__global__ void __launch_bounds__(256) leaf_outer_kernel(int64_t N, int m, int K, const double* __restrict__ A,
                                                         int64_t lda, const TB* __restrict__ B, int64_t ldb,
                                                         double alpha, double beta, const double* __restrict__ Tadd,
                                                         double* __restrict__ out) {
  __shared__ double sA[32][64 + 1];
  __shared__ double sB[32][64 + 1];
  const int b = blockIdx.x;
  const int i0 = blockIdx.y * 64, j0 = blockIdx.z * 64;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t row0 = (int64_t)b * m;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = 0.0;
  for (int k0 = 0; k0 < K; k0 += 32) {
    for (int e = tid; e < 32 * 64; e += 256) {
      const int ii = e & 63, kk = e >> 6;
      const int k = k0 + kk;
      sA[kk][ii] = (k < K && i0 + ii < m) ? A[(int64_t)k * lda + row0 + i0 + ii] : 0.0;
      sB[kk][ii] = (k < K && j0 + ii < m) ? (double)B[(int64_t)k * ldb + row0 + j0 + ii] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 32; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = sA[kk][tx + 16 * a];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = sB[kk][ty + 16 * c];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] += av[a] * bv[c];
    }
    __syncthreads();
  }
  double* ob = out + (size_t)b * m * m;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int j = j0 + ty + 16 * c;
    if (j >= m) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = i0 + tx + 16 * a;
      if (i >= m) continue;
      double v = alpha * acc[a][c];
      if (beta != 0.0) v += beta * ob[(size_t)j * m + i];
      if (Tadd) v += Tadd[(int64_t)i * N + row0 + j];
      ob[(size_t)j * m + i] = v;
    }
  }
}

template <typename TB>
cudaError_t launch_leaf_outer(int64_t N, int m, int K, const double* A, int64_t lda, const TB* B, int64_t ldb,
                              double alpha, double beta, const double* Tadd, double* out, cudaStream_t s) {
  ProfScope prof_(KC_LEAF_MATVEC, s);
  const int nleaf = (int)(N / m);
  note_work((8.0 + sizeof(TB)) * (double)N * K +
                8.0 * ((double)N * m * (beta != 0.0 ? 2 : 1) + (Tadd ? (double)N * m : 0.0)),
            2.0 * (double)N * m * K);
  dim3 grid(nleaf, (m + 63) / 64, (m + 63) / 64);
  { leaf_outer_kernel<TB><<<grid, 256, 0, s>>>(N, m, K, A, lda, B, ldb, alpha, beta, Tadd, out); note_launches(1); }
  return cudaGetLastError();
}
template cudaError_t launch_leaf_outer<double>(int64_t, int, int, const double*, int64_t, const double*, int64_t,
                                               double, double, const double*, double*, cudaStream_t);
template cudaError_t launch_leaf_outer<float>(int64_t, int, int, const double*, int64_t, const float*, int64_t,
                                              double, double, const double*, double*, cudaStream_t);

// H_alpha for the children of every parent at child level c, from
// G = K~^{-T}: the first child gets G21 = G(r:2r, 0:r), the second G12 =
// G(0:r, r:2r). Written as r x r column-major slots per child (node index),
// H and, if HT != null, H^T.
__global__ void coupling_h_kernel(int r, const double* __restrict__ Kinv, double* __restrict__ H,
                                  double* __restrict__ HT) {
  const int n = 2 * r;
  const int64_t j = blockIdx.x;
  const double* Kj = Kinv + (size_t)j * n * n;
  for (int e = threadIdx.x; e < 2 * r * r; e += blockDim.x) {
    const int child = e / (r * r);
    const int a = (e % (r * r)) % r, b = (e % (r * r)) / r;
    // G(p, q) = Kinv(q, p) = Kj[p * n + q]
    const double v = child == 0 ? Kj[(size_t)(r + a) * n + b] : Kj[(size_t)a * n + r + b];
    const int64_t node = 2 * j + child;
    H[(size_t)node * r * r + (size_t)b * r + a] = v;
    if (HT) HT[(size_t)node * r * r + (size_t)a * r + b] = v;
  }
}

cudaError_t launch_coupling_h(const Factor& F, int c, double* H, double* HT, cudaStream_t s) {
  ProfScope prof_(KC_VECTOR, s);
  const int r = F.d.r;
  const int64_t parents = (int64_t)1 << (c - 1);
  note_work(8.0 * parents * (4.0 * r * r + 4.0 * r * r), 0.0);
  { coupling_h_kernel<<<(unsigned)parents, 128, 0, s>>>(r, F.K + F.Koff[c] * 4 * r * r, H, HT); note_launches(1); }
  return cudaGetLastError();
}

}  // namespace hodlr
