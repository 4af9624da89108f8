// Leaf stage of the low-precision factor for leaves of at most 128 rows: each
// leaf block is inverted in shared memory (FP32 Gauss-Jordan elimination with
// partial pivoting, whose pivots and row swaps are those of getrf, so the
// log-determinant is unchanged) and the leaf "solves" of Alg. 1 / Alg. 2
// (D_b^{-1} applied to Y_big rows or to right-hand sides) become small dense
// GEMMs with D_b^{-1}, free of the serial dependence of substitutions.
#include "gj.cuh"

namespace hodlr {

// One CTA per leaf: D_b (FP64) -> FP32 in shared memory -> D_b^{-1} (FP32) in
// the factor's leaf buffer, log|det D_b| and sign, status on a zero pivot or
// a non-finite entry. Leaves of up to 64 rows are inverted by Gauss-Jordan
// with partial pivoting directly; larger leaves (up to 128 rows) as 2 x 2
// blocks [[A, B], [C, E]] with a 64-row leading block:
//   X = A^{-1} B, S = E - C X, Y = C A^{-1}, Z = S^{-1} Y,
//   D^{-1} = [[A^{-1} + X Z, -X S^{-1}], [-Z, S^{-1}]],
// each of A and S inverted by Gauss-Jordan with partial pivoting within the
// block (log|det D| = log|det A| + log|det S|).
__global__ void __launch_bounds__(256) leaf_inv_kernel(int m, const double* __restrict__ D, float* __restrict__ Dinv,
                                                       double* __restrict__ leaf_ld, DevStatus* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lda = m + 1;
  float* A = reinterpret_cast<float*>(smem_raw);
  float* T = A + (size_t)m * lda;  // 64 x 64 scratch
  float* scol = T + 64 * 64;
  float* srow = scol + 64;
  float* spv = srow + 64;
  int* spiv = reinterpret_cast<int*>(spv + 64);
  int* spos = spiv + 64;
  __shared__ double s_la1, s_la2;
  __shared__ int s_neg1, s_neg2, s_sing1, s_sing2, s_bad;
  const int b = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) { s_bad = 0; s_la2 = 0.0; s_neg2 = 0; s_sing2 = -1; }
  __syncthreads();
  const double* Db = D + (size_t)b * m * m;
  int bad = 0;
  for (int e = tid; e < m * m; e += nt) {
    const double v = Db[e];
    bad |= !isfinite(v);
    A[(size_t)(e / m) * lda + (e % m)] = (float)v;
  }
  if (bad) atomicOr(&s_bad, 1);
  __syncthreads();
  if (s_bad && tid == 0) set_status(st, HODLR_ERR_NONFINITE, b, 0);
  const int m1 = m > 64 ? 64 : m, m2 = m - m1;
  float* A11 = A;
  float* A12 = A + (size_t)m1 * lda;
  float* A21 = A + m1;
  float* A22 = A + (size_t)m1 * lda + m1;
  gj_invert_smem<float>(A11, m1, lda, spiv, spv, scol, srow, spos, &s_la1, &s_neg1, &s_sing1);
  gj_unscramble<float>(A11, m1, lda, spos, T);
  if (m2 > 0) {
    smem_gemm<float>(m1, m2, m1, 1.f, A11, lda, A12, lda, 0.f, T, m1);  // X = A^{-1} B
    __syncthreads();
    for (int e = tid; e < m1 * m2; e += nt) A12[(size_t)(e / m1) * lda + e % m1] = T[e];
    __syncthreads();
    smem_gemm<float>(m2, m2, m1, -1.f, A21, lda, A12, lda, 1.f, A22, lda);  // S = E - C X
    __syncthreads();
    smem_gemm<float>(m2, m1, m1, 1.f, A21, lda, A11, lda, 0.f, T, m2);  // Y = C A^{-1}
    __syncthreads();
    for (int e = tid; e < m2 * m1; e += nt) A21[(size_t)(e / m2) * lda + e % m2] = T[e];
    __syncthreads();
    gj_invert_smem<float>(A22, m2, lda, spiv, spv, scol, srow, spos, &s_la2, &s_neg2, &s_sing2);
    gj_unscramble<float>(A22, m2, lda, spos, T);
    smem_gemm<float>(m2, m1, m2, 1.f, A22, lda, A21, lda, 0.f, T, m2);  // Z = S^{-1} Y
    __syncthreads();
    for (int e = tid; e < m2 * m1; e += nt) A21[(size_t)(e / m2) * lda + e % m2] = -T[e];  // [21] = -Z
    __syncthreads();
    smem_gemm<float>(m1, m1, m2, -1.f, A12, lda, A21, lda, 1.f, A11, lda);  // [11] = A^{-1} + X Z
    __syncthreads();
    smem_gemm<float>(m1, m2, m2, 1.f, A12, lda, A22, lda, 0.f, T, m1);  // X S^{-1}
    __syncthreads();
    for (int e = tid; e < m1 * m2; e += nt) A12[(size_t)(e / m1) * lda + e % m1] = -T[e];  // [12]
    __syncthreads();
  }
  float* out = Dinv + (size_t)b * m * m;
  for (int e = tid; e < m * m; e += nt) out[e] = A[(size_t)(e / m) * lda + (e % m)];
  if (tid == 0) {
    const int sing = s_sing1 >= 0 ? s_sing1 : (s_sing2 >= 0 ? m1 + s_sing2 : -1);
    leaf_ld[2 * b] = s_la1 + s_la2;
    leaf_ld[2 * b + 1] = sing >= 0 ? 0.0 : ((s_neg1 ^ s_neg2) ? -1.0 : 1.0);
    if (sing >= 0) set_status(st, HODLR_ERR_SINGULAR_LEAF, b, sing);
  }
}

bool leaf_uses_inverse(const Factor& F) { return F.prec != HODLR_PREC_FP64 && F.d.m <= 128; }

cudaError_t launch_leaf_inv(const Factor& F, const double* D, cudaStream_t s) {
  const int m = F.d.m;
  const int nleaf = 1 << F.d.L;
  const size_t sm = (size_t)m * (m + 1) * 4 + 64 * 64 * 4 + 3 * 64 * 4 + 2 * 64 * 4;
  note_work((8.0 + 4.0) * nleaf * m * m, 2.0 * (double)m * m * m * nleaf);
  cudaFuncSetAttribute(leaf_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  { leaf_inv_kernel<<<nleaf, 256, sm, s>>>(m, D, static_cast<float*>(F.lu), F.leaf_ld, F.status); note_launches(1); }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// out(I_b, cols) = op(Dinv_b) * in(I_b, cols), op = identity or transpose.
// Wide: CTA = one leaf x 64 columns, all m <= 128 rows; K = m staged 32 at a
// time; thread tile 8 rows x 4 columns. In-place safe: a CTA reads every input
// row of its columns before it writes.
template <typename TIN, typename TOUT>
__global__ void __launch_bounds__(256) leaf_apply_wide_kernel(int m, const float* __restrict__ Dinv, const TIN* in,
                                                              int64_t ldin, TOUT* out, int64_t ldout, int ncols,
                                                              int trans) {
  __shared__ float sA[32][128 + 4];  // [kk][i] = op(Dinv)(i, k0 + kk)
  __shared__ float sB[32][64 + 4];   // [kk][j] = in(k0 + kk, j0 + j)
  const int b = blockIdx.x;
  const int j0 = blockIdx.y * 64;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const float* Ab = Dinv + (size_t)b * m * m;
  const int64_t row0 = (int64_t)b * m;
  float acc[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = 0.f;
  for (int k0 = 0; k0 < m; k0 += 32) {
    for (int e = tid; e < 32 * 128; e += 256) {
      const int i = e & 127, kk = e >> 7;
      const int k = k0 + kk;
      float v = 0.f;
      if (i < m && k < m) v = trans ? Ab[(size_t)i * m + k] : Ab[(size_t)k * m + i];
      sA[kk][i] = v;
    }
    for (int e = tid; e < 32 * 64; e += 256) {
      const int kk = e & 31, j = e >> 5;
      const int k = k0 + kk;
      sB[kk][j] = (k < m && j0 + j < ncols) ? conv<float>(in[(int64_t)(j0 + j) * ldin + row0 + k]) : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 32; ++kk) {
      float av[8], bv[4];
#pragma unroll
      for (int a = 0; a < 8; ++a) av[a] = sA[kk][ty + 16 * a];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = sB[kk][tx + 16 * c];
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] += av[a] * bv[c];
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int j = j0 + tx + 16 * c;
    if (j >= ncols) continue;
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int i = ty + 16 * a;
      if (i < m) out[(int64_t)j * ldout + row0 + i] = conv<TOUT>(acc[a][c]);
    }
  }
}

// Narrow (ncols <= 8): thread i of the CTA owns row i; the leaf's right-hand
// sides are staged in shared memory first (in-place safe).
template <typename TIN, typename TOUT, int KC>
__global__ void __launch_bounds__(128) leaf_apply_narrow_kernel(int m, const float* __restrict__ Dinv, const TIN* in,
                                                                int64_t ldin, TOUT* out, int64_t ldout, int ncols,
                                                                int trans) {
  __shared__ float sx[128 * KC];
  const int b = blockIdx.x;
  const float* Ab = Dinv + (size_t)b * m * m;
  const int64_t row0 = (int64_t)b * m;
  for (int e = threadIdx.x; e < m * KC; e += blockDim.x) {
    const int k = e % m, c = e / m;
    sx[k * KC + c] = c < ncols ? conv<float>(in[(int64_t)c * ldin + row0 + k]) : 0.f;
  }
  __syncthreads();
  const int i = threadIdx.x;
  if (i >= m) return;
  float acc[KC];
#pragma unroll
  for (int c = 0; c < KC; ++c) acc[c] = 0.f;
  for (int k = 0; k < m; ++k) {
    const float a = trans ? Ab[(size_t)i * m + k] : Ab[(size_t)k * m + i];
#pragma unroll
    for (int c = 0; c < KC; ++c) acc[c] += a * sx[k * KC + c];
  }
#pragma unroll
  for (int c = 0; c < KC; ++c)
    if (c < ncols) out[(int64_t)c * ldout + row0 + i] = conv<TOUT>(acc[c]);
}

template <typename TIN, typename TOUT>
cudaError_t launch_leaf_apply_inv(const Factor& F, const TIN* in, int64_t ldin, TOUT* out, int64_t ldout, int ncols,
                                  int trans, cudaStream_t s) {
  const int m = F.d.m;
  const int nleaf = 1 << F.d.L;
  const float* Dinv = static_cast<const float*>(F.lu);
  const double Nd = (double)nleaf * m;
  note_work((sizeof(TIN) + sizeof(TOUT)) * Nd * ncols + 4.0 * Nd * m, 2.0 * m * Nd * ncols);
  if (ncols <= 8) {
    const int th = ((m + 31) / 32) * 32;
    if (ncols == 1)
      { leaf_apply_narrow_kernel<TIN, TOUT, 1><<<nleaf, th, 0, s>>>(m, Dinv, in, ldin, out, ldout, ncols, trans); note_launches(1); }
    else if (ncols <= 2)
      { leaf_apply_narrow_kernel<TIN, TOUT, 2><<<nleaf, th, 0, s>>>(m, Dinv, in, ldin, out, ldout, ncols, trans); note_launches(1); }
    else if (ncols <= 4)
      { leaf_apply_narrow_kernel<TIN, TOUT, 4><<<nleaf, th, 0, s>>>(m, Dinv, in, ldin, out, ldout, ncols, trans); note_launches(1); }
    else
      { leaf_apply_narrow_kernel<TIN, TOUT, 8><<<nleaf, th, 0, s>>>(m, Dinv, in, ldin, out, ldout, ncols, trans); note_launches(1); }
  } else {
    dim3 grid(nleaf, (ncols + 63) / 64);
    { leaf_apply_wide_kernel<TIN, TOUT><<<grid, 256, 0, s>>>(m, Dinv, in, ldin, out, ldout, ncols, trans); note_launches(1); }
  }
  return cudaGetLastError();
}

template cudaError_t launch_leaf_apply_inv<double, float>(const Factor&, const double*, int64_t, float*, int64_t, int,
                                                          int, cudaStream_t);
template cudaError_t launch_leaf_apply_inv<double, __nv_bfloat16>(const Factor&, const double*, int64_t,
                                                                  __nv_bfloat16*, int64_t, int, int, cudaStream_t);
template cudaError_t launch_leaf_apply_inv<float, float>(const Factor&, const float*, int64_t, float*, int64_t, int,
                                                         int, cudaStream_t);

}  // namespace hodlr
