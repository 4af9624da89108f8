// In-place Gauss-Jordan inversion with partial pivoting of a small matrix in
// shared memory, by a whole CTA (leaf inverses of the low-precision factor,
// 2r x 2r coupling matrices).
#pragma once

#include "hodlr_internal.cuh"

namespace hodlr {

// A: n x n, column-major with leading dimension lda = n + 1 (the padding
// keeps row accesses free of bank conflicts). Per column k: (a) warp 0 finds
// the pivot (first max |a_ik|, i >= k, as LAPACK's getrf); (b) rows k and p
// are exchanged in all columns but k, the pivot row scaled by 1/piv is saved
// to srow and column k (read with the exchange applied) to scol; (c) every
// entry is updated: a_ij -= scol[i] * srow[j] (i != k, j != k), a_kj = srow[j],
// a_ik = -scol[i] / piv, a_kk = 1 / piv. The pivots go to spv; afterwards the
// columns are put back in order (the row exchanges undone in reverse on the
// columns): column j of the inverse is column spos[j] of A. The pivots and
// row exchanges are those of LU with partial pivoting, so
// log|det| = sum log|spv[k]| and sign = parity of negative pivots and swaps.
// Returns the first zero-pivot column in *sing (or -1) and, in *la / *neg,
// the log-determinant pieces (FP64, summed in a fixed order).
template <typename T>
__device__ void gj_invert_smem(T* A, int n, int lda, int* spiv, T* spv, T* scol, T* srow, int* spos, double* la,
                               int* neg, int* sing) {
  __shared__ int s_p;
  __shared__ T s_pv;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int k = 0; k < n; ++k) {
    if (warp == 0) {
      T best = T(-1);
      int bi = n;
      for (int i = k + lane; i < n; i += 32) {
        const T v = fabs(A[(size_t)k * lda + i]);
        if (v > best) { best = v; bi = i; }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const T ov = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if (lane == 0) {
        const int p = bi < n ? bi : k;
        s_p = p;
        s_pv = A[(size_t)k * lda + p];
        spiv[k] = p;
        spv[k] = s_pv;
      }
    }
    __syncthreads();
    const int p = s_p;
    const T piv = s_pv;
    const T rp = piv != T(0) ? T(1) / piv : T(0);
    for (int j = tid; j < n; j += nt) {
      if (j != k) {
        const T a = A[(size_t)j * lda + k], b = A[(size_t)j * lda + p];
        A[(size_t)j * lda + p] = a;
        A[(size_t)j * lda + k] = b;
        srow[j] = b * rp;
      }
      const int src = j == k ? p : (j == p ? k : j);
      scol[j] = A[(size_t)k * lda + src];
    }
    __syncthreads();
    for (int j = warp; j < n; j += nw) {
      T* Aj = A + (size_t)j * lda;
      if (j == k) {
        for (int i = lane; i < n; i += 32) Aj[i] = (i == k) ? rp : -scol[i] * rp;
      } else {
        const T sj = srow[j];
        for (int i = lane; i < n; i += 32) Aj[i] = (i == k) ? sj : Aj[i] - scol[i] * sj;
      }
    }
    __syncthreads();
  }
  if (warp == 0) {
    double l = 0.0;
    int ng = 0, sg = n;
    for (int k = lane; k < n; k += 32) {
      const T v = spv[k];
      l += log(fabs((double)v));
      ng ^= (v < T(0)) ^ (spiv[k] != k);
      if (v == T(0) && k < sg) sg = k;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      l += __shfl_down_sync(0xffffffffu, l, off);
      ng ^= __shfl_down_sync(0xffffffffu, ng, off);
      sg = min(sg, __shfl_down_sync(0xffffffffu, sg, off));
    }
    if (lane == 0) {
      *la = l;
      *neg = ng;
      *sing = sg < n ? sg : -1;
      for (int j = 0; j < n; ++j) spos[j] = j;
      for (int kk = n - 1; kk >= 0; --kk) {
        const int t = spos[kk];
        spos[kk] = spos[spiv[kk]];
        spos[spiv[kk]] = t;
      }
    }
  }
  __syncthreads();
}

// C (m x n, ldc) = alpha * A (m x k, lda) * B (k x n, ldb) + beta * C, all in
// shared memory, column-major, by the whole CTA (warps over columns of C,
// lanes over rows). Callers separate dependent calls with __syncthreads.
// Each thread owns 4 x 4 outputs (rows tx + 16a, columns ty + 16b of a
// 64 x 64 tile, tx = tid % 16, ty = tid / 16 for 256 threads), so every
// k step costs 8 shared loads for 16 FMAs.
template <typename T>
__device__ void smem_gemm(int m, int n, int k, T alpha, const T* A, int lda, const T* B, int ldb, T beta, T* C,
                          int ldc) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int tyn = blockDim.x >> 4;
  for (int i0 = 0; i0 < m; i0 += 64)
    for (int j0 = 0; j0 < n; j0 += 4 * tyn) {
      T acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
      int ii[4], jj[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        ii[a] = i0 + tx + 16 * a;
        jj[a] = j0 + ty + tyn * a;
      }
      for (int t = 0; t < k; ++t) {
        T av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = ii[a] < m ? A[(size_t)t * lda + ii[a]] : T(0);
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = jj[b] < n ? B[(size_t)jj[b] * ldb + t] : T(0);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
          if (ii[a] < m && jj[b] < n) {
            T* cp = C + (size_t)jj[b] * ldc + ii[a];
            *cp = alpha * acc[a][b] + (beta != T(0) ? beta * *cp : T(0));
          }
    }
}

// After gj_invert_smem: put the inverse's columns in order (column j of the
// inverse is column spos[j] of A), using tmp (n x n, ld n) as scratch.
template <typename T>
__device__ void gj_unscramble(T* A, int n, int lda, const int* spos, T* tmp) {
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    tmp[(size_t)j * n + i] = A[(size_t)spos[j] * lda + i];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e % n, j = e / n;
    A[(size_t)j * lda + i] = tmp[(size_t)j * n + i];
  }
  __syncthreads();
}

}  // namespace hodlr
