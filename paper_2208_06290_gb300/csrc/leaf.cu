// Leaf stage: batched LU with partial pivoting of the 2^L leaf blocks and the
// batched triangular solves with them (Alg. 1 leaf loop; Alg. 3 first two steps;
// Alg. 2 / Alg. 4 leaf step).
#include <type_traits>

#include "hodlr_internal.cuh"

namespace hodlr {

// ---------------------------------------------------------------------------
// Block-wide partial-pivot argmax over A(k..n-1, k) of a column-major matrix
// (ld = n) held in shared or global memory. Ties go to the smallest row index,
// as LAPACK i?amax does. Run by warp 0; result in *s_piv (n if the column is
// entirely NaN).
template <typename T>
__device__ __forceinline__ void warp_pivot_search(const T* A, int n, int ld, int k, int* s_piv, T* s_pval) {
  const int lane = threadIdx.x & 31;
  T best = T(-1);
  int bi = n;
  for (int i = k + lane; i < n; i += 32) {
    T v = fabs(A[(size_t)k * ld + i]);
    if (v > best) { best = v; bi = i; }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    T ov = __shfl_down_sync(0xffffffffu, best, off);
    int oi = __shfl_down_sync(0xffffffffu, bi, off);
    if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
  }
  if (lane == 0) { *s_piv = bi; *s_pval = best; }
}

// ---------------------------------------------------------------------------
// K1: leaf LU with partial pivoting, right-looking, one CTA per leaf.
// SMEM: the block lives in shared memory; otherwise it is factored in place
// in the LU buffer (global, L2-resident while the CTA runs).
template <typename TL, bool SMEM>
__global__ void __launch_bounds__(256) leaf_lu_kernel(int m, const double* D,  // may alias LU (in place)
                                                      TL* LU, int* __restrict__ perm,
                                                      double* __restrict__ leaf_ld, DevStatus* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  TL* A = SMEM ? reinterpret_cast<TL*>(smem_raw) : LU + (size_t)b * m * m;
  int* sperm = reinterpret_cast<int*>(smem_raw + (SMEM ? (size_t)m * m * sizeof(TL) : 0));
  TL* scol = reinterpret_cast<TL*>(sperm + ((m + 3) & ~3));
  __shared__ int s_piv, s_bad, s_swaps, s_sing;
  __shared__ TL s_pval;
  if (tid == 0) { s_bad = 0; s_swaps = 0; s_sing = -1; }
  __syncthreads();
  const double* Db = D + (size_t)b * m * m;
  int bad = 0;
  for (int e = tid; e < m * m; e += nt) {
    double v = Db[e];
    if (!isfinite(v)) bad = 1;
    A[e] = conv<TL>(v);
  }
  for (int i = tid; i < m; i += nt) sperm[i] = i;
  if (bad) atomicOr(&s_bad, 1);
  __syncthreads();
  if (s_bad && tid == 0) set_status(st, HODLR_ERR_NONFINITE, b, 0);

  for (int k = 0; k < m; ++k) {
    if (tid < 32) warp_pivot_search(A, m, m, k, &s_piv, &s_pval);
    __syncthreads();
    int p = s_piv;
    if (p >= m) p = k;
    if (p != k) {
      for (int j = tid; j < m; j += nt) {
        TL t = A[(size_t)j * m + k];
        A[(size_t)j * m + k] = A[(size_t)j * m + p];
        A[(size_t)j * m + p] = t;
      }
      if (tid == 0) {
        int t = sperm[k]; sperm[k] = sperm[p]; sperm[p] = t;
        s_swaps ^= 1;
      }
    }
    __syncthreads();
    const TL piv = A[(size_t)k * m + k];
    if (piv != TL(0)) {
      for (int i = k + 1 + tid; i < m; i += nt) {
        TL l = A[(size_t)k * m + i] / piv;
        A[(size_t)k * m + i] = l;
        scol[i] = l;
      }
    } else {
      if (tid == 0 && s_sing < 0) s_sing = k;
      for (int i = k + 1 + tid; i < m; i += nt) scol[i] = TL(0);
    }
    __syncthreads();
    const int n = m - k - 1;
    for (int e = tid; e < n * n; e += nt) {
      const int i = k + 1 + e % n;
      const int j = k + 1 + e / n;
      A[(size_t)j * m + i] -= scol[i] * A[(size_t)j * m + k];
    }
    __syncthreads();
  }
  if (tid == 0 && s_sing >= 0) set_status(st, HODLR_ERR_SINGULAR_LEAF, b, s_sing);
  // log|det D_b| and its sign, FP64
  if (tid < 32) {
    double la = 0.0;
    int neg = 0;
    for (int i = tid; i < m; i += 32) {
      double u = (double)A[(size_t)i * m + i];
      la += log(fabs(u));
      neg ^= (u < 0.0);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      la += __shfl_down_sync(0xffffffffu, la, off);
      neg ^= __shfl_down_sync(0xffffffffu, neg, off);
    }
    if (tid == 0) {
      leaf_ld[2 * b] = la;
      leaf_ld[2 * b + 1] = (s_sing >= 0) ? 0.0 : ((neg ^ s_swaps) ? -1.0 : 1.0);
    }
  }
  if (SMEM) {
    TL* out = LU + (size_t)b * m * m;
    for (int e = tid; e < m * m; e += nt) out[e] = A[e];
  }
  for (int i = tid; i < m; i += nt) perm[(size_t)b * m + i] = sperm[i];
}

template <typename TL>
static cudaError_t leaf_lu_dispatch(const Factor& F, const double* D, cudaStream_t s) {
  const int m = F.d.m;
  const int nleaf = 1 << F.d.L;
  const size_t aux = (size_t)((m + 3) & ~3) * sizeof(int) + (size_t)m * sizeof(TL) + 16;
  const size_t full = (size_t)m * m * sizeof(TL) + aux;
  TL* lu = static_cast<TL*>(F.lu);
  note_work((8.0 + sizeof(TL)) * nleaf * m * m + 4.0 * nleaf * m, 2.0 / 3.0 * m * m * (double)m * nleaf);
  if (full <= 160 * 1024) {
    cudaFuncSetAttribute(leaf_lu_kernel<TL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)full);
    { leaf_lu_kernel<TL, true><<<nleaf, 256, full, s>>>(m, D, lu, F.perm, F.leaf_ld, F.status); note_launches(1); }
  } else {
    { leaf_lu_kernel<TL, false><<<nleaf, 256, aux, s>>>(m, D, lu, F.perm, F.leaf_ld, F.status); note_launches(1); }
  }
  return cudaGetLastError();
}

cudaError_t launch_leaf_lu(const Factor& F, const double* D, cudaStream_t s) {
  ProfScope prof_(KC_LEAF_LU, s);
  if (leaf_uses_inverse(F)) return launch_leaf_inv(F, D, s);
  if (F.prec == HODLR_PREC_FP64) return leaf_lu_dispatch<double>(F, D, s);
  return leaf_lu_dispatch<float>(F, D, s);
}

// ---------------------------------------------------------------------------
// K2 / K6 / K8-leaf: X_b <- D_b^{-1} X_b (trans 0) or D_b^{-T} X_b (trans 1).
// One warp owns CPW right-hand-side columns of one leaf; lane l holds rows
// l, l+32, ... in registers, so the substitutions need no block barrier: the
// pivot row value moves by warp shuffle and each L / U column is read once
// per warp (coalesced, through L1/L2) for CPW columns at a time.
// SMEM: the CTA first copies the leaf's LU factor and permutation to shared
// memory and its warps then sweep all column groups of the leaf (one LU load
// per leaf instead of one per column group).
// The divisions by the pivots u_kk are multiplications by their reciprocals,
// formed once per CTA (within an ulp of the quotient): a double division is a
// multi-instruction sequence on the FP64 pipe, and one per column and pivot
// cost several times the substitutions' own FMAs.
template <typename TL, typename TIN, typename TOUT, int RPL, int CPW, bool SMEM>
__global__ void __launch_bounds__(256) leaf_solve_kernel(int m, const TL* __restrict__ LU,
                                                         const int* __restrict__ perm, const TIN* in,
                                                         int64_t ldin, TOUT* out, int64_t ldout, int ncols,
                                                         int trans) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int b = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const TL* A = LU + (size_t)b * m * m;
  const int* pb = perm + (size_t)b * m;
  __shared__ TL s_rcp[256];  // 1 / u_kk (m <= 256)
  for (int e = threadIdx.x; e < m; e += blockDim.x) s_rcp[e] = TL(1) / A[(size_t)e * m + e];
  __syncthreads();
  if (SMEM) {
    TL* sA = reinterpret_cast<TL*>(smem_raw);
    int* sp = reinterpret_cast<int*>(sA + (size_t)m * m);
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) sA[e] = A[e];
    for (int e = threadIdx.x; e < m; e += blockDim.x) sp[e] = pb[e];
    __syncthreads();
    A = sA;
    pb = sp;
  }
  const int64_t row0 = (int64_t)b * m;
  const int cstride = SMEM ? nwarps * CPW : 0;
  for (int col0 = SMEM ? warp * CPW : (blockIdx.y * nwarps + warp) * CPW; col0 < ncols;
       col0 += SMEM ? cstride : ncols) {
  TL x[CPW][RPL];
#pragma unroll
  for (int s = 0; s < RPL; ++s) {
    const int i = lane + 32 * s;
    const int src = (i < m) ? (trans ? i : pb[i]) : 0;
#pragma unroll
    for (int c = 0; c < CPW; ++c) {
      const int col = col0 + c;
      x[c][s] = (i < m && col < ncols) ? conv<TL>(in[(int64_t)col * ldin + row0 + src]) : TL(0);
    }
  }
  if (!trans) {
    // forward: unit lower L
#pragma unroll
    for (int kb = 0; kb < RPL; ++kb) {
      for (int kk = 0; kk < 32; ++kk) {
        const int k = kb * 32 + kk;
        if (k >= m) break;
        TL xk[CPW];
#pragma unroll
        for (int c = 0; c < CPW; ++c) xk[c] = __shfl_sync(0xffffffffu, x[c][kb], kk);
#pragma unroll
        for (int s = kb; s < RPL; ++s) {
          const int i = lane + 32 * s;
          if (i > k && i < m) {
            const TL l = A[(size_t)k * m + i];
#pragma unroll
            for (int c = 0; c < CPW; ++c) x[c][s] -= l * xk[c];
          }
        }
      }
    }
    // backward: upper U
#pragma unroll
    for (int kb = RPL - 1; kb >= 0; --kb) {
      for (int kk = 31; kk >= 0; --kk) {
        const int k = kb * 32 + kk;
        if (k >= m) continue;
        const TL rk = s_rcp[k];
        TL xk[CPW];
#pragma unroll
        for (int c = 0; c < CPW; ++c) {
          const TL v = __shfl_sync(0xffffffffu, x[c][kb], kk) * rk;
          if (lane == kk) x[c][kb] = v;
          xk[c] = v;
        }
#pragma unroll
        for (int s = 0; s <= kb; ++s) {
          const int i = lane + 32 * s;
          if (i < k) {
            const TL u = A[(size_t)k * m + i];
#pragma unroll
            for (int c = 0; c < CPW; ++c) x[c][s] -= u * xk[c];
          }
        }
      }
    }
#pragma unroll
    for (int s = 0; s < RPL; ++s) {
      const int i = lane + 32 * s;
      if (i < m) {
#pragma unroll
        for (int c = 0; c < CPW; ++c)
          if (col0 + c < ncols) out[(int64_t)(col0 + c) * ldout + row0 + i] = conv<TOUT>(x[c][s]);
      }
    }
  } else {
    // D = P^T L U, so D^T = U^T L^T P: forward with U^T (non-unit lower),
    // backward with L^T (unit upper), then scatter by the permutation.
#pragma unroll
    for (int kb = 0; kb < RPL; ++kb) {
      for (int kk = 0; kk < 32; ++kk) {
        const int k = kb * 32 + kk;
        if (k >= m) break;
        const TL rk = s_rcp[k];
        TL xk[CPW];
#pragma unroll
        for (int c = 0; c < CPW; ++c) {
          const TL v = __shfl_sync(0xffffffffu, x[c][kb], kk) * rk;
          if (lane == kk) x[c][kb] = v;
          xk[c] = v;
        }
#pragma unroll
        for (int s = kb; s < RPL; ++s) {
          const int i = lane + 32 * s;
          if (i > k && i < m) {
            const TL u = A[(size_t)i * m + k];  // U(k, i) = U^T(i, k)
#pragma unroll
            for (int c = 0; c < CPW; ++c) x[c][s] -= u * xk[c];
          }
        }
      }
    }
#pragma unroll
    for (int kb = RPL - 1; kb >= 0; --kb) {
      for (int kk = 31; kk >= 0; --kk) {
        const int k = kb * 32 + kk;
        if (k >= m) continue;
        TL xk[CPW];
#pragma unroll
        for (int c = 0; c < CPW; ++c) xk[c] = __shfl_sync(0xffffffffu, x[c][kb], kk);
#pragma unroll
        for (int s = 0; s <= kb; ++s) {
          const int i = lane + 32 * s;
          if (i < k) {
            const TL l = A[(size_t)i * m + k];  // L(k, i) = L^T(i, k)
#pragma unroll
            for (int c = 0; c < CPW; ++c) x[c][s] -= l * xk[c];
          }
        }
      }
    }
#pragma unroll
    for (int s = 0; s < RPL; ++s) {
      const int i = lane + 32 * s;
      if (i < m) {
        const int dst = pb[i];
#pragma unroll
        for (int c = 0; c < CPW; ++c)
          if (col0 + c < ncols) out[(int64_t)(col0 + c) * ldout + row0 + dst] = conv<TOUT>(x[c][s]);
      }
    }
  }
  }
}

template <typename TL, typename TIN, typename TOUT, int RPL, int CPW>
static cudaError_t leaf_solve_cpw(const Factor& F, const TIN* in, int64_t ldin, TOUT* out, int64_t ldout,
                                  int ncols, int trans, cudaStream_t s) {
  const int nleaf = 1 << F.d.L;
  const int m = F.d.m;
  const int cols_per_cta = 8 * CPW;
  const double Nd = (double)nleaf * m;
  note_work((sizeof(TIN) + sizeof(TOUT)) * Nd * ncols + sizeof(TL) * Nd * m + 4.0 * Nd, 2.0 * m * Nd * ncols);
  const size_t sm = (size_t)m * m * sizeof(TL) + (size_t)m * sizeof(int);
  if (ncols >= 2 * cols_per_cta && sm <= 160 * 1024) {
    cudaFuncSetAttribute(leaf_solve_kernel<TL, TIN, TOUT, RPL, CPW, true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    { leaf_solve_kernel<TL, TIN, TOUT, RPL, CPW, true><<<nleaf, 256, sm, s>>>(
        m, static_cast<const TL*>(F.lu), F.perm, in, ldin, out, ldout, ncols, trans); note_launches(1); }
  } else {
    dim3 grid(nleaf, (ncols + cols_per_cta - 1) / cols_per_cta);
    { leaf_solve_kernel<TL, TIN, TOUT, RPL, CPW, false><<<grid, 256, 0, s>>>(
        m, static_cast<const TL*>(F.lu), F.perm, in, ldin, out, ldout, ncols, trans); note_launches(1); }
  }
  return cudaGetLastError();
}

// Columns per warp: 4 (FP64) or 8 (FP32) registers' worth, fewer when the
// right-hand side is narrower, so no FLOPs go to padding columns.
template <typename TL, typename TIN, typename TOUT, int RPL>
static cudaError_t leaf_solve_rpl(const Factor& F, const TIN* in, int64_t ldin, TOUT* out, int64_t ldout,
                                  int ncols, int trans, cudaStream_t s) {
  constexpr int CPWMAX = sizeof(TL) == 8 ? 4 : 8;
  if (ncols == 1) return leaf_solve_cpw<TL, TIN, TOUT, RPL, 1>(F, in, ldin, out, ldout, ncols, trans, s);
  if (ncols == 2 || CPWMAX == 2) return leaf_solve_cpw<TL, TIN, TOUT, RPL, 2>(F, in, ldin, out, ldout, ncols, trans, s);
  if (ncols <= 4 || CPWMAX == 4) return leaf_solve_cpw<TL, TIN, TOUT, RPL, 4>(F, in, ldin, out, ldout, ncols, trans, s);
  return leaf_solve_cpw<TL, TIN, TOUT, RPL, CPWMAX>(F, in, ldin, out, ldout, ncols, trans, s);
}

template <typename TL, typename TIN, typename TOUT>
static cudaError_t leaf_solve_tl(const Factor& F, const TIN* in, int64_t ldin, TOUT* out, int64_t ldout,
                                 int ncols, int trans, cudaStream_t s) {
  const int m = F.d.m;
  if (m <= 32) return leaf_solve_rpl<TL, TIN, TOUT, 1>(F, in, ldin, out, ldout, ncols, trans, s);
  if (m <= 64) return leaf_solve_rpl<TL, TIN, TOUT, 2>(F, in, ldin, out, ldout, ncols, trans, s);
  if (m <= 128) return leaf_solve_rpl<TL, TIN, TOUT, 4>(F, in, ldin, out, ldout, ncols, trans, s);
  return leaf_solve_rpl<TL, TIN, TOUT, 8>(F, in, ldin, out, ldout, ncols, trans, s);
}

template <typename TIN, typename TOUT>
cudaError_t launch_leaf_solve(const Factor& F, const TIN* in, int64_t ldin, TOUT* out, int64_t ldout,
                              int ncols, int trans, cudaStream_t s) {
  ProfScope prof_(KC_LEAF_SOLVE, s);
  if (ncols <= 0) return cudaSuccess;
  if (leaf_uses_inverse(F)) return launch_leaf_apply_inv<TIN, TOUT>(F, in, ldin, out, ldout, ncols, trans, s);
  if (F.prec == HODLR_PREC_FP64) return leaf_solve_tl<double>(F, in, ldin, out, ldout, ncols, trans, s);
  return leaf_solve_tl<float>(F, in, ldin, out, ldout, ncols, trans, s);
}

template cudaError_t launch_leaf_solve<double, double>(const Factor&, const double*, int64_t, double*, int64_t,
                                                       int, int, cudaStream_t);
template cudaError_t launch_leaf_solve<double, float>(const Factor&, const double*, int64_t, float*, int64_t,
                                                      int, int, cudaStream_t);
template cudaError_t launch_leaf_solve<double, __nv_bfloat16>(const Factor&, const double*, int64_t,
                                                              __nv_bfloat16*, int64_t, int, int, cudaStream_t);
template cudaError_t launch_leaf_solve<float, float>(const Factor&, const float*, int64_t, float*, int64_t,
                                                     int, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Leaf part of the FP64 matvec: Y_b = D_b X_b. Thread i of the CTA owns row i
// of the leaf; KC columns of X_b are staged in shared memory per CTA.
template <int KC>
__global__ void __launch_bounds__(256) leaf_matvec_kernel(int m, const double* __restrict__ D,
                                                          const double* __restrict__ X, int64_t ldx,
                                                          double* __restrict__ Y, int64_t ldy, int k) {
  extern __shared__ double sx[];  // m x KC, [j][c]
  const int b = blockIdx.x;
  const int c0 = blockIdx.y * KC;
  const int kc = min(KC, k - c0);
  const double* Db = D + (size_t)b * m * m;
  const int64_t row0 = (int64_t)b * m;
  for (int e = threadIdx.x; e < m * KC; e += blockDim.x) {
    const int j = e % m, c = e / m;
    sx[j * KC + c] = (c < kc) ? X[(int64_t)(c0 + c) * ldx + row0 + j] : 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double acc[KC];
#pragma unroll
    for (int c = 0; c < KC; ++c) acc[c] = 0.0;
    for (int j = 0; j < m; ++j) {
      const double d = Db[(size_t)j * m + i];
#pragma unroll
      for (int c = 0; c < KC; ++c) acc[c] += d * sx[j * KC + c];
    }
#pragma unroll
    for (int c = 0; c < KC; ++c)
      if (c < kc) Y[(int64_t)(c0 + c) * ldy + row0 + i] = acc[c];
  }
}

template <int KC>
static void leaf_matvec_go(const hodlr_desc& d, const double* D, const double* X, int64_t ldx, double* Y,
                           int64_t ldy, int k, cudaStream_t s) {
  const int m = d.m;
  const int nleaf = 1 << d.L;
  const int threads = m >= 256 ? 256 : ((m + 31) / 32) * 32;
  dim3 grid(nleaf, (k + KC - 1) / KC);
  const size_t sm = (size_t)m * KC * sizeof(double);
  if (sm > 48 * 1024) cudaFuncSetAttribute(leaf_matvec_kernel<KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  { leaf_matvec_kernel<KC><<<grid, threads, sm, s>>>(m, D, X, ldx, Y, ldy, k); note_launches(1); }
}

cudaError_t launch_leaf_matvec(const hodlr_desc& d, const double* D, const double* X, int64_t ldx, double* Y,
                               int64_t ldy, int k, cudaStream_t s) {
  ProfScope prof_(KC_LEAF_MATVEC, s);
  const int m = d.m;
  const int nleaf = 1 << d.L;
  note_work(8.0 * ((double)m * m * nleaf + 2.0 * (double)d.N * k), 2.0 * m * (double)d.N * k);
  if (k == 1) leaf_matvec_go<1>(d, D, X, ldx, Y, ldy, k, s);
  else if (k <= 2) leaf_matvec_go<2>(d, D, X, ldx, Y, ldy, k, s);
  else if (k <= 4) leaf_matvec_go<4>(d, D, X, ldx, Y, ldy, k, s);
  else if (k <= 8) leaf_matvec_go<8>(d, D, X, ldx, Y, ldy, k, s);
  else leaf_matvec_go<32>(d, D, X, ldx, Y, ldy, k, s);
  return cudaGetLastError();
}

}  // namespace hodlr
