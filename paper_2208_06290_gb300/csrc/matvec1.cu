// FP64 HODLR matvec y = A x for one right-hand side in four launches
// (Eq. e:rank: y = D x + sum over levels and siblings of U_alpha (V_beta^T x_beta)):
//   1. per leaf b: the projections of x(I_b) on every basis column,
//      p_b = V(I_b, 0:rL)^T x(I_b)  (all levels at once, V streamed once);
//   2. per level c and node alpha: s_c(alpha) = sum of p_b(block c-1) over
//      the leaves of alpha (fixed order; runs of 64 leaves, then runs per node);
//   3. per leaf b: y(I_b) = D_b x(I_b) + U(I_b, 0:rL) t_b, where block c-1 of
//      t_b is s_c(sibling of b's level-c ancestor)  (U and D streamed once).
// The levels are independent in a matvec, unlike in the solves.
#include "hodlr_internal.cuh"

namespace hodlr {

template <typename TA>
__device__ __forceinline__ TA butterfly_reduce32(TA (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool upper = (lane & s) != 0;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const TA send = upper ? v[i] : v[i + s];
      const TA keep = upper ? v[i + s] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  return v[0];
}

// 1. One CTA (4 warps) per leaf; warp w takes 32-column groups w, w+4, ...;
// lane l accumulates rows l, l+32, ... of the leaf; the butterfly leaves the
// column total of group column l in lane l.
__global__ void __launch_bounds__(128) mv1_leaf_project_kernel(int m, int rL, const double* __restrict__ V,
                                                               int64_t ldv, const double* __restrict__ x,
                                                               double* __restrict__ pleaf) {
  const int b = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = (int64_t)b * m;
  for (int g = warp; g * 32 < rL; g += 4) {
    double acc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = 0.0;
    for (int i = lane; i < m; i += 32) {
      const double xv = x[row0 + i];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int col = g * 32 + j;
        if (col < rL) acc[j] += V[(int64_t)col * ldv + row0 + i] * xv;
      }
    }
    const double t = butterfly_reduce32(acc);
    if (g * 32 + lane < rL) pleaf[(size_t)b * rL + g * 32 + lane] = t;
  }
}

// 1 (m = 128, 16-byte aligned V and x, even ldv). One warp per (leaf b, 16
// basis columns): lane l covers rows 4l .. 4l+3 of the leaf (two 16-byte
// loads per column, fully coalesced), then a transposed butterfly over the
// lane bits 3..0 and one exchange across bit 4 leave column l % 16's total in
// lanes l and l + 16.
__global__ void __launch_bounds__(256) mv1_leaf_project16_kernel(int rL, int ngroups, int64_t nleaf,
                                                                 const double* __restrict__ V, int64_t ldv,
                                                                 const double* __restrict__ x,
                                                                 double* __restrict__ pleaf) {
  const int lane = threadIdx.x & 31;
  const int64_t item = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (item >= nleaf * ngroups) return;  // whole warp
  const int64_t b = item / ngroups;
  const int c0 = (int)(item % ngroups) * 16;
  const int64_t row = b * 128 + 4 * lane;
  double xv[4];
  load4(x + row, xv);
  double v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    v[j] = 0.0;
    if (c0 + j < rL) {
      double a[4];
      load4(V + (int64_t)(c0 + j) * ldv + row, a);
      v[j] = fma(a[3], xv[3], fma(a[2], xv[2], fma(a[1], xv[1], a[0] * xv[0])));
    }
  }
#pragma unroll
  for (int s = 8; s >= 1; s >>= 1) {
    const bool upper = (lane & s) != 0;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const double send = upper ? v[i] : v[i + s];
      const double keep = upper ? v[i + s] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  const double t = v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);
  if (lane < 16 && c0 + lane < rL) pleaf[(size_t)b * rL + c0 + lane] = t;
}

// 1 (m = 128, 4 | nleaf, 16-byte aligned V and x, even ldv). One warp per
// (4 consecutive leaves, 16 basis columns): the 8 lanes of group g cover
// leaf 4w + g, lane q of the group rows 16q .. 16q+15 (eight 16-byte loads
// per column), so each lane's partial is a 16-row dot product and the
// per-leaf totals take a transposed butterfly over the group's 3 lane bits
// (14 FP64 adds per lane against 256 FMAs; the FP64 pipe is this kernel's
// bound). Lane q of a group ends with the totals of columns 2q and 2q + 1
// of its leaf.
__global__ void __launch_bounds__(256) mv1_leaf_project_g8_kernel(int rL, int ngroups, int64_t nleaf,
                                                                  const double* __restrict__ V, int64_t ldv,
                                                                  const double* __restrict__ x,
                                                                  double* __restrict__ pleaf) {
  const int lane = threadIdx.x & 31;
  const int64_t item = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (item >= (nleaf / 4) * ngroups) return;  // whole warp
  const int64_t b = (item / ngroups) * 4 + (lane >> 3);
  const int c0 = (int)(item % ngroups) * 16;
  const int q = lane & 7;
  const int64_t row = b * 128 + 16 * q;
  double xv[16];
#pragma unroll
  for (int t = 0; t < 16; t += 4) {
    double a[4];
    load4(x + row + t, a);
    xv[t] = a[0];
    xv[t + 1] = a[1];
    xv[t + 2] = a[2];
    xv[t + 3] = a[3];
  }
  double v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    v[j] = 0.0;
    if (c0 + j < rL) {
      const double* col = V + (int64_t)(c0 + j) * ldv + row;
      double acc = 0.0;
#pragma unroll
      for (int t = 0; t < 16; t += 4) {
        double a[4];
        load4(col + t, a);
        acc = fma(a[0], xv[t], acc);
        acc = fma(a[1], xv[t + 1], acc);
        acc = fma(a[2], xv[t + 2], acc);
        acc = fma(a[3], xv[t + 3], acc);
      }
      v[j] = acc;
    }
  }
  // transposed butterfly over lane bits 2, 1, 0 (within the group of 8):
  // after the step on bit s the lanes with that bit set keep the upper half
  // of the remaining columns
  int base = 0;
#pragma unroll
  for (int s = 4, h = 8; s >= 1; s >>= 1, h >>= 1) {
    const bool upper = (lane & s) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const double send = upper ? v[i] : v[i + h];
      const double keep = upper ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
    base += upper ? h : 0;
  }
  // v[0], v[1]: totals of columns c0 + base, c0 + base + 1 of leaf b
  if (c0 + base < rL) pleaf[(size_t)b * rL + c0 + base] = v[0];
  if (c0 + base + 1 < rL) pleaf[(size_t)b * rL + c0 + base + 1] = v[1];
}

// 2a. Partial sums over runs of at most 64 consecutive leaves (never across
// a node boundary), all levels in one launch: one CTA of r threads per
// (level c, run), runs numbered level by level; thread j sums column
// (c-1) r + j over the run in leaf order.
// 2b. Per (level c, node), all levels in one launch: the node's runs summed
// in order.
constexpr int kMvRun = 64;

__host__ __device__ inline int64_t mv1_runs(int L, int c) {
  const int64_t per_node = (int64_t)1 << (L - c);
  return ((int64_t)1 << c) * ((per_node + kMvRun - 1) / kMvRun);
}

__host__ __device__ inline int64_t mv1_runs_before(int L, int c) {
  int64_t t = 0;
  for (int cc = 1; cc < c; ++cc) t += mv1_runs(L, cc);
  return t;
}

__global__ void mv1_run_sum_kernel(int L, int r, const double* __restrict__ pleaf, double* __restrict__ runs) {
  const int64_t id = blockIdx.x;
  int c = 1;
  while (c < L && id >= mv1_runs_before(L, c + 1)) ++c;
  const int64_t run = id - mv1_runs_before(L, c);
  const int64_t per_node = (int64_t)1 << (L - c);
  const int64_t len = per_node < kMvRun ? per_node : kMvRun;
  const int64_t b0 = run * len;
  const int rL = r * L;
  const int j = threadIdx.x;
  if (j >= r) return;
  double acc = 0.0;
  for (int64_t b = 0; b < len; ++b) acc += pleaf[(size_t)(b0 + b) * rL + (c - 1) * r + j];
  runs[(size_t)id * r + j] = acc;
}

__global__ void mv1_node_sum_kernel(int L, int r, const double* __restrict__ runs, double* __restrict__ S) {
  const int64_t id = blockIdx.x;  // = (2^c - 2) + alpha
  int c = 1;
  while (id >= ((int64_t)2 << c) - 2) ++c;
  const int64_t alpha = id - (((int64_t)1 << c) - 2);
  const int64_t per_node = (int64_t)1 << (L - c);
  const int64_t rpn = (per_node + kMvRun - 1) / kMvRun;
  const int64_t base = mv1_runs_before(L, c) + alpha * rpn;
  const int j = threadIdx.x;
  if (j >= r) return;
  double acc = 0.0;
  for (int64_t q = 0; q < rpn; ++q) acc += runs[(size_t)(base + q) * r + j];
  S[(size_t)id * r + j] = acc;
}

// 3. One CTA per leaf: gather t_b (rL values) and x(I_b) into shared memory,
// then thread per row: y = D_b x_b + U(row, :) t_b.
__global__ void __launch_bounds__(256) mv1_leaf_apply_kernel(int m, int L, int r, const double* __restrict__ D,
                                                             const double* __restrict__ U, int64_t ldu,
                                                             const double* __restrict__ x,
                                                             const double* __restrict__ S, double* __restrict__ y) {
  extern __shared__ double sh[];
  const int rL = r * L;
  double* t = sh;          // rL
  double* xs = sh + rL;    // m
  const int b = blockIdx.x;
  const int64_t row0 = (int64_t)b * m;
  for (int e = threadIdx.x; e < rL; e += blockDim.x) {
    const int c = e / r + 1, j = e % r;
    const int64_t alpha = (int64_t)b >> (L - c);            // b's ancestor at level c
    const int64_t id = (((int64_t)1 << c) - 2) + (alpha ^ 1);  // its sibling
    t[e] = S[(size_t)id * r + j];
  }
  for (int e = threadIdx.x; e < m; e += blockDim.x) xs[e] = x[row0 + e];
  __syncthreads();
  const double* Db = D + (size_t)b * m * m;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double acc = 0.0;
    for (int jj = 0; jj < m; ++jj) acc += Db[(size_t)jj * m + i] * xs[jj];
    for (int e = 0; e < rL; ++e) acc += U[(int64_t)e * ldu + row0 + i] * t[e];
    y[row0 + i] = acc;
  }
}

size_t matvec1_scratch_elems(const hodlr_desc& d) {
  const size_t nleaf = (size_t)1 << d.L;
  const size_t runs = (size_t)mv1_runs_before(d.L, d.L + 1);
  return nleaf * (size_t)d.r * d.L + ((size_t)2 << d.L) * (size_t)d.r + runs * (size_t)d.r;
}

cudaError_t launch_matvec1(const hodlr_desc& d, const double* D, const double* U, const double* V, const double* x,
                           double* y, double* scratch, cudaStream_t s) {
  const int m = d.m, L = d.L, r = d.r, rL = r * L;
  const int64_t nleaf = (int64_t)1 << L;
  double* pleaf = scratch;
  double* S = scratch + (size_t)nleaf * rL;
  double* runs = S + ((size_t)2 << L) * r;
  {
    ProfScope prof_(KC_MATVEC, s);
    note_work(8.0 * ((double)d.N * rL + d.N + nleaf * rL), 2.0 * d.N * rL);
    const bool vec16 = m == 128 && ((reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(x)) % 16 == 0) &&
                       d.ldv % 2 == 0;
    if (vec16 && nleaf % 4 == 0) {
      const int ngroups = (rL + 15) / 16;
      const int64_t warps = nleaf / 4 * ngroups;
      { mv1_leaf_project_g8_kernel<<<(unsigned)((warps + 7) / 8), 256, 0, s>>>(rL, ngroups, nleaf, V, d.ldv, x, pleaf); note_launches(1); }
    } else if (vec16) {
      const int ngroups = (rL + 15) / 16;
      const int64_t warps = nleaf * ngroups;
      { mv1_leaf_project16_kernel<<<(unsigned)((warps + 7) / 8), 256, 0, s>>>(rL, ngroups, nleaf, V, d.ldv, x, pleaf); note_launches(1); }
    } else {
      { mv1_leaf_project_kernel<<<(unsigned)nleaf, 128, 0, s>>>(m, rL, V, d.ldv, x, pleaf); note_launches(1); }
    }
  }
  {
    ProfScope prof_(KC_REDUCE, s);
    const int64_t pairs = ((int64_t)2 << L) - 2;
    note_work(8.0 * ((double)nleaf * rL + pairs * r), (double)nleaf * rL);
    const int th = ((r + 31) / 32) * 32;
    { mv1_run_sum_kernel<<<(unsigned)mv1_runs_before(L, L + 1), th, 0, s>>>(L, r, pleaf, runs); note_launches(1); }
    { mv1_node_sum_kernel<<<(unsigned)pairs, th, 0, s>>>(L, r, runs, S); note_launches(1); }
  }
  {
    ProfScope prof_(KC_MATVEC, s);
    note_work(8.0 * ((double)d.N * m + (double)d.N * rL + 2.0 * d.N), 2.0 * d.N * (m + rL));
    const size_t sm = (size_t)(rL + m) * sizeof(double);
    const int th = m >= 256 ? 256 : ((m + 31) / 32) * 32;
    { mv1_leaf_apply_kernel<<<(unsigned)nleaf, th, sm, s>>>(m, L, r, D, U, d.ldu, x, S, y); note_launches(1); }
  }
  return cudaGetLastError();
}

}  // namespace hodlr
