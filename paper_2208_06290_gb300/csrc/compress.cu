// GPU construction of the HODLR approximation of a kernel or boundary-integral
// matrix (Sec. 2.2): leaf blocks evaluated exactly (FP64), every off-diagonal
// sibling block A(I_alpha, I_beta) compressed to the fixed rank r by a
// partial-pivoted cross approximation (the approximate partial-pivoted LU the
// paper's kernel experiments used for this step on the CPU):
//
//   i_0 = first row of the block;  for k = 0 .. r-1:
//     rho(j)  = M(i_k, j) - sum_{l<k} u_l(i_k) v_l(j)          (residual row)
//     j_k     = argmax over unused j of |rho(j)|  (first maximum)
//     v_k     = rho / rho(j_k)
//     u_k(i)  = M(i, j_k) - sum_{l<k} u_l(i) v_l(j_k)         (residual column)
//     i_{k+1} = argmax over rows other than i_0 .. i_k of |u_k(i)|
//   A(I_alpha, I_beta) ~= sum_k u_k v_k^T = U_alpha V_beta^T.
//
// A residual that vanishes (rank exhausted) ends the block: its remaining u, v
// are zero. Kernel matrices are symmetric: one cross per sibling pair gives
// A(I_beta, I_alpha) = V_beta U_alpha^T, so U_big = V_big. The BIE matrix is
// not: both blocks of a pair are compressed.
//
// GPU form: all blocks of a level advance together, two launches per rank
// step: (1) one thread per column position forms the residual row of its
// block and the blocks' pivot columns are chosen by 64-bit atomic maxima of
// (|rho| bits, -j) keys (order-independent, so the choice is deterministic:
// largest |rho|, then the lowest column); (2) one thread per position forms
// v_k from the stored row and u_k of its block and chooses the next pivot
// rows the same way. Entries are rounded to FP32 (evaluated from FP64
// geometry), the residual updates are FP32 (from FP32 working copies of U and
// V); U and V are stored in FP64.
#include <cmath>
#include <vector>

#include "hodlr_internal.cuh"

namespace hodlr {
namespace {

struct Kern {
  int kind;        // hodlr_kernel
  int dim;
  const double* pts;  // N x dim, row-major
  double scale, nugget;
  int64_t N;
  float tol;       // stop a block once |pivot_k| <= tol |pivot_0| (0: fixed rank)
};

// A step is live when its residual row had a nonzero entry and (after the
// first step) its pivot is above the block's tolerance.
__device__ __forceinline__ bool step_live(unsigned long long ck, int k, float tol, const float* delta0,
                                          int64_t blk) {
  if ((ck >> 32) <= 1ull) return false;  // empty key or a vanishing residual
  if (k == 0 || tol <= 0.f) return true;
  const float piv = __uint_as_float((uint32_t)(ck >> 32) - 1u);
  return piv > tol * delta0[blk];
}

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr int kGeo = 6;  // BIE geometry per point: x, y, normal (2), weight, curvature
constexpr size_t kWsAlign = 256;  // every workspace piece starts 256-byte aligned
inline size_t ws_align(size_t x) { return (x + kWsAlign - 1) / kWsAlign * kWsAlign; }

// Star curve rho(t) = 1 + 0.3 cos(5 t), t_i = 2 pi i / N (trapezoid rule):
// point, outward unit normal, weight w_i = |gamma'(t_i)| 2 pi / N and
// curvature, in FP64.
__device__ __forceinline__ void star_point(int64_t i, int64_t N, double& x, double& y, double& nx, double& ny,
                                           double& w, double& kappa) {
  const double t = (double)i * (kTwoPi / (double)N);
  const double rho = 1.0 + 0.3 * cos(5.0 * t), drho = -1.5 * sin(5.0 * t), ddrho = -7.5 * cos(5.0 * t);
  const double c = cos(t), s = sin(t);
  x = rho * c;
  y = rho * s;
  const double tx = drho * c - rho * s, ty = drho * s + rho * c;
  const double sp = sqrt(tx * tx + ty * ty);
  nx = ty / sp;
  ny = -tx / sp;
  w = sp * (kTwoPi / (double)N);
  kappa = (rho * rho + 2.0 * drho * drho - rho * ddrho) / pow(rho * rho + drho * drho, 1.5);
}

// Entry A(i, j), i != j (off-diagonal blocks), returned in FP32. The BIE
// entry is evaluated in FP64 from the FP64 geometry (x, y, normal, weight
// per point): for neighbouring points n(y).(x - y) is second order in the
// spacing while x - y is first order, so FP32 coordinates would lose most of
// its digits. The kernels take the squared distance in FP64 and the
// exponential in FP32.
__device__ __forceinline__ float kernel_entry(const Kern& K, const double* __restrict__ g, int64_t i, int64_t j) {
  if (K.kind == HODLR_KERNEL_BIE_STAR) {
    // double layer: n(y).(x - y) / (2 pi |x - y|^2) w_y   (x = point i, y = point j)
    const double* gi = g + kGeo * i;
    const double* gj = g + kGeo * j;
    const double dx = gi[0] - gj[0], dy = gi[1] - gj[1];
    return (float)((gj[2] * dx + gj[3] * dy) / (kTwoPi * (dx * dx + dy * dy)) * gj[4]);
  }
  double d2 = 0.0;
  for (int a = 0; a < K.dim; ++a) {
    const double d = g[(size_t)K.dim * i + a] - g[(size_t)K.dim * j + a];
    d2 = fma(d, d, d2);
  }
  if (K.kind == HODLR_KERNEL_GAUSSIAN) return expf((float)(-d2 / (2.0 * K.scale * K.scale)));
  const float a = (float)(1.7320508075688772 * sqrt(d2) / K.scale);  // Matern-3/2
  return (1.f + a) * expf(-a);
}

__global__ void geometry_kernel(Kern K, double* __restrict__ g) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < K.N; i += (int64_t)gridDim.x * blockDim.x) {
    if (K.kind == HODLR_KERNEL_BIE_STAR) {
      double x, y, nx, ny, w, kap;
      star_point(i, K.N, x, y, nx, ny, w, kap);
      double* gi = g + kGeo * i;
      gi[0] = x;
      gi[1] = y;
      gi[2] = nx;
      gi[3] = ny;
      gi[4] = w;
      gi[5] = kap;
    } else {
      for (int a = 0; a < K.dim; ++a) g[(size_t)K.dim * i + a] = K.pts[(size_t)K.dim * i + a];
    }
  }
}

// Leaf blocks D_b (column-major m x m), FP64, from the FP64 geometry: BIE:
// the kernel off the diagonal and the smooth-quadrature diagonal
// -1/2 - w_i kappa_i / (4 pi); kernel matrices: k(|x_i - x_j|) + nugget on
// the diagonal.
__global__ void leaf_eval_kernel(Kern K, const double* __restrict__ g, int m, double* __restrict__ D) {
  const int64_t total = K.N * (int64_t)m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / ((int64_t)m * m);
    const int rem = (int)(e % ((int64_t)m * m));
    const int jj = rem / m, ii = rem % m;
    const int64_t i = b * m + ii, j = b * m + jj;
    double v;
    if (K.kind == HODLR_KERNEL_BIE_STAR) {
      const double* gi = g + kGeo * i;
      const double* gj = g + kGeo * j;
      if (i == j) {
        v = -0.5 - gi[4] * gi[5] / (2.0 * kTwoPi);
      } else {
        const double dx = gi[0] - gj[0], dy = gi[1] - gj[1];
        v = (gj[2] * dx + gj[3] * dy) / (kTwoPi * (dx * dx + dy * dy)) * gj[4];
      }
    } else {
      double d2 = 0.0;
      for (int a = 0; a < K.dim; ++a) {
        const double d = g[(size_t)K.dim * i + a] - g[(size_t)K.dim * j + a];
        d2 += d * d;
      }
      if (K.kind == HODLR_KERNEL_GAUSSIAN) {
        v = exp(-d2 / (2.0 * K.scale * K.scale));
      } else {
        const double a = sqrt(3.0) * sqrt(d2) / K.scale;
        v = (1.0 + a) * exp(-a);
      }
      if (i == j) v += K.nugget;
    }
    D[e] = v;
  }
}

// key = (|x| bits << 32) | (0xffffffff - local index): the atomic maximum is
// the largest |x|, then the lowest index. NaN ranks above every number.
__device__ __forceinline__ unsigned long long abs_key(float x, int64_t local) {
  uint32_t ab = __float_as_uint(x) & 0x7fffffffu;
  if (ab > 0x7f800000u) ab = 0x7f800000u;
  return ((unsigned long long)(ab + 1u) << 32) | (unsigned long long)(0xffffffffu - (uint32_t)local);
}
__device__ __forceinline__ int64_t key_index(unsigned long long key) {
  return (int64_t)(0xffffffffu - (uint32_t)(key & 0xffffffffull));
}

// Warp-aggregated atomic max of per-lane keys into keys[blk] (lanes of the
// warp may belong to different blocks).
__device__ __forceinline__ void key_max(unsigned long long* keys, int64_t blk, unsigned long long key, bool valid) {
  const unsigned mask = __ballot_sync(0xffffffffu, valid);
  if (!valid) return;
  const int64_t b0 = __shfl_sync(mask, blk, __ffs(mask) - 1);
  const bool same = __all_sync(mask, blk == b0);
  if (same && mask == 0xffffffffu) {
    unsigned long long k = key;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long t = __shfl_xor_sync(0xffffffffu, k, o);
      k = t > k ? t : k;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(keys + blk, k);
  } else {
    atomicMax(keys + blk, key);
  }
}

// Step (1): residual rows rho of every block's current pivot row, and the
// pivot columns. Thread per column position g (node beta = g / n is the
// column set of block beta ^ 1).
__global__ void aca_row_kernel(Kern K, const double* __restrict__ geo, int64_t n, int c, int r, int k, int sym,
                               const float* __restrict__ U32, const float* __restrict__ V32, float* __restrict__ rho,
                               const int* __restrict__ prow, const int* __restrict__ pcol,
                               unsigned long long* __restrict__ colkey) {
  const int64_t N = K.N;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g - threadIdx.x < N;
       g += (int64_t)gridDim.x * blockDim.x) {
    const bool in = g < N;
    const int64_t gg = in ? g : N - 1;
    const int64_t beta = gg / n, blk = beta ^ 1;
    const bool active = in && (!sym || (blk & 1) == 0);
    float x = 0.f;
    unsigned long long key = 0;
    if (active) {
      const int64_t jl = gg - beta * n;
      const int ik = prow[(size_t)blk * r + k];  // local pivot row of this step; -1: block exhausted
      if (ik >= 0) {
        const int64_t gi = blk * n + ik;
        x = kernel_entry(K, geo, gi, gg);
        for (int l = 0; l < k; ++l) x -= U32[(size_t)l * N + gi] * V32[(size_t)l * N + gg];
        bool used = false;
        for (int l = 0; l < k; ++l) used |= pcol[(size_t)blk * r + l] == (int)jl;
        key = used ? 0ull : abs_key(x, jl);
      }
      rho[gg] = x;
    }
    key_max(colkey, blk, key, active);
  }
}

// Step (2): v_k of every block from its residual row and pivot, u_k (residual
// column at the pivot column) and the next pivot rows. Thread per position g:
// as a row of node alpha = g / n (block alpha) it forms u_k(g); as a column
// of node beta = g / n (block beta ^ 1) it forms v_k(g).
__global__ void aca_col_kernel(Kern K, const double* __restrict__ geo, int64_t n, int c, int r, int k, int sym,
                               float* __restrict__ U32, float* __restrict__ V32, const float* __restrict__ rho,
                               int* __restrict__ prow, int* __restrict__ pcol,
                               const unsigned long long* __restrict__ colkey, unsigned long long* __restrict__ rowkey,
                               double* __restrict__ Ub, double* __restrict__ Vb, int64_t ldu, int64_t ldv,
                               float* __restrict__ delta0) {
  const int64_t N = K.N;
  const int colblk = (c - 1) * r + k;  // column of U_big / V_big
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g - threadIdx.x < N;
       g += (int64_t)gridDim.x * blockDim.x) {
    const bool in = g < N;
    const int64_t gg = in ? g : N - 1;
    const int64_t node = gg / n;
    // v_k at column gg (block node ^ 1)
    {
      const int64_t blk = node ^ 1;
      if (in && (!sym || (blk & 1) == 0)) {
        const unsigned long long ck = colkey[blk];
        const bool live = step_live(ck, k, K.tol, delta0, blk);  // ck is 0 for a finished block
        // rho of block blk lives on node = blk ^ 1's positions
        const float piv = live ? rho[node * n + key_index(ck)] : 0.f;
        const float v = piv != 0.f ? rho[gg] / piv : 0.f;
        V32[(size_t)k * N + gg] = v;
        if (sym) {
          Ub[(size_t)colblk * ldu + gg] = (double)v;  // U(I_beta) = V(I_beta) for a symmetric kernel
          Vb[(size_t)colblk * ldv + gg] = (double)v;
        } else {
          Vb[(size_t)colblk * ldv + gg] = (double)v;
        }
      }
    }
    // u_k at row gg (block node)
    const int64_t blk = node;
    const bool active = in && (!sym || (blk & 1) == 0);
    unsigned long long key = 0;
    if (active) {
      const unsigned long long ck = colkey[blk];
      const bool live = step_live(ck, k, K.tol, delta0, blk);
      const int64_t jk = key_index(ck);
      const int64_t gj = (blk ^ 1) * n + jk;
      const int64_t il = gg - blk * n;
      float u = 0.f;
      if (live) {  // rows and columns of an off-diagonal block are disjoint
        u = kernel_entry(K, geo, gg, gj);
        for (int l = 0; l < k; ++l) u -= U32[(size_t)l * N + gg] * V32[(size_t)l * N + gj];
      }
      U32[(size_t)k * N + gg] = u;
      Ub[(size_t)colblk * ldu + gg] = (double)u;
      if (sym) Vb[(size_t)colblk * ldv + gg] = (double)u;
      bool used = false;
      for (int l = 0; l <= k; ++l) used |= prow[(size_t)blk * r + l] == (int)il;
      key = (used || !live) ? 0ull : abs_key(u, il);
      if (il == 0) {
        pcol[(size_t)blk * r + k] = live ? (int)jk : -1;
        if (k == 0) delta0[blk] = live ? __uint_as_float((uint32_t)(ck >> 32) - 1u) : 0.f;
      }
    }
    key_max(rowkey, blk, key, active);
  }
}

// Next pivot rows from the row keys; a block whose residual vanished or fell
// below the tolerance is marked done (-1) and its remaining u, v are zero.
__global__ void aca_next_row_kernel(int64_t nblk, int r, int k, const unsigned long long* __restrict__ rowkey,
                                    int* __restrict__ prow) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long key = rowkey[b];
    prow[(size_t)b * r + k + 1] = key ? (int)key_index(key) : -1;  // -1: block done
  }
}

// Rank of every block of a level: its live steps (pivot column >= 0).
__global__ void aca_ranks_kernel(int64_t nblk, int r, const int* __restrict__ pcol, int32_t* __restrict__ ranks) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += (int64_t)gridDim.x * blockDim.x) {
    int k = 0;
    while (k < r && pcol[(size_t)b * r + k] >= 0) ++k;
    ranks[b] = k;
  }
}

unsigned grid_n(int64_t N) {
  int64_t b = (N + 255) / 256;
  return (unsigned)(b < 152 * 16 ? b : 152 * 16);
}

}  // namespace

size_t compress_workspace_bytes(const hodlr_desc& d) {
  const size_t N = (size_t)d.N, r = (size_t)d.r;
  size_t off = 0;
  auto take = [&](size_t bytes) { off += ws_align(bytes); };
  take(N * kGeo * sizeof(double));      // FP64 geometry / points
  take(2 * N * r * sizeof(float));      // FP32 working copies of one level's U, V columns
  take(N * sizeof(float));              // residual rows
  take(2 * r * ((size_t)1 << d.L) * sizeof(unsigned long long));  // column / row keys of every step
  take(2 * r * ((size_t)1 << d.L) * sizeof(int));                 // pivot rows / columns
  take(((size_t)1 << d.L) * sizeof(float));                       // first pivots of one level's blocks
  return off;
}

}  // namespace hodlr

using namespace hodlr;

extern "C" hodlr_status hodlr_compress_workspace_size(const hodlr_desc* desc, size_t* bytes) {
  hodlr_status st = check_desc_ext(desc);
  if (st != HODLR_OK) return st;
  if (!bytes) return HODLR_ERR_ARG;
  *bytes = compress_workspace_bytes(*desc);
  return HODLR_OK;
}

extern "C" hodlr_status hodlr_compress(const hodlr_desc* desc, const hodlr_kernel_desc* kern, double* D, double* U,
                                       double* V, int32_t* pivots, int32_t* ranks, void* workspace,
                                       size_t workspace_bytes, hodlr_stream_t stream) {
  hodlr_status st = check_desc_ext(desc);
  if (st != HODLR_OK) return st;
  if (!kern || !D || !U || !V) return HODLR_ERR_ARG;
  if (kern->kind != HODLR_KERNEL_BIE_STAR && kern->kind != HODLR_KERNEL_GAUSSIAN &&
      kern->kind != HODLR_KERNEL_MATERN32)
    return HODLR_ERR_ARG;
  if (kern->kind != HODLR_KERNEL_BIE_STAR && (!kern->points || kern->dim < 1 || kern->dim > 3 || !(kern->scale > 0.0)))
    return HODLR_ERR_ARG;
  if (!(kern->tol >= 0.0 && kern->tol < 1.0)) return HODLR_ERR_ARG;
  if (desc->N >= ((int64_t)1 << 31)) return HODLR_ERR_ARG;  // local indices are 32-bit
  const hodlr_desc& d = *desc;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kWsAlign) || workspace_bytes < compress_workspace_bytes(d))
    return HODLR_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t N = d.N;
  const int r = d.r, L = d.L;
  char* w = static_cast<char*>(workspace);
  size_t off = 0;
  auto take = [&](size_t bytes) { char* p = w + off; off += ws_align(bytes); return p; };
  double* geo = reinterpret_cast<double*>(take((size_t)N * kGeo * sizeof(double)));
  float* U32 = reinterpret_cast<float*>(take((size_t)N * r * sizeof(float)));
  float* V32 = reinterpret_cast<float*>(take((size_t)N * r * sizeof(float)));
  float* rho = reinterpret_cast<float*>(take((size_t)N * sizeof(float)));
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(
      take(2 * (size_t)r * ((size_t)1 << L) * sizeof(unsigned long long)));
  int* piv = reinterpret_cast<int*>(take(2 * (size_t)r * ((size_t)1 << L) * sizeof(int)));
  float* delta0 = reinterpret_cast<float*>(take(((size_t)1 << L) * sizeof(float)));
  Kern K{kern->kind, kern->kind == HODLR_KERNEL_BIE_STAR ? 2 : kern->dim, kern->points, kern->scale,
         kern->nugget, N, (float)kern->tol};
  const int sym = kern->kind == HODLR_KERNEL_BIE_STAR ? 0 : 1;
  ProfScope prof_(KC_COMPRESS, s);
  note_work(8.0 * (double)N * d.m + 16.0 * (double)N * r * L, 2.0 * (double)N * r * r * L);
  geometry_kernel<<<grid_n(N), 256, 0, s>>>(K, geo);
  note_launches(1);
  {
    const int64_t tot = N * (int64_t)d.m;
    int64_t gb = (tot + 255) / 256;
    if (gb > 152 * 32) gb = 152 * 32;
    leaf_eval_kernel<<<(unsigned)gb, 256, 0, s>>>(K, geo, d.m, D);
    note_launches(1);
  }
  if (cudaGetLastError() != cudaSuccess) return HODLR_ERR_CUDA;
  for (int c = 1; c <= L; ++c) {
    const int64_t n = N >> c;
    const int64_t nblk = (int64_t)1 << c;
    unsigned long long* colkey = keys;                        // [r][nblk]
    unsigned long long* rowkey = keys + (size_t)r * nblk;     // [r][nblk]
    int* prow = piv;                                          // [nblk][r]
    int* pcol = piv + (size_t)r * nblk;                       // [nblk][r]
    if (cudaMemsetAsync(keys, 0, 2 * (size_t)r * nblk * sizeof(unsigned long long), s) != cudaSuccess ||
        cudaMemsetAsync(piv, 0, 2 * (size_t)r * nblk * sizeof(int), s) != cudaSuccess)
      return HODLR_ERR_CUDA;
    for (int k = 0; k < r; ++k) {
      aca_row_kernel<<<grid_n(N), 256, 0, s>>>(K, geo, n, c, r, k, sym, U32, V32, rho, prow, pcol,
                                               colkey + (size_t)k * nblk);
      aca_col_kernel<<<grid_n(N), 256, 0, s>>>(K, geo, n, c, r, k, sym, U32, V32, rho, prow, pcol,
                                               colkey + (size_t)k * nblk, rowkey + (size_t)k * nblk, U, V, d.ldu,
                                               d.ldv, delta0);
      note_launches(2);
      if (k + 1 < r) {
        aca_next_row_kernel<<<(unsigned)((nblk + 255) / 256), 256, 0, s>>>(nblk, r, k, rowkey + (size_t)k * nblk,
                                                                           prow);
        note_launches(1);
      }
    }
    if (ranks) {  // ranks of level c's blocks at offset 2^c - 2
      aca_ranks_kernel<<<(unsigned)((nblk + 255) / 256), 256, 0, s>>>(nblk, r, pcol, ranks + (nblk - 2));
      note_launches(1);
    }
    if (pivots) {
      // pivots of level c: [block][k] rows, then [block][k] columns (local indices)
      int32_t* pl = pivots + (size_t)2 * r * (((int64_t)1 << c) - 2);
      if (cudaMemcpyAsync(pl, piv, 2 * (size_t)r * nblk * sizeof(int), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return HODLR_ERR_CUDA;
    }
    if (cudaGetLastError() != cudaSuccess) return HODLR_ERR_CUDA;
  }
  return HODLR_OK;
}

// ---------------------------------------------------------------------------
// Variable ranks per level (Eq. e:u with per-level widths): the ragged U_big
// / V_big hold level c's bases in columns off_c .. off_c + r_c - 1, each
// node's basis left-aligned (a node of lower rank has zero columns at the
// right). The same matrix in the uniform layout of width r >= max r_c has the
// level blocks zero-padded on the right, which every other entry point takes.
namespace hodlr {
namespace {

__global__ void pack_level_ranks_kernel(int64_t N, int r, int L, const int* __restrict__ lr,
                                        const int* __restrict__ off, const double* __restrict__ Ur, int64_t ldur,
                                        const double* __restrict__ Vr, int64_t ldvr, double* __restrict__ U,
                                        int64_t ldu, double* __restrict__ V, int64_t ldv) {
  const int col = blockIdx.y;  // uniform column (c - 1) r + j
  const int c = col / r + 1, j = col % r;
  const bool live = j < lr[c - 1];
  const int64_t src = live ? (int64_t)(off[c - 1] + j) : 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    U[(int64_t)col * ldu + i] = live ? Ur[src * ldur + i] : 0.0;
    V[(int64_t)col * ldv + i] = live ? Vr[src * ldvr + i] : 0.0;
  }
}

}  // namespace
}  // namespace hodlr

extern "C" hodlr_status hodlr_pack_level_ranks(const hodlr_desc* desc, const int32_t* level_ranks, const double* Ur,
                                               int64_t ldur, const double* Vr, int64_t ldvr, double* U, double* V,
                                               void* workspace, size_t workspace_bytes, hodlr_stream_t stream) {
  hodlr_status st = check_desc_ext(desc);
  if (st != HODLR_OK) return st;
  const hodlr_desc& d = *desc;
  if (!level_ranks || !Ur || !Vr || !U || !V || ldur < d.N || ldvr < d.N) return HODLR_ERR_ARG;
  std::vector<int> lr(d.L), off(d.L);
  int tot = 0;
  for (int c = 0; c < d.L; ++c) {
    if (level_ranks[c] < 0 || level_ranks[c] > d.r) return HODLR_ERR_ARG;
    lr[c] = level_ranks[c];
    off[c] = tot;
    tot += lr[c];
  }
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kWsAlign) ||
      workspace_bytes < 2 * (size_t)d.L * sizeof(int))
    return HODLR_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int* dlr = static_cast<int*>(workspace);
  int* doff = dlr + d.L;
  std::vector<int> h(2 * d.L);
  for (int c = 0; c < d.L; ++c) {
    h[c] = lr[c];
    h[d.L + c] = off[c];
  }
  if (cudaMemcpyAsync(dlr, h.data(), h.size() * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return HODLR_ERR_CUDA;
  {
    ProfScope prof_(KC_VECTOR, s);
    note_work(16.0 * (double)d.N * (tot + d.r * d.L), 0.0);
    pack_level_ranks_kernel<<<dim3(grid_n(d.N), d.r * d.L), 256, 0, s>>>(d.N, d.r, d.L, dlr, doff, Ur, ldur, Vr,
                                                                         ldvr, U, d.ldu, V, d.ldv);
    note_launches(1);
  }
  // the host vector must outlive the asynchronous copy
  if (cudaStreamSynchronize(s) != cudaSuccess) return HODLR_ERR_CUDA;
  return cudaGetLastError() == cudaSuccess ? HODLR_OK : HODLR_ERR_CUDA;
}
