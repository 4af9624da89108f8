// Level stage of the factorization and solves (Alg. 1 / Alg. 3 level loop,
// Alg. 2 / Alg. 4 level loop): projections onto the level's bases, the 2r x 2r
// coupling systems and the rank-r updates.
#include "gj.cuh"

namespace hodlr {

template <typename T> struct AccOf { using type = float; };
template <> struct AccOf<double> { using type = double; };

// ---------------------------------------------------------------------------
// Projection partials. For child level c and chunk q (rows [q*ch, (q+1)*ch)),
// P[q] (r x ncols, ld r, FP64) = Bas(rows, block)^T * R(rows, 0:ncols).
// CTA = one chunk x 64 columns; the chunk is streamed 32 rows at a time
// through shared memory and every thread keeps an (RT/16) x 4 register tile.
template <typename TB, typename TR, typename TA, int RT>
__global__ void __launch_bounds__(256) project_kernel(int64_t N, int r, int c, const TB* __restrict__ Bas,
                                                      int64_t ldb, int bas_block, const TR* __restrict__ R,
                                                      int64_t ldr, int ncols, double* __restrict__ P) {
  constexpr int NV = RT / 16;
  __shared__ TA sB[32][RT + 1];
  __shared__ TA sR[32][64 + 1];
  const int64_t ch = chunk_rows(N, c);
  const int64_t q = blockIdx.x;
  const int64_t row0 = q * ch;
  const int j0 = blockIdx.y * 64;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const TB* B0 = Bas + (int64_t)bas_block * r * ldb + row0;
  const TR* R0 = R + row0;
  TA acc[NV][4];
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[v][u] = TA(0);
  for (int64_t k0 = 0; k0 < ch; k0 += 32) {
    const int kn = (ch - k0) < 32 ? (int)(ch - k0) : 32;
    for (int e = tid; e < 32 * RT; e += 256) {
      const int kk = e & 31, col = e >> 5;
      sB[kk][col] = (col < r && kk < kn) ? conv<TA>(B0[(int64_t)col * ldb + k0 + kk]) : TA(0);
    }
    for (int e = tid; e < 32 * 64; e += 256) {
      const int kk = e & 31, col = e >> 5;
      sR[kk][col] = (j0 + col < ncols && kk < kn) ? conv<TA>(R0[(int64_t)(j0 + col) * ldr + k0 + kk]) : TA(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      TA bv[NV], rv[4];
#pragma unroll
      for (int v = 0; v < NV; ++v) bv[v] = sB[kk][ty + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u) rv[u] = sR[kk][tx + 16 * u];
#pragma unroll
      for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[v][u] += bv[v] * rv[u];
    }
    __syncthreads();
  }
  double* Pq = P + (size_t)q * r * ncols;
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int row = ty + 16 * v, col = j0 + tx + 16 * u;
      if (row < r && col < ncols) Pq[(size_t)col * r + row] = (double)acc[v][u];
    }
}

// Skinny variant for ncols <= 8 (solves and residuals with few right-hand
// sides): thread t streams rows row0+t, row0+t+256, ... of the chunk and keeps
// a 16 x KC register tile for basis columns j0..j0+15; the 256 partial tiles
// are reduced by warp shuffles and then across warps in a fixed order.
template <typename TB, typename TR, typename TA, int KC>
__global__ void __launch_bounds__(256) project_skinny_kernel(int64_t N, int r, int c, const TB* __restrict__ Bas,
                                                             int64_t ldb, int bas_block, const TR* __restrict__ R,
                                                             int64_t ldr, int ncols, double* __restrict__ P) {
  __shared__ TA sred[8][16 * KC];
  const int64_t ch = chunk_rows(N, c);
  const int64_t q = blockIdx.x;
  const int64_t row0 = q * ch;
  const int j0 = blockIdx.y * 16;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int jn = (r - j0) < 16 ? (r - j0) : 16;
  const TB* B0 = Bas + ((int64_t)bas_block * r + j0) * ldb + row0;
  const TR* R0 = R + row0;
  TA acc[16][KC];
#pragma unroll
  for (int jj = 0; jj < 16; ++jj)
#pragma unroll
    for (int cc = 0; cc < KC; ++cc) acc[jj][cc] = TA(0);
  for (int64_t i = tid; i < ch; i += 256) {
    TA xv[KC];
#pragma unroll
    for (int cc = 0; cc < KC; ++cc) xv[cc] = cc < ncols ? conv<TA>(R0[(int64_t)cc * ldr + i]) : TA(0);
#pragma unroll
    for (int jj = 0; jj < 16; ++jj) {
      if (jj < jn) {
        const TA b = conv<TA>(B0[(int64_t)jj * ldb + i]);
#pragma unroll
        for (int cc = 0; cc < KC; ++cc) acc[jj][cc] += b * xv[cc];
      }
    }
  }
#pragma unroll
  for (int jj = 0; jj < 16; ++jj)
#pragma unroll
    for (int cc = 0; cc < KC; ++cc) {
      TA v = acc[jj][cc];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0) sred[warp][jj * KC + cc] = v;
    }
  __syncthreads();
  if (tid < 16 * KC) {
    const int jj = tid / KC, cc = tid % KC;
    TA v = TA(0);
#pragma unroll
    for (int w = 0; w < 8; ++w) v += sred[w][tid];
    if (jj < jn && cc < ncols) P[(size_t)q * r * ncols + (size_t)cc * r + j0 + jj] = (double)v;
  }
}

// One right-hand side (k = 1): one warp per chunk. Lane l streams rows l,
// l+32, ... of the chunk and accumulates all RT <= 64 basis-column products;
// a butterfly transpose-reduce (31 shuffles per 32 columns) then leaves the
// chunk total of column j in lane j % 32, which writes it. No shared memory,
// no block barrier; fixed summation order.
template <typename TA>
__device__ __forceinline__ TA warp_transpose_reduce32(TA (&v)[32]) {
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

// The same on 16 values: lane l ends with value l % 16 summed over the 16
// lanes of its half-warp.
template <typename TA>
__device__ __forceinline__ TA warp_transpose_reduce16(TA (&v)[16]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int s = 8; s >= 1; s >>= 1) {
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

// One right-hand side: wpc warps (1, 2, 4 or 8) per row chunk, 8 / wpc chunks
// per CTA; warp w of a chunk sums rows [w ch/wpc, (w+1) ch/wpc) (lane l rows
// l, l+32, ...), the transposed butterfly leaves column j's sum in lane j, and
// the chunk's warps are added in a fixed order through shared memory.
template <typename TB, typename TR, typename TA, int RT>
__global__ void __launch_bounds__(256) project_k1_kernel(int64_t N, int r, int c, const TB* __restrict__ Bas,
                                                         int64_t ldb, int bas_block, const TR* __restrict__ R,
                                                         double* __restrict__ P, int wpc) {
  __shared__ TA sPart[8][RT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cpb = 8 / wpc;
  const int sub = warp / wpc, w = warp % wpc;
  const int64_t q = (int64_t)blockIdx.x * cpb + sub;
  const bool active = q < num_chunks(N, c);
  const int64_t ch = chunk_rows(N, c);
  const int64_t rpw = ch / wpc;
  const int64_t row0 = q * ch + w * rpw;
  TA acc[RT];
#pragma unroll
  for (int j = 0; j < RT; ++j) acc[j] = TA(0);
  if (active) {
    const TB* B0 = Bas + (int64_t)bas_block * r * ldb + row0;
    const TR* R0 = R + row0;
    for (int64_t i = lane; i < rpw; i += 32) {
      const TA x = conv<TA>(R0[i]);
#pragma unroll
      for (int j = 0; j < RT; ++j)
        if (j < r) acc[j] += conv<TA>(B0[(int64_t)j * ldb + i]) * x;
    }
  }
#pragma unroll
  for (int g = 0; g < RT / 32; ++g) {
    TA v[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = acc[g * 32 + j];
    sPart[warp][g * 32 + lane] = warp_transpose_reduce32(v);
  }
  __syncthreads();
  if (active && w == 0) {
    double* Pq = P + (size_t)q * r;
    for (int j = lane; j < r; j += 32) {
      TA t = sPart[sub * wpc][j];
      for (int ww = 1; ww < wpc; ++ww) t += sPart[sub * wpc + ww][j];
      Pq[j] = (double)t;
    }
  }
}

// Vector variant of the one-column projection: lane l of a warp covers rows
// 4l .. 4l+3 of each 128-row slab of its range (one 8- or 16-byte access per
// rank column), then the same transposed butterfly and in-order warp sums.
template <typename TB, typename TR, typename TA, int RT>
__global__ void __launch_bounds__(256) project_k1v_kernel(int64_t N, int r, int c, const TB* __restrict__ Bas,
                                                          int64_t ldb, int bas_block, const TR* __restrict__ R,
                                                          double* __restrict__ P, int wpc) {
  __shared__ TA sPart[8][RT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cpb = 8 / wpc;
  const int sub = warp / wpc, w = warp % wpc;
  const int64_t q = (int64_t)blockIdx.x * cpb + sub;
  const bool active = q < num_chunks(N, c);
  const int64_t ch = chunk_rows(N, c);
  const int64_t rpw = ch / wpc;
  const int64_t row0 = q * ch + w * rpw;
  TA acc[RT];
#pragma unroll
  for (int j = 0; j < RT; ++j) acc[j] = TA(0);
  if (active) {
    const TB* B0 = Bas + (int64_t)bas_block * r * ldb + row0 + 4 * lane;
    const TR* R0 = R + row0 + 4 * lane;
    for (int64_t i = 0; i < rpw; i += 128) {
      TA x[4];
      load4(R0 + i, x);
#pragma unroll
      for (int j = 0; j < RT; ++j)
        if (j < r) {
          TA b[4];
          load4(B0 + (int64_t)j * ldb + i, b);
          acc[j] += b[0] * x[0] + b[1] * x[1] + b[2] * x[2] + b[3] * x[3];
        }
    }
  }
#pragma unroll
  for (int g = 0; g < RT / 32; ++g) {
    TA v[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = acc[g * 32 + j];
    sPart[warp][g * 32 + lane] = warp_transpose_reduce32(v);
  }
  __syncthreads();
  if (active && w == 0) {
    double* Pq = P + (size_t)q * r;
    for (int j = lane; j < r; j += 32) {
      TA t = sPart[sub * wpc][j];
      for (int ww = 1; ww < wpc; ++ww) t += sPart[sub * wpc + ww][j];
      Pq[j] = (double)t;
    }
  }
}

// ---------------------------------------------------------------------------
// One right-hand side, low-precision panels (the preconditioner solve of the
// iterative solvers): the level loop of Alg. 2 in two launches per level.
// Rows are handled in 1024-row CTAs, a warp per 128-row slab, lane l rows
// 4l .. 4l+3 (one 8- or 16-byte access per basis column).
//
// solve_k1_level_kernel<UPD, PROJ>: with UPD, x(rows) += Y_own W(node) for the
// update of level cu (W = -K~^{-1}(rows of the node, :) [s_second; s_first],
// from solve_k1_parent_kernel); with PROJ, the projection of level cp on the
// updated x (still in registers): per warp the transposed butterfly leaves the
// slab's partial of basis column j in lane j, and the warps of one part
// (min(n_p, 1024) rows, n_p = N >> cp) add their partials in FP64 in warp
// order, so that each node of level cp has max(n_p / 1024, 1) parts.
// A level kernel reads the own-basis block of level cu and the basis block
// of level cp once: the update of level c and the projection of level c - 1
// share one pass over x. Registers are held to 32 for BF16 panels (eight CTAs
// per SM: the 1024-row CTAs of N = 2^20 then run in one wave).
template <typename TB, bool UPD, bool PROJ>
__global__ void __launch_bounds__(256, sizeof(TB) == 2 ? 8 : 6) solve_k1_level_kernel(int64_t N, int r, int cu, const TB* __restrict__ Yu,
                                                             int64_t ldy, const float* __restrict__ W, int cp,
                                                             const TB* __restrict__ Vp, int64_t ldv,
                                                             float* __restrict__ x, double* __restrict__ parts) {
  __shared__ double sPart[8][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t row = (int64_t)blockIdx.x * 1024 + 4 * threadIdx.x;
  const bool valid = row < N;  // whole warps (N is a multiple of 128)
  float xv[4] = {0.f, 0.f, 0.f, 0.f};
  if (valid) load4(x + row, xv);
  if constexpr (UPD) {
    const int64_t node = row / (N >> cu);  // one node per warp (nodes of >= 128 rows)
    const float wl = (valid && lane < r) ? W[node * r + lane] : 0.f;
    if (valid) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
      for (int j = 0; j < 32; ++j) {
        if (j < r) {
          float b[4];
          load4(Yu + (int64_t)j * ldy + row, b);
          const float w = __shfl_sync(0xffffffffu, wl, j);
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[q] = fmaf(b[q], w, acc[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) xv[q] += acc[q];
      store4(x + row, xv);
    }
  }
  if constexpr (PROJ) {
    // basis columns in two halves of 16 (16 accumulators live at a time):
    // a 16-wide transposed butterfly leaves column h*16 + (l % 16) summed over
    // each half-warp in lane l, and one more exchange adds the two halves
    float t = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float acc[16];
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        const int j = h * 16 + jj;
        acc[jj] = 0.f;
        if (valid && j < r) {
          float b[4];
          load4(Vp + (int64_t)j * ldv + row, b);
          acc[jj] = b[0] * xv[0] + b[1] * xv[1] + b[2] * xv[2] + b[3] * xv[3];
        }
      }
      float th = warp_transpose_reduce16(acc);
      th += __shfl_xor_sync(0xffffffffu, th, 16);
      if ((lane >> 4) == h) t = th;
    }
    const int64_t np = N >> cp;
    const int gw = (int)((np < 1024 ? np : 1024) / 128);  // warps per part
    if (gw == 1) {
      if (valid && lane < r) parts[(size_t)(blockIdx.x * 8 + warp) * r + lane] = (double)t;
    } else {
      sPart[warp][lane] = (double)t;
      __syncthreads();
      if (valid && warp % gw == 0 && lane < r) {
        double a = sPart[warp][lane];
        for (int w2 = 1; w2 < gw; ++w2) a += sPart[warp + w2][lane];
        parts[(size_t)((blockIdx.x * 8 + warp) / gw) * r + lane] = a;
      }
    }
  }
}

// One CTA per parent at level c: the children's projections (sums of their
// ppn parts, fixed order: part q by group q % G of the NT / 32 = G groups,
// then the groups in order), then W = -K~^{-1} [s_second; s_first]
// (Eq. e:k; rows 0..r-1 of the right-hand side from the second child) in
// FP64, rows 0..r-1 for the first child and r..2r-1 for the second, rounded to
// FP32 for the update. NT = 1024 at the top levels (many parts, few parents),
// else 256.
template <int NT>
__global__ void __launch_bounds__(NT) solve_k1_parent_kernel(int r, int64_t ppn, const double* __restrict__ parts,
                                                             const double* __restrict__ Kinv,
                                                             float* __restrict__ W) {
  constexpr int G = NT / 32;   // part groups
  constexpr int KP = NT / 64;  // term groups of the K~^{-1} product
  __shared__ double sSum[G][2][32];
  __shared__ double sRhs[64];
  __shared__ double sW[KP][64];
  const int t = threadIdx.x, lane = t & 31, g = t >> 5;
  const int64_t p = blockIdx.x;
  const int n2 = 2 * r;
  double a0 = 0.0, a1 = 0.0;
  if (lane < r) {
    const double* c0 = parts + (size_t)(2 * p) * ppn * r + lane;
    const double* c1 = parts + (size_t)(2 * p + 1) * ppn * r + lane;
#pragma unroll 4
    for (int64_t q = g; q < ppn; q += G) {
      a0 += c0[(size_t)q * r];
      a1 += c1[(size_t)q * r];
    }
  }
  sSum[g][0][lane] = a0;
  sSum[g][1][lane] = a1;
  __syncthreads();
  if (t < 64) {
    const int ch = t >> 5;  // 0: first child, 1: second
    double s = sSum[0][ch][lane];
#pragma unroll
    for (int gg = 1; gg < G; ++gg) s += sSum[gg][ch][lane];
    if (lane < r) sRhs[ch ? lane : r + lane] = s;  // [s_second; s_first]
  }
  __syncthreads();
  {
    const int o = t & 63, part = t >> 6;  // output row o of K~^{-1}, terms q = part, part + KP, ...
    const double* Kj = Kinv + (size_t)p * n2 * n2;
    double a = 0.0;
    if (o < n2)
      for (int q = part; q < n2; q += KP) a += Kj[(size_t)q * n2 + o] * sRhs[q];
    sW[part][o] = a;
  }
  __syncthreads();
  if (t < n2) {
    double w = sW[0][t];
#pragma unroll
    for (int pp = 1; pp < KP; ++pp) w += sW[pp][t];
    const int ch = t >= r ? 1 : 0;
    W[(size_t)(2 * p + ch) * r + (t - ch * r)] = (float)-w;
  }
}

size_t solve_k1_parts_elems(const hodlr_desc& d) { return (size_t)(d.N / 128) * d.r; }

template <typename TB>
bool solve_k1_supported(const Factor& F, const TB* Y, const TB* Vp, int64_t ldvp, const float* x) {
  const hodlr_desc& d = F.d;
  // leaves of 128 * 2^j rows: every node of every level is a whole number of
  // 128-row warps, and nodes of 1024 rows or more a whole number of parts
  return d.r <= 32 && d.m % 128 == 0 && (d.m & (d.m - 1)) == 0 && d.N % 4 == 0 && ldvp % 4 == 0 &&
         reinterpret_cast<uintptr_t>(Y) % 16 == 0 &&
         reinterpret_cast<uintptr_t>(Vp) % 16 == 0 && reinterpret_cast<uintptr_t>(x) % 16 == 0;
}

template <typename TB>
cudaError_t launch_solve_k1_level(const hodlr_desc& d, bool upd, bool proj, int cu, const TB* Yu, const float* W,
                                  int cp, const TB* Vp, int64_t ldv, float* x, double* parts, cudaStream_t s) {
  const int64_t N = d.N;
  const int r = d.r;
  ProfScope prof_(upd ? KC_UPDATE : KC_PROJECT, s);
  const double pb = proj ? (double)(N / std::min<int64_t>(N >> cp, 1024)) * 8.0 * r : 0.0;
  note_work((upd ? sizeof(TB) * (double)N * r + 4.0 * N + 4.0 * (double)(1ll << cu) * r : 0.0) +
                (proj ? sizeof(TB) * (double)N * r : 0.0) + 4.0 * N + pb,
            (upd ? 2.0 * N * r : 0.0) + (proj ? 2.0 * N * r : 0.0));
  const unsigned g = (unsigned)((N + 1023) / 1024);
  if (upd && proj)
    solve_k1_level_kernel<TB, true, true><<<g, 256, 0, s>>>(N, r, cu, Yu, N, W, cp, Vp, ldv, x, parts);
  else if (upd)
    solve_k1_level_kernel<TB, true, false><<<g, 256, 0, s>>>(N, r, cu, Yu, N, W, cp, Vp, ldv, x, parts);
  else
    solve_k1_level_kernel<TB, false, true><<<g, 256, 0, s>>>(N, r, cu, Yu, N, W, cp, Vp, ldv, x, parts);
  note_launches(1);
  return cudaGetLastError();
}

// Forward solve (Alg. 2 after the leaf stage), one column in FP32 with
// panels TB: the projection of level L, then per level c = L .. 1 the parent
// kernel and the level kernel (update of c with the projection of c - 1).
template <typename TB>
cudaError_t launch_solve_k1_chain(const Factor& F, const TB* Y, const TB* Vp, int64_t ldvp, float* x,
                                  double* parts, float* W, cudaStream_t s) {
  const hodlr_desc& d = F.d;
  const int64_t N = d.N;
  const int r = d.r, L = d.L;
  cudaError_t e;
  if ((e = launch_solve_k1_level<TB>(d, false, true, 0, nullptr, nullptr, L, Vp + (int64_t)(L - 1) * r * ldvp, ldvp,
                                     x, parts, s)) != cudaSuccess)
    return e;
  for (int c = L; c >= 1; --c) {
    const int64_t nc = N >> c;
    const int64_t ppn = nc >= 1024 ? nc / 1024 : 1;
    {
      ProfScope prof_(KC_COUPLING_APPLY, s);
      const int64_t parents = (int64_t)1 << (c - 1);
      note_work(8.0 * (double)(1ll << c) * ppn * r + 8.0 * parents * 4.0 * r * r + 4.0 * (double)(1ll << c) * r,
                parents * 2.0 * (2.0 * r) * (2.0 * r));
      const double* Kc = F.K + F.Koff[c] * 4 * r * r;
      if (ppn >= 64)
        solve_k1_parent_kernel<1024><<<(unsigned)parents, 1024, 0, s>>>(r, ppn, parts, Kc, W);
      else
        solve_k1_parent_kernel<256><<<(unsigned)parents, 256, 0, s>>>(r, ppn, parts, Kc, W);
      note_launches(1);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const TB* Yu = Y + (int64_t)(c - 1) * r * N;
    const TB* Vn = c > 1 ? Vp + (int64_t)(c - 2) * r * ldvp : nullptr;
    if ((e = launch_solve_k1_level<TB>(d, true, c > 1, c, Yu, W, c - 1, Vn, ldvp, x, parts, s)) != cudaSuccess)
      return e;
  }
  return cudaSuccess;
}
template bool solve_k1_supported<__nv_bfloat16>(const Factor&, const __nv_bfloat16*, const __nv_bfloat16*, int64_t,
                                                const float*);
template bool solve_k1_supported<float>(const Factor&, const float*, const float*, int64_t, const float*);
template cudaError_t launch_solve_k1_chain<__nv_bfloat16>(const Factor&, const __nv_bfloat16*, const __nv_bfloat16*,
                                                         int64_t, float*, double*, float*, cudaStream_t);
template cudaError_t launch_solve_k1_chain<float>(const Factor&, const float*, const float*, int64_t, float*, double*,
                                                 float*, cudaStream_t);

int project_k1_warps(int64_t ch) {
  int w = 1;
  while (w < 8 && ch >= (int64_t)256 * w && ch % (2 * w) == 0) w *= 2;  // >= 128 rows per warp
  return w;
}

template <typename TB, typename TR>
cudaError_t launch_project(int64_t N, int r, int c, const TB* Bas, int64_t ldb, int bas_block, const TR* R,
                           int64_t ldr, int ncols, double* P, int acc_fp64, cudaStream_t s) {
  ProfScope prof_(KC_PROJECT, s);
  if (ncols <= 0) return cudaSuccess;
  dim3 grid((unsigned)num_chunks(N, c), (ncols + 63) / 64);
  using TA = typename AccOf<TR>::type;
  note_work(sizeof(TB) * (double)N * r + sizeof(TR) * (double)N * ncols + 8.0 * num_chunks(N, c) * r * ncols,
            2.0 * N * r * (double)ncols);
  if (ncols == 1 && r > 16) {
    const int wpc = project_k1_warps(chunk_rows(N, c));
    const int64_t cpb = 8 / wpc;
    const unsigned g1 = (unsigned)((num_chunks(N, c) + cpb - 1) / cpb);
    const bool vec = (chunk_rows(N, c) / wpc) % 128 == 0 && ldb % 4 == 0 &&
                     reinterpret_cast<uintptr_t>(Bas) % 16 == 0 && reinterpret_cast<uintptr_t>(R) % 16 == 0;
    if (vec && r <= 32)
      { project_k1v_kernel<TB, TR, TA, 32><<<g1, 256, 0, s>>>(N, r, c, Bas, ldb, bas_block, R, P, wpc); note_launches(1); }
    else if (vec)
      { project_k1v_kernel<TB, TR, TA, 64><<<g1, 256, 0, s>>>(N, r, c, Bas, ldb, bas_block, R, P, wpc); note_launches(1); }
    else if (r <= 32)
      { project_k1_kernel<TB, TR, TA, 32><<<g1, 256, 0, s>>>(N, r, c, Bas, ldb, bas_block, R, P, wpc); note_launches(1); }
    else
      { project_k1_kernel<TB, TR, TA, 64><<<g1, 256, 0, s>>>(N, r, c, Bas, ldb, bas_block, R, P, wpc); note_launches(1); }
    return cudaGetLastError();
  }
  if (ncols <= 8) {
    dim3 g2((unsigned)num_chunks(N, c), (r + 15) / 16);
    if (ncols == 1)
      { project_skinny_kernel<TB, TR, TA, 1><<<g2, 256, 0, s>>>(N, r, c, Bas, ldb, bas_block, R, ldr, ncols, P); note_launches(1); }
    else if (ncols <= 2)
      { project_skinny_kernel<TB, TR, TA, 2><<<g2, 256, 0, s>>>(N, r, c, Bas, ldb, bas_block, R, ldr, ncols, P); note_launches(1); }
    else if (ncols <= 4)
      { project_skinny_kernel<TB, TR, TA, 4><<<g2, 256, 0, s>>>(N, r, c, Bas, ldb, bas_block, R, ldr, ncols, P); note_launches(1); }
    else
      { project_skinny_kernel<TB, TR, TA, 8><<<g2, 256, 0, s>>>(N, r, c, Bas, ldb, bas_block, R, ldr, ncols, P); note_launches(1); }
    return cudaGetLastError();
  }
  if (r <= 16)
    { project_kernel<TB, TR, TA, 16><<<grid, 256, 0, s>>>(N, r, c, Bas, ldb, bas_block, R, ldr, ncols, P); note_launches(1); }
  else if (r <= 32)
    { project_kernel<TB, TR, TA, 32><<<grid, 256, 0, s>>>(N, r, c, Bas, ldb, bas_block, R, ldr, ncols, P); note_launches(1); }
  else
    { project_kernel<TB, TR, TA, 64><<<grid, 256, 0, s>>>(N, r, c, Bas, ldb, bas_block, R, ldr, ncols, P); note_launches(1); }
  (void)acc_fp64;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Rank-r update: R(rows, 0:ncols) += alpha * Bas(rows, block) * W(node')
// for a 64-row x 64-column tile (rows of one node). W is FP64 (r x ncols, ld r).
template <typename TB, typename TR, typename TA, int RT>
__global__ void __launch_bounds__(256) update_kernel(int64_t N, int r, int c, const TB* __restrict__ Bas,
                                                     int64_t ldb, int bas_block, TR* __restrict__ R, int64_t ldr,
                                                     int ncols, const double* __restrict__ Wbase, int64_t wstride,
                                                     int swap_sibling, double alpha) {
  constexpr int KT = RT < 32 ? RT : 32;  // inner-dimension tile
  __shared__ TA sB[KT][64 + 1];  // [k][row]
  __shared__ TA sW[KT][64 + 1];  // [k][col]
  // tiles of 64 rows laid out node by node; the last tile of a node is ragged
  const int64_t n = N >> c;
  const int64_t tpn = (n + 63) / 64;
  const int64_t node = blockIdx.x / tpn;
  const int64_t t0 = (blockIdx.x % tpn) * 64;
  const int rt = (n - t0) < 64 ? (int)(n - t0) : 64;
  const int64_t row0 = node * n + t0;
  const double* W = Wbase + (node ^ swap_sibling) * wstride;
  const int j0 = blockIdx.y * 64;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const TB* B0 = Bas + (int64_t)bas_block * r * ldb + row0;
  TA acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = TA(0);
  for (int k0 = 0; k0 < r; k0 += KT) {
    for (int e = tid; e < 64 * KT; e += 256) {
      const int i = e & 63, kk = e >> 6;
      sB[kk][i] = (k0 + kk < r && i < rt) ? conv<TA>(B0[(int64_t)(k0 + kk) * ldb + i]) : TA(0);
    }
    for (int e = tid; e < 64 * KT; e += 256) {
      const int kk = e % KT, col = e / KT;
      sW[kk][col] = (k0 + kk < r && j0 + col < ncols) ? conv<TA>(alpha * W[(size_t)(j0 + col) * r + k0 + kk])
                                                      : TA(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < KT; ++kk) {
      TA bv[4], wv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) bv[a] = sB[kk][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) wv[b] = sW[kk][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += bv[a] * wv[b];
    }
    __syncthreads();
  }
  TR* R0 = R + row0;
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int col = j0 + ty + 16 * b;
    if (col >= ncols) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = tx + 16 * a;
      if (i < rt) {
        TR* p = R0 + (int64_t)col * ldr + i;
        *p = conv<TR>(conv<TA>(*p) + acc[a][b]);
      }
    }
  }
}

// Skinny variant for ncols <= 8: one thread per row, W(node') (times alpha)
// staged in shared memory and read by broadcast; tiles of 256 rows laid out
// node by node.
template <typename TB, typename TR, typename TA, int KC>
__global__ void __launch_bounds__(256) update_skinny_kernel(int64_t N, int r, int c, const TB* __restrict__ Bas,
                                                            int64_t ldb, int bas_block, TR* __restrict__ R,
                                                            int64_t ldr, int ncols, const double* __restrict__ Wbase,
                                                            int64_t wstride, int swap_sibling, double alpha) {
  __shared__ TA sW[64][KC];
  const int64_t n = N >> c;
  const int64_t tpn = (n + 255) / 256;
  const int64_t node = blockIdx.x / tpn;
  const int64_t t0 = (blockIdx.x % tpn) * 256;
  const double* W = Wbase + (node ^ swap_sibling) * wstride;
  for (int e = threadIdx.x; e < r * KC; e += 256) {
    const int j = e / KC, cc = e % KC;
    sW[j][cc] = cc < ncols ? conv<TA>(alpha * W[(size_t)cc * r + j]) : TA(0);
  }
  __syncthreads();
  const int64_t i = t0 + threadIdx.x;
  if (i >= n) return;
  const int64_t row = node * n + i;
  const TB* B0 = Bas + (int64_t)bas_block * r * ldb + row;
  TA acc[KC];
#pragma unroll
  for (int cc = 0; cc < KC; ++cc) acc[cc] = TA(0);
  for (int j = 0; j < r; ++j) {
    const TA b = conv<TA>(B0[(int64_t)j * ldb]);
#pragma unroll
    for (int cc = 0; cc < KC; ++cc) acc[cc] += b * sW[j][cc];
  }
#pragma unroll
  for (int cc = 0; cc < KC; ++cc)
    if (cc < ncols) {
      TR* p = R + (int64_t)cc * ldr + row;
      *p = conv<TR>(conv<TA>(*p) + acc[cc]);
    }
}

// One right-hand side, rows in fours: thread t of a 1024-row tile (tiles laid
// out node by node) updates rows 4t .. 4t+3 with vector loads of the basis
// (one 8- or 16-byte access per rank column) and of x.
template <typename TB, typename TR, typename TA>
__global__ void __launch_bounds__(256) update_k1v_kernel(int64_t N, int r, int c, const TB* __restrict__ Bas,
                                                         int64_t ldb, int bas_block, TR* __restrict__ R,
                                                         const double* __restrict__ Wbase, int64_t wstride,
                                                         int swap_sibling, double alpha) {
  __shared__ TA sW[64];
  const int64_t n = N >> c;
  const int64_t tpn = (n + 1023) / 1024;
  const int64_t node = blockIdx.x / tpn;
  const int64_t t0 = (blockIdx.x % tpn) * 1024;
  const double* W = Wbase + (node ^ swap_sibling) * wstride;
  for (int j = threadIdx.x; j < r; j += 256) sW[j] = conv<TA>(alpha * W[j]);
  __syncthreads();
  const int64_t i = t0 + 4 * threadIdx.x;
  if (i >= n) return;
  const int64_t row = node * n + i;
  const TB* B0 = Bas + (int64_t)bas_block * r * ldb + row;
  TA acc[4] = {TA(0), TA(0), TA(0), TA(0)};
#pragma unroll 8
  for (int j = 0; j < r; ++j) {
    TA b[4];
    load4(B0 + (int64_t)j * ldb, b);
    const TA w = sW[j];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] += b[q] * w;
  }
  TA x[4];
  load4(R + row, x);
#pragma unroll
  for (int q = 0; q < 4; ++q) x[q] += acc[q];
  store4(R + row, x);
}

template <typename TB, typename TR>
cudaError_t launch_update(int64_t N, int r, int c, const TB* Bas, int64_t ldb, int bas_block, TR* R, int64_t ldr,
                          int ncols, const double* Wbase, int64_t wstride, int swap_sibling, double alpha,
                          int acc_fp64, cudaStream_t s) {
  ProfScope prof_(KC_UPDATE, s);
  if (ncols <= 0) return cudaSuccess;
  const int64_t n = N >> c;
  const int64_t tpn = (n + 63) / 64;
  dim3 grid((unsigned)(((int64_t)1 << c) * tpn), (ncols + 63) / 64);
  note_work(sizeof(TB) * (double)N * r + 2.0 * sizeof(TR) * (double)N * ncols + 8.0 * (double)(1ll << c) * r * ncols,
            2.0 * N * r * (double)ncols);
  if (ncols <= 8) {
    using TA2 = typename AccOf<TR>::type;
    const int64_t tpn2 = (n + 255) / 256;
    const unsigned g2 = (unsigned)(((int64_t)1 << c) * tpn2);
    const bool vec1 = ncols == 1 && n % 4 == 0 && ldb % 4 == 0 &&
                      reinterpret_cast<uintptr_t>(Bas) % 16 == 0 && reinterpret_cast<uintptr_t>(R) % 16 == 0;
    if (vec1) {
      const int64_t tpn4 = (n + 1023) / 1024;
      const unsigned g4 = (unsigned)(((int64_t)1 << c) * tpn4);
      { update_k1v_kernel<TB, TR, TA2><<<g4, 256, 0, s>>>(N, r, c, Bas, ldb, bas_block, R, Wbase, wstride, swap_sibling, alpha); note_launches(1); }
    } else if (ncols == 1)
      { update_skinny_kernel<TB, TR, TA2, 1><<<g2, 256, 0, s>>>(N, r, c, Bas, ldb, bas_block, R, ldr, ncols, Wbase, wstride, swap_sibling, alpha); note_launches(1); }
    else if (ncols <= 2)
      { update_skinny_kernel<TB, TR, TA2, 2><<<g2, 256, 0, s>>>(N, r, c, Bas, ldb, bas_block, R, ldr, ncols, Wbase, wstride, swap_sibling, alpha); note_launches(1); }
    else if (ncols <= 4)
      { update_skinny_kernel<TB, TR, TA2, 4><<<g2, 256, 0, s>>>(N, r, c, Bas, ldb, bas_block, R, ldr, ncols, Wbase, wstride, swap_sibling, alpha); note_launches(1); }
    else
      { update_skinny_kernel<TB, TR, TA2, 8><<<g2, 256, 0, s>>>(N, r, c, Bas, ldb, bas_block, R, ldr, ncols, Wbase, wstride, swap_sibling, alpha); note_launches(1); }
    return cudaGetLastError();
  }
  using TA = typename AccOf<TR>::type;
  (void)acc_fp64;
  if (r <= 16)
    { update_kernel<TB, TR, TA, 16><<<grid, 256, 0, s>>>(N, r, c, Bas, ldb, bas_block, R, ldr, ncols, Wbase,
                                                       wstride, swap_sibling, alpha); note_launches(1); }
  else if (r <= 32)
    { update_kernel<TB, TR, TA, 32><<<grid, 256, 0, s>>>(N, r, c, Bas, ldb, bas_block, R, ldr, ncols, Wbase,
                                                       wstride, swap_sibling, alpha); note_launches(1); }
  else
    { update_kernel<TB, TR, TA, 64><<<grid, 256, 0, s>>>(N, r, c, Bas, ldb, bas_block, R, ldr, ncols, Wbase,
                                                       wstride, swap_sibling, alpha); note_launches(1); }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// K4: coupling matrices of the parents of child level c, in FP64.
// K~ = [[I, T_b], [T_a, I]] with T_x = V_x^T Y_x summed over the chunk
// partials of child x (own block = slot columns r(c-1) .. rc-1). Its diagonal
// blocks are identities, so (the pivot-free use of this form) its inverse
// follows from the Schur complement S = I - T_a T_b (r x r):
//   K~^{-1} = [[I + T_b S^{-1} T_a, -T_b S^{-1}], [-S^{-1} T_a, S^{-1}]],
// det K~ = det S. S is inverted in shared memory by Gauss-Jordan with partial
// pivoting (gj.cuh), which also gives log|det S| and its sign.
__global__ void __launch_bounds__(256) coupling_factor_kernel(int64_t N, int r, int c,
                                                              const double* __restrict__ P, int64_t cpn_read,
                                                              double* __restrict__ Kinv,
                                                              double* __restrict__ node_ld, DevStatus* st,
                                                              int64_t heap_first) {
  extern __shared__ double sK[];
  const int lds = r + 1;
  double* Sm = sK;                       // r x r (ld r+1): S, then S^{-1}
  double* Ta = Sm + (size_t)r * lds;     // r x r (ld r)
  double* Tb = Ta + (size_t)r * r;       // r x r (ld r)
  double* M1 = Tb + (size_t)r * r;       // r x r (ld r): S^{-1} T_a, also GJ scratch
  double* scol = M1 + (size_t)r * r;
  double* srow = scol + r;
  double* spv = srow + r;
  int* spiv = reinterpret_cast<int*>(spv + r);
  int* spos = spiv + r;
  __shared__ double s_la;
  __shared__ int s_neg, s_sing;
  const int64_t j = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t cpn = chunks_per_node(N, c);
  const size_t slot = (size_t)r * r * c;
  const int anc = r * (c - 1);
  const int64_t qa = 2 * j * cpn, qb = (2 * j + 1) * cpn;
  for (int e = tid; e < r * r; e += nt) {
    const int row = e % r, col = e / r;
    double a = 0.0, b = 0.0;
    for (int64_t q = 0; q < cpn_read; ++q) {
      a += P[(qa + q) * slot + (size_t)(anc + col) * r + row];
      b += P[(qb + q) * slot + (size_t)(anc + col) * r + row];
    }
    Ta[e] = a;
    Tb[e] = b;
  }
  __syncthreads();
  smem_gemm<double>(r, r, r, -1.0, Ta, r, Tb, r, 0.0, Sm, lds);  // S = -T_a T_b
  __syncthreads();
  for (int e = tid; e < r; e += nt) Sm[(size_t)e * lds + e] += 1.0;  // S = I - T_a T_b
  __syncthreads();
  gj_invert_smem<double>(Sm, r, lds, spiv, spv, scol, srow, spos, &s_la, &s_neg, &s_sing);
  gj_unscramble<double>(Sm, r, lds, spos, M1);
  smem_gemm<double>(r, r, r, 1.0, Sm, lds, Ta, r, 0.0, M1, r);  // M1 = S^{-1} T_a
  __syncthreads();
  const int n = 2 * r;
  double* out = Kinv + (size_t)j * n * n;
  // [11] = I + T_b M1, [12] = -T_b S^{-1}, [21] = -M1, [22] = S^{-1}
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int col = warp; col < n; col += nw) {
    for (int row = lane; row < n; row += 32) {
      double v;
      if (row < r && col < r) {
        double acc = (row == col) ? 1.0 : 0.0;
        for (int t = 0; t < r; ++t) acc += Tb[(size_t)t * r + row] * M1[(size_t)col * r + t];
        v = acc;
      } else if (row < r) {
        double acc = 0.0;
        for (int t = 0; t < r; ++t) acc += Tb[(size_t)t * r + row] * Sm[(size_t)(col - r) * lds + t];
        v = -acc;
      } else if (col < r) {
        v = -M1[(size_t)col * r + (row - r)];
      } else {
        v = Sm[(size_t)(col - r) * lds + (row - r)];
      }
      out[(size_t)col * n + row] = v;
    }
  }
  if (tid == 0) {
    node_ld[2 * j] = s_la;
    node_ld[2 * j + 1] = (s_sing >= 0) ? 0.0 : (s_neg ? -1.0 : 1.0);
    if (s_sing >= 0) set_status(st, HODLR_ERR_SINGULAR_COUPLING, heap_first + j, r + s_sing);
  }
}

cudaError_t launch_coupling_factor(const Factor& F, int c, cudaStream_t s) {
  ProfScope prof_(KC_COUPLING, s);
  const int r = F.d.r;
  const int n = 2 * r;
  const int64_t parents = (int64_t)1 << (c - 1);
  const size_t sm = ((size_t)r * (r + 1) + 3 * (size_t)r * r + 3 * (size_t)r) * sizeof(double) +
                    2 * (size_t)r * sizeof(int);
  if (sm > 48 * 1024)
    cudaFuncSetAttribute(coupling_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  note_work(8.0 * num_chunks(F.d.N, c) * r * r + 8.0 * parents * n * n, parents * 2.0 / 3.0 * n * n * (double)n);
  if (coupling_warp_supported(F)) return launch_coupling_factor_warp(F, c, s);
  { coupling_factor_kernel<<<(unsigned)parents, 256, sm, s>>>(F.d.N, r, c, F.P, F.P_reduced ? 1 : chunks_per_node(F.d.N, c), F.K + F.Koff[c] * n * n,
                                                             F.node_ld + 2 * F.Koff[c], F.status,
                                                             (int64_t)1 << (c - 1)); note_launches(1); }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Coupling application: for every parent and a 32-column tile of the
// right-hand side, out = Kinv * rhs (or Kinv^T * rhs), with
//   rhs = [from first; from second] summed over chunk partials,
//   first = beta, second = alpha   (factor and solve: K~ [w_a; w_b] = [s_b; s_a])
//   first = alpha, second = beta   (adjoint: K~^T t = [s_a; s_b]),
// and out rows 0..r-1 written to alpha's first slot, rows r..2r-1 to beta's.
// Slots are r x sw (ld r); the right-hand side is columns [0, nrhs).
template <typename TA, int NR>
__global__ void __launch_bounds__(256) coupling_apply_kernel(int64_t N, int r, int c, double* P, int64_t sw,
                                                             int nrhs, const double* __restrict__ Kinv,
                                                             int first_is_beta, int trans, int64_t cpn_read) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = 2 * r;
  TA* sKc = reinterpret_cast<TA*>(smem_raw);  // [n][33]: Kinv(i, kb + kk) (or Kinv^T)
  TA* sRhs = sKc + (size_t)n * 33;            // [n][33]: right-hand side, this CTA's columns
  const int64_t j = blockIdx.x;
  const int c0 = blockIdx.y * 32;
  const int tid = threadIdx.x;
  const int col = tid & 31, rg = tid >> 5;
  const int64_t cpn = chunks_per_node(N, c);
  const size_t slot = (size_t)r * sw;
  const int64_t qa = 2 * j * cpn, qb = (2 * j + 1) * cpn;
  const int64_t qfirst = first_is_beta ? qb : qa, qsecond = first_is_beta ? qa : qb;
  const double* Kj = Kinv + (size_t)j * n * n;
  // gather the right-hand side (FP64 sum of the chunk partials)
  for (int e = tid; e < n * 32; e += 256) {
    const int i = e % n, cc = e / n;
    double acc = 0.0;
    if (c0 + cc < nrhs) {
      const int64_t q0 = i < r ? qfirst : qsecond;
      const int row = i < r ? i : i - r;
      for (int64_t q = 0; q < cpn_read; ++q) acc += P[(q0 + q) * slot + (size_t)(c0 + cc) * r + row];
    }
    sRhs[i * 33 + cc] = (TA)acc;
  }
  TA acc[NR];
#pragma unroll
  for (int a = 0; a < NR; ++a) acc[a] = TA(0);
  for (int kb = 0; kb < n; kb += 32) {
    __syncthreads();
    for (int e = tid; e < n * 32; e += 256) {
      const int i = e % n, kk = e / n;
      const int kg = kb + kk;
      double v = 0.0;
      if (kg < n) v = trans ? Kj[(size_t)i * n + kg] : Kj[(size_t)kg * n + i];
      sKc[i * 33 + kk] = (TA)v;
    }
    __syncthreads();
    const int kn = min(32, n - kb);
    for (int kk = 0; kk < kn; ++kk) {
      const TA xv = sRhs[(kb + kk) * 33 + col];
#pragma unroll
      for (int a = 0; a < NR; ++a) {
        const int i = rg + 8 * a;
        if (i < n) acc[a] += sKc[i * 33 + kk] * xv;
      }
    }
  }
  __syncthreads();  // every CTA reads all its partials before any write below
  if (c0 + col < nrhs) {
#pragma unroll
    for (int a = 0; a < NR; ++a) {
      const int i = rg + 8 * a;
      if (i < n) {
        const int64_t q = i < r ? qa : qb;
        const int row = i < r ? i : i - r;
        P[q * slot + (size_t)(c0 + col) * r + row] = (double)acc[a];
      }
    }
  }
}

template <typename TA>
static cudaError_t coupling_apply(int64_t N, int r, int c, double* P, int64_t sw, int nrhs, const double* Kinv,
                                  int first_is_beta, int trans, cudaStream_t s, int64_t cpn_read = -1) {
  if (cpn_read < 0) cpn_read = chunks_per_node(N, c);
  if (nrhs <= 0) return cudaSuccess;
  dim3 grid(1u << (c - 1), (nrhs + 31) / 32);
  const int n = 2 * r;
  const double parents = (double)(1ll << (c - 1));
  note_work(8.0 * ((double)num_chunks(N, c) * r * nrhs + parents * n * n + 2.0 * parents * r * nrhs),
            parents * 2.0 * n * n * (double)nrhs);
  const size_t sm = (size_t)2 * n * 33 * sizeof(TA);
  if (n <= 32) {
    { coupling_apply_kernel<TA, 4><<<grid, 256, sm, s>>>(N, r, c, P, sw, nrhs, Kinv, first_is_beta, trans, cpn_read); note_launches(1); }
  } else if (n <= 64) {
    { coupling_apply_kernel<TA, 8><<<grid, 256, sm, s>>>(N, r, c, P, sw, nrhs, Kinv, first_is_beta, trans, cpn_read); note_launches(1); }
  } else {
    cudaFuncSetAttribute(coupling_apply_kernel<TA, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    { coupling_apply_kernel<TA, 16><<<grid, 256, sm, s>>>(N, r, c, P, sw, nrhs, Kinv, first_is_beta, trans, cpn_read); note_launches(1); }
  }
  return cudaGetLastError();
}

cudaError_t launch_coupling_apply_any(const Factor& F, int c, double* P, int64_t sw, int nrhs, int first_is_beta,
                                      int trans, cudaStream_t s) {
  ProfScope prof_(KC_COUPLING_APPLY, s);
  const int r = F.d.r;
  const double* Kc = F.K + F.Koff[c] * 4 * r * r;
  return coupling_apply<double>(F.d.N, r, c, P, sw, nrhs, Kc, first_is_beta, trans, s);
}

// Factor: W' = Kinv [W_beta; W_alpha] for the ancestor columns of every parent.
cudaError_t launch_coupling_factor_apply(const Factor& F, int c, cudaStream_t s) {
  ProfScope prof_(KC_COUPLING_APPLY, s);
  const int r = F.d.r;
  const int anc = r * (c - 1);
  const double* Kc = F.K + F.Koff[c] * 4 * r * r;
  const int64_t cr = F.P_reduced ? 1 : chunks_per_node(F.d.N, c);
  if (F.prec == HODLR_PREC_FP64) return coupling_apply<double>(F.d.N, r, c, F.P, (int64_t)r * c, anc, Kc, 1, 0, s, cr);
  return coupling_apply<float>(F.d.N, r, c, F.P, (int64_t)r * c, anc, Kc, 1, 0, s, cr);
}

// Skinny coupling solve (k <= 8 right-hand sides), FP64: n = 2r threads per
// parent, thread i gathers row i of the right-hand side (sum of chunk
// partials) and then forms row i of Kinv * rhs (Kinv read column by column,
// coalesced) or of Kinv^T * rhs.
template <int KC>
__global__ void __launch_bounds__(256) coupling_solve_skinny_kernel(int64_t N, int r, int c, double* P, int k,
                                                                    const double* __restrict__ Kinv,
                                                                    int first_is_beta, int trans, int64_t cpn_read) {
  __shared__ double sRhs[256 * KC];
  const int n = 2 * r;
  const int ppc = 256 / n;  // parents per CTA
  const int slot_in_cta = threadIdx.x / n;
  const int i = threadIdx.x % n;
  const int64_t parents = (int64_t)1 << (c - 1);
  const int64_t j = (int64_t)blockIdx.x * ppc + slot_in_cta;
  const bool active = slot_in_cta < ppc && j < parents;
  const int64_t cpn = chunks_per_node(N, c);
  const size_t slot = (size_t)r * k;
  const int64_t qa = 2 * j * cpn, qb = (2 * j + 1) * cpn;
  double* rhs = sRhs + slot_in_cta * n * KC;
  if (active) {
    const int64_t q0 = (i < r) == (first_is_beta != 0) ? qb : qa;
    const int row = i < r ? i : i - r;
#pragma unroll
    for (int cc = 0; cc < KC; ++cc) {
      double acc = 0.0;
      if (cc < k)
        for (int64_t q = 0; q < cpn_read; ++q) acc += P[(q0 + q) * slot + (size_t)cc * r + row];
      rhs[i * KC + cc] = acc;
    }
  }
  __syncthreads();
  double acc[KC];
#pragma unroll
  for (int cc = 0; cc < KC; ++cc) acc[cc] = 0.0;
  if (active) {
    const double* Kj = Kinv + (size_t)j * n * n;
#pragma unroll 16
    for (int jj = 0; jj < n; ++jj) {
      const double kv = trans ? Kj[(size_t)i * n + jj] : Kj[(size_t)jj * n + i];
#pragma unroll
      for (int cc = 0; cc < KC; ++cc) acc[cc] += kv * rhs[jj * KC + cc];
    }
  }
  __syncthreads();  // all reads of this CTA's partials done before the writes
  if (!active) return;
  const int64_t q = i < r ? qa : qb;
  const int row = i < r ? i : i - r;
#pragma unroll
  for (int cc = 0; cc < KC; ++cc)
    if (cc < k) P[q * slot + (size_t)cc * r + row] = acc[cc];
}

template <int KC>
static cudaError_t coupling_solve_skinny(int64_t N, int r, int c, double* P, int k, const double* Kinv,
                                         int first_is_beta, int trans, cudaStream_t s, int64_t cpn_read) {
  const int n = 2 * r;
  const int ppc = 256 / n;
  const int64_t parents = (int64_t)1 << (c - 1);
  const unsigned grid = (unsigned)((parents + ppc - 1) / ppc);
  note_work(8.0 * ((double)num_chunks(N, c) * r * k + parents * n * n + 2.0 * parents * r * k),
            parents * 2.0 * n * n * (double)k);
  { coupling_solve_skinny_kernel<KC><<<grid, 256, 0, s>>>(N, r, c, P, k, Kinv, first_is_beta, trans, cpn_read); note_launches(1); }
  return cudaGetLastError();
}

// Solve / adjoint: w = Kinv [s_beta; s_alpha] or t = Kinv^T [s_alpha; s_beta], FP64.
cudaError_t launch_coupling_solve(const Factor& F, int c, double* P, int k, int trans, cudaStream_t s,
                                  bool reduced) {
  ProfScope prof_(KC_COUPLING_APPLY, s);
  const int r = F.d.r;
  const double* Kc = F.K + F.Koff[c] * 4 * r * r;
  const int fib = trans ? 0 : 1;
  const int64_t cr = reduced ? 1 : chunks_per_node(F.d.N, c);
  if (k == 1) return coupling_solve_skinny<1>(F.d.N, r, c, P, k, Kc, fib, trans, s, cr);
  if (k <= 2) return coupling_solve_skinny<2>(F.d.N, r, c, P, k, Kc, fib, trans, s, cr);
  if (k <= 4) return coupling_solve_skinny<4>(F.d.N, r, c, P, k, Kc, fib, trans, s, cr);
  if (k <= 8) return coupling_solve_skinny<8>(F.d.N, r, c, P, k, Kc, fib, trans, s, cr);
  return coupling_apply<double>(F.d.N, r, c, P, k, k, Kc, fib, trans, s, cr);
}

// ---------------------------------------------------------------------------
// Sum the chunk partials of each node into the node's first slot (FP64,
// fixed order).
// Few chunks per node: one thread per slot element sums them in order.
__global__ void reduce_chunks_thread_kernel(int64_t N, int r, int c, double* P, int ncols) {
  const int64_t cpn = chunks_per_node(N, c);
  const int64_t node = blockIdx.x;
  const size_t slot = (size_t)r * ncols;
  const int64_t e = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
  if (e >= (int64_t)slot) return;
  double acc = 0.0;
  for (int64_t q = 0; q < cpn; ++q) acc += P[(node * cpn + q) * slot + e];
  P[node * cpn * slot + e] = acc;
}

// Many chunks per node: one warp per slot element, lanes sum strided chunks,
// then a fixed-order butterfly; the result goes to the node's first slot.
__global__ void reduce_chunks_kernel(int64_t N, int r, int c, double* P, int ncols) {
  const int64_t cpn = chunks_per_node(N, c);
  const int64_t node = blockIdx.x;
  const size_t slot = (size_t)r * ncols;
  const int lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.y * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (e >= (int64_t)slot) return;
  double acc = 0.0;
  for (int64_t q = lane; q < cpn; q += 32) acc += P[(node * cpn + q) * slot + e];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) P[node * cpn * slot + e] = acc;
}

cudaError_t launch_reduce_chunks(int64_t N, int r, int c, double* P, int ncols, cudaStream_t s) {
  ProfScope prof_(KC_REDUCE, s);
  if (chunks_per_node(N, c) == 1) return cudaSuccess;
  const size_t slot = (size_t)r * ncols;
  if (chunks_per_node(N, c) < 32) {
    dim3 g1(1u << c, (unsigned)((slot + 255) / 256));
    note_work(8.0 * ((double)num_chunks(N, c) + (double)(1ll << c)) * slot, (double)num_chunks(N, c) * slot);
    { reduce_chunks_thread_kernel<<<g1, 256, 0, s>>>(N, r, c, P, ncols); note_launches(1); }
    return cudaGetLastError();
  }
  dim3 grid(1u << c, (unsigned)((slot + 7) / 8));
  note_work(8.0 * ((double)num_chunks(N, c) + (double)(1ll << c)) * slot, (double)num_chunks(N, c) * slot);
  { reduce_chunks_kernel<<<grid, 256, 0, s>>>(N, r, c, P, ncols); note_launches(1); }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Deterministic FP64 sum of the log-determinant pieces: leaves then parents.
__global__ void logdet_reduce_kernel(const double* leaf_ld, int64_t nleaf, const double* node_ld, int64_t nnode,
                                     double* out) {
  __shared__ double sla[256];
  __shared__ int sneg[256], szero[256];
  const int tid = threadIdx.x;
  double la = 0.0;
  int neg = 0, zero = 0;
  for (int64_t i = tid; i < nleaf + nnode; i += 256) {
    const double* p = i < nleaf ? leaf_ld + 2 * i : node_ld + 2 * (i - nleaf);
    la += p[0];
    neg ^= (p[1] < 0.0);
    zero |= (p[1] == 0.0);
  }
  sla[tid] = la;
  sneg[tid] = neg;
  szero[tid] = zero;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (tid < w) {
      sla[tid] += sla[tid + w];
      sneg[tid] ^= sneg[tid + w];
      szero[tid] |= szero[tid + w];
    }
    __syncthreads();
  }
  if (tid == 0) {
    out[0] = szero[0] ? 0.0 : (sneg[0] ? -1.0 : 1.0);
    out[1] = sla[0];
  }
}

cudaError_t launch_logdet_reduce(const Factor& F, cudaStream_t s) {
  ProfScope prof_(KC_LOGDET, s);
  const int64_t nleaf = (int64_t)1 << F.d.L;
  note_work(32.0 * nleaf, 2.0 * nleaf);
  { logdet_reduce_kernel<<<1, 256, 0, s>>>(F.leaf_ld, nleaf, F.node_ld, nleaf - 1, F.ld_out); note_launches(1); }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Explicit instantiations
#define HODLR_INST(TB, TR)                                                                                      \
  template cudaError_t launch_project<TB, TR>(int64_t, int, int, const TB*, int64_t, int, const TR*, int64_t, \
                                              int, double*, int, cudaStream_t);                                 \
  template cudaError_t launch_update<TB, TR>(int64_t, int, int, const TB*, int64_t, int, TR*, int64_t, int,   \
                                             const double*, int64_t, int, double, int, cudaStream_t);
HODLR_INST(double, double)
HODLR_INST(float, double)
HODLR_INST(float, float)
HODLR_INST(__nv_bfloat16, __nv_bfloat16)
HODLR_INST(__nv_bfloat16, float)
#undef HODLR_INST

}  // namespace hodlr
