// Leaf stage of the low-precision factor for leaves of at most 128 rows: each
// leaf block is inverted (FP32 Gauss-Jordan elimination with partial
// pivoting, whose pivots are those of getrf, so the log-determinant is
// unchanged) and the leaf "solves" of Alg. 1 / Alg. 2
// (D_b^{-1} applied to Y_big rows or to right-hand sides) become small dense
// GEMMs with D_b^{-1}, free of the serial dependence of substitutions.
#include "hodlr_internal.cuh"

namespace hodlr {

// One CTA (256 threads, 16 x 16) per leaf: D_b (FP64) -> FP32 (rounded toward
// zero on the integer pipe), padded to an
// MB x MB matrix with the identity (MB = 64 or 128), inverted in registers by
// Gauss-Jordan elimination with partial pivoting over all MB rows; thread
// (ty, tx) holds the TT x TT block (TT = MB / 16) of rows ty*TT.. and columns
// tx*TT.., with ty = lane % 16 and tx = 2 warp + lane / 16, so that each
// column group lives in one half-warp. Rows are never exchanged: at step k the
// pivot row p_k is the unused row with the largest |a_ik| (lowest row on
// ties, as getrf's first maximum) and the exchange step turns row p_k into
// unknown k and column k into equation p_k, so that at the end entry (r, c) of
// the tableau is D^{-1}(step(r), p_c) and is written there.
// Rows are kept unscaled: the tableau row r is the stored row times
// 1 / pivot(step(r)) once row r has been a pivot row (the rank-1 update is
// linear in each row, so the scale commutes with later steps), and every
// stored row is scaled once after the last step. Per step, two barriers:
// (1) the half-warp owning column k finds the pivot with shuffles and
// publishes the multipliers f_i / pivot (0 for the pivot row, whose entry k
// becomes 1), (2) the owners of row p_k stage their blocks in shared memory;
// every thread then applies the rank-1 update a_ij -= (f_i / pivot) a_pj to
// its block. The pivots are getrf's pivots with rows in the order p_0, p_1,
// ..., so log|det D_b| = sum log|pivot| and the sign is the parity of the
// negative pivots and of the inversions of (p_k). Writes D_b^{-1} (FP32,
// column-major) to the factor's leaf buffer, the log-determinant pieces, and
// the status on a zero pivot or a non-finite entry.
// If Dtc is given (m = MB = 128), D_b^{-1} is also written in the K-major
// core-matrix layout of a tcgen05 operand (8-row x 16-byte cores: element
// (i, k) at float (i/8)*1024 + (k/4)*32 + (i%8)*4 + k%4), the A operand of
// the tensor-core leaf apply.
template <int MB>
__global__ void __launch_bounds__(256, 2) leaf_inv_kernel(int m, const double* __restrict__ D,
                                                          float* __restrict__ Dinv, float* __restrict__ Dtc,
                                                          int* __restrict__ perm, int64_t N,
                                                          double* __restrict__ leaf_ld, DevStatus* st) {
  constexpr int TT = MB / 16;
  constexpr int TG = TT / 4;            // float4 groups of a thread's rows / columns
  constexpr int LD = MB + 1;
  constexpr int BLK = TT * TT + 4;      // staged block stride (floats): the two half-warps hit different banks
  extern __shared__ float s_stage[];    // MB x LD: input, then output staging
  // multipliers of step k (double-buffered by step parity); rows ty*TT + 4g + e
  // at float ((g * 16 + ty) * 4 + e), so that a quarter-warp reads 128
  // contiguous bytes
  __shared__ __align__(16) float s_f[2][MB];
  __shared__ __align__(16) float s_blk[16 * BLK];  // blocks of the owners of the pivot row
  __shared__ float2 s_pv[2];                        // (pivot value, pivot row as int bits)
  __shared__ int s_prow[MB];                        // p_k
  __shared__ int s_step[MB];                        // step that took row r
  __shared__ float s_piv[MB];
  __shared__ int s_bad;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ty = lane & 15, tx = (warp << 1) | (lane >> 4);
  const int b = blockIdx.x;
  if (tid == 0) s_bad = 0;
  const double* Db = D + (size_t)b * m * m;
  bool bad = false;
  // eight loads in flight per thread before any is used (the leaf is read
  // once, from HBM)
  for (int e0 = 0; e0 < MB * MB; e0 += 8 * 256) {
    double xv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * 256 + tid;
      const int c = e / MB, r = e % MB;
      xv[u] = (r < m && c < m) ? Db[(size_t)c * m + r] : (r == c ? 1.0 : 0.0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * 256 + tid;
      const int c = e / MB, r = e % MB;
      bad |= !f64_finite_bits(xv[u]);
      s_stage[c * LD + r] = __uint_as_float(f64_to_f32_trunc_bits(xv[u]));
    }
  }
  __syncthreads();
  if (bad) atomicOr(&s_bad, 1);
  float a[TT][TT];
#pragma unroll
  for (int ii = 0; ii < TT; ++ii)
#pragma unroll
    for (int jj = 0; jj < TT; ++jj) a[ii][jj] = s_stage[(tx * TT + jj) * LD + ty * TT + ii];
  uint32_t used = 0;  // bit ii: row ty*TT+ii has been a pivot row

  for (int kb = 0; kb < 16; ++kb) {
    const bool col_owner = tx == kb;  // one half-warp
#pragma unroll
    for (int kk = 0; kk < TT; ++kk) {
      const int k = kb * TT + kk;
      const int buf = k & 1;
      // (1) the half-warp owning column k: the pivot (largest |a_ik| over the
      // unused rows, lowest row on ties; NaN ranks as +inf so that the order
      // stays total), then the scaled multipliers and column k of the
      // tableau (1 in the pivot row, 0 elsewhere; the update below writes
      // -f_i / pivot there)
      if (warp == (kb >> 1)) {
        unsigned long long bkey = 0;  // (|a| bits, 255 - row): larger |a|, then the lower row; 0 = used
        float bval = 0.f;
        if (col_owner) {
#pragma unroll
          for (int ii = 0; ii < TT; ++ii) {
            const float x = a[ii][kk];
            uint32_t ab = __float_as_uint(x) & 0x7fffffffu;
            if (ab > 0x7f800000u) ab = 0x7f800000u;
            const unsigned long long key =
                ((used >> ii) & 1u) ? 0ull : ((unsigned long long)ab << 8) | (unsigned long long)(255 - (ty * TT + ii));
            if (key > bkey) {
              bkey = key;
              bval = x;
            }
          }
        }
        unsigned long long wkey = bkey;
#pragma unroll
        for (int off = 8; off > 0; off >>= 1) wkey = max(wkey, __shfl_xor_sync(0xffffffffu, wkey, off));
        const int p = 255 - (int)(wkey & 255ull);
        const float piv = __shfl_sync(0xffffffffu, bval, (lane & 16) | (p / TT));
        if (col_owner) {
          const float rp = piv != 0.f ? 1.f / piv : 0.f;
#pragma unroll
          for (int ii = 0; ii < TT; ++ii) {
            const int row = ty * TT + ii;
            const float x = a[ii][kk];
            s_f[buf][((ii >> 2) * 16 + ty) * 4 + (ii & 3)] = row == p ? 0.f : x * rp;
            a[ii][kk] = row == p ? 1.f : 0.f;
          }
          if (ty == 0) {
            s_pv[buf] = make_float2(piv, __int_as_float(p));
            s_prow[k] = p;
            s_step[p] = k;
            s_piv[k] = piv;
          }
        }
      }
      __syncthreads();
      const int p = __float_as_int(s_pv[buf].y);
      const int pg = p / TT, pi = p % TT;
      // (2) owners of row p stage their whole blocks (static register indices)
      if (ty == pg) {
        float4* o = reinterpret_cast<float4*>(s_blk + tx * BLK);
#pragma unroll
        for (int ii = 0; ii < TT; ++ii)
#pragma unroll
          for (int g = 0; g < TG; ++g)
            o[ii * TG + g] = make_float4(a[ii][4 * g], a[ii][4 * g + 1], a[ii][4 * g + 2], a[ii][4 * g + 3]);
        used |= 1u << pi;
      }
      __syncthreads();
      // rank-1 update of every block (the pivot row has multiplier 0)
      float f[TT], q[TT];
#pragma unroll
      for (int g = 0; g < TG; ++g) {
        const float4 fv = reinterpret_cast<const float4*>(s_f[buf])[g * 16 + ty];
        const float4 qv = reinterpret_cast<const float4*>(s_blk + tx * BLK)[pi * TG + g];
        f[4 * g] = fv.x; f[4 * g + 1] = fv.y; f[4 * g + 2] = fv.z; f[4 * g + 3] = fv.w;
        q[4 * g] = qv.x; q[4 * g + 1] = qv.y; q[4 * g + 2] = qv.z; q[4 * g + 3] = qv.w;
      }
#pragma unroll
      for (int ii = 0; ii < TT; ++ii)
#pragma unroll
        for (int jj = 0; jj < TT; ++jj) a[ii][jj] = fmaf(-f[ii], q[jj], a[ii][jj]);
    }
  }
  // every row has been a pivot row once: scale it by 1 / its pivot
#pragma unroll
  for (int ii = 0; ii < TT; ++ii) {
    const float pv = s_piv[s_step[ty * TT + ii]];
    const float sc = pv != 0.f ? 1.f / pv : 0.f;
#pragma unroll
    for (int jj = 0; jj < TT; ++jj) a[ii][jj] *= sc;
  }
  // D^{-1}(step(r), p_c) = tableau(r, c): the tableau T is written as it is
  // (staged, then column-major), with p and step
#pragma unroll
  for (int ii = 0; ii < TT; ++ii)
#pragma unroll
    for (int jj = 0; jj < TT; ++jj) {
      const int r = ty * TT + ii, c = tx * TT + jj;
      s_stage[c * LD + r] = a[ii][jj];
    }
  for (int e = tid; e < m; e += 256) {
    perm[(size_t)b * m + e] = s_prow[e];
    perm[(size_t)N + (size_t)b * m + e] = s_step[e];
  }
  __syncthreads();
  float* out = Dinv + (size_t)b * m * m;
  for (int e = tid; e < m * m; e += 256) out[e] = s_stage[(e / m) * LD + (e % m)];
  if (Dtc) {
    float4* o = reinterpret_cast<float4*>(Dtc + (size_t)b * MB * MB);
    for (int e4 = tid; e4 < MB * MB / 4; e4 += 256) {
      const int il = e4 & 7, kq = (e4 >> 3) % (MB / 4), ig = e4 / (2 * MB);
      const int i = ig * 8 + il, k = kq * 4;
      o[e4] = make_float4(s_stage[k * LD + i], s_stage[(k + 1) * LD + i], s_stage[(k + 2) * LD + i],
                          s_stage[(k + 3) * LD + i]);
    }
  }
  if (warp == 0) {
    double la = 0.0;
    int ng = 0, sg = m, inv = 0;
    for (int k = lane; k < m; k += 32) {
      const float v = s_piv[k];
      la += log(fabs((double)v));
      ng ^= v < 0.f ? 1 : 0;
      if (v == 0.f && k < sg) sg = k;
      const int pk = s_prow[k];
      for (int k2 = k + 1; k2 < m; ++k2) inv += s_prow[k2] < pk ? 1 : 0;
    }
    ng ^= inv & 1;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      la += __shfl_down_sync(0xffffffffu, la, off);
      ng ^= __shfl_down_sync(0xffffffffu, ng, off);
      sg = min(sg, __shfl_down_sync(0xffffffffu, sg, off));
    }
    if (lane == 0) {
      if (s_bad) set_status(st, HODLR_ERR_NONFINITE, b, 0);
      leaf_ld[2 * b] = la;
      leaf_ld[2 * b + 1] = sg < m ? 0.0 : (ng ? -1.0 : 1.0);
      if (sg < m) set_status(st, HODLR_ERR_SINGULAR_LEAF, b, sg);
    }
  }
}

bool leaf_uses_inverse(const Factor& F) { return F.prec != HODLR_PREC_FP64 && F.d.m <= 128; }

cudaError_t launch_leaf_inv(const Factor& F, const double* D, cudaStream_t s) {
  const int m = F.d.m;
  const int nleaf = 1 << F.d.L;
  // D_b read (FP64), D_b^{-1} written (FP32), plus its tensor-core operand copy
  note_work((8.0 + 4.0 + (F.leaf_tc ? 4.0 : 0.0)) * nleaf * m * m, 2.0 * (double)m * m * m * nleaf);
  if (leaf_inv_tc_supported(F))
    return launch_leaf_inv_tc(F, D, F.leaf_tc ? reinterpret_cast<float*>(F.P) : nullptr, s);
  if (m > 64) {
    const size_t sm = (size_t)128 * 129 * 4;
    cudaFuncSetAttribute(leaf_inv_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    float* Dtc = F.leaf_tc ? reinterpret_cast<float*>(F.P) : nullptr;  // m == 128 here
    { leaf_inv_kernel<128><<<nleaf, 256, sm, s>>>(m, D, static_cast<float*>(F.lu), Dtc, F.perm, F.d.N, F.leaf_ld, F.status); note_launches(1); }
  } else {
    const size_t sm = (size_t)64 * 65 * 4;
    { leaf_inv_kernel<64><<<nleaf, 256, sm, s>>>(m, D, static_cast<float*>(F.lu), nullptr, F.perm, F.d.N, F.leaf_ld, F.status); note_launches(1); }
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// out(I_b, cols) = op(Dinv_b) * in(I_b, cols), op = identity or transpose.
// Wide: CTA = one leaf x 64 columns, all m <= 128 rows; K = m staged 32 at a
// time; thread tile 8 rows x 4 columns. In-place safe: a CTA reads every input
// row of its columns before it writes.
template <typename TIN, typename TOUT>
__global__ void __launch_bounds__(256) leaf_apply_wide_kernel(int m, const float* __restrict__ Dinv,
                                                              const int* __restrict__ perm, int64_t N, const TIN* in,
                                                              int64_t ldin, TOUT* out, int64_t ldout, int ncols,
                                                              int trans) {
  __shared__ float sA[32][128 + 4];  // [kk][i] = op(T)(i, k0 + kk)
  __shared__ float sB[32][64 + 4];   // [kk][j] = in(gather(k0 + kk), j0 + j)
  __shared__ int s_g[128], s_s[128];  // gather (inputs) and scatter (outputs) rows of the leaf
  const int b = blockIdx.x;
  const int j0 = blockIdx.y * 64;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const float* Ab = Dinv + (size_t)b * m * m;
  const int64_t row0 = (int64_t)b * m;
  // T holds D^{-1}(step(r), p_c) at (r, c): D^{-1} x = scatter_step(T gather_p(x)),
  // D^{-T} x = scatter_p(T^T gather_step(x))
  const int* pp = perm + (size_t)b * m;
  const int* ps = perm + (size_t)N + (size_t)b * m;
  for (int e = tid; e < m; e += 256) {
    s_g[e] = trans ? ps[e] : pp[e];
    s_s[e] = trans ? pp[e] : ps[e];
  }
  __syncthreads();
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
      sB[kk][j] = (k < m && j0 + j < ncols) ? conv<float>(in[(int64_t)(j0 + j) * ldin + row0 + s_g[k]]) : 0.f;
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
      if (i < m) out[(int64_t)j * ldout + row0 + s_s[i]] = conv<TOUT>(acc[a][c]);
    }
  }
}

// Narrow (ncols <= 8): thread i of the CTA owns row i; the leaf's right-hand
// sides are staged in shared memory first (in-place safe).
template <typename TIN, typename TOUT, int KC>
__global__ void __launch_bounds__(128) leaf_apply_narrow_kernel(int m, const float* __restrict__ Dinv,
                                                                const int* __restrict__ perm, int64_t N, const TIN* in,
                                                                int64_t ldin, TOUT* out, int64_t ldout, int ncols,
                                                                int trans) {
  __shared__ float sx[128 * KC];
  const int b = blockIdx.x;
  const float* Ab = Dinv + (size_t)b * m * m;
  const int64_t row0 = (int64_t)b * m;
  // T holds D^{-1}(step(r), p_c) at (r, c): inputs gathered by p (D^{-1}) or
  // step (D^{-T}), outputs scattered by the other
  const int* pg = perm + (trans ? (size_t)N : 0) + (size_t)b * m;
  const int* ps = perm + (trans ? 0 : (size_t)N) + (size_t)b * m;
  for (int e = threadIdx.x; e < m * KC; e += blockDim.x) {
    const int k = e % m, c = e / m;
    sx[k * KC + c] = c < ncols ? conv<float>(in[(int64_t)c * ldin + row0 + pg[k]]) : 0.f;
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
  const int oi = ps[i];
#pragma unroll
  for (int c = 0; c < KC; ++c)
    if (c < ncols) out[(int64_t)c * ldout + row0 + oi] = conv<TOUT>(acc[c]);
}

// m = 128, D^{-1} (not transposed), at most 8 columns: warp w takes the K
// range 32w .. 32w+31 and lane l rows 4l .. 4l+3, one 16-byte load of T per
// column k (each warp reads 512 contiguous bytes per load); the four warps'
// partial sums are added in shared memory.
template <typename TIN, typename TOUT, int KC>
__global__ void __launch_bounds__(128) leaf_apply_n128_kernel(const float* __restrict__ Dinv,
                                                              const int* __restrict__ perm, int64_t N, const TIN* in,
                                                              int64_t ldin, TOUT* out, int64_t ldout, int ncols) {
  constexpr int m = 128;
  __shared__ float sx[m * KC];
  __shared__ float4 sp[4][32][KC];
  const int b = blockIdx.x;
  const float4* A4 = reinterpret_cast<const float4*>(Dinv + (size_t)b * m * m);
  const int64_t row0 = (int64_t)b * m;
  const int* pg = perm + (size_t)b * m;       // inputs gathered by p
  const int* ps = perm + (size_t)N + (size_t)b * m;  // outputs scattered by step
  for (int e = threadIdx.x; e < m * KC; e += blockDim.x) {
    const int k = e % m, c = e / m;
    sx[k * KC + c] = c < ncols ? conv<float>(in[(int64_t)c * ldin + row0 + pg[k]]) : 0.f;
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float4 acc[KC];
#pragma unroll
  for (int c = 0; c < KC; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 8
  for (int kk = 0; kk < 32; ++kk) {
    const int k = w * 32 + kk;
    const float4 a = __ldg(A4 + k * 32 + lane);  // T(4 lane .. 4 lane + 3, k)
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      const float x = sx[k * KC + c];
      acc[c].x += a.x * x;
      acc[c].y += a.y * x;
      acc[c].z += a.z * x;
      acc[c].w += a.w * x;
    }
  }
#pragma unroll
  for (int c = 0; c < KC; ++c) sp[w][lane][c] = acc[c];
  __syncthreads();
  const int i = threadIdx.x, ln = i >> 2, cp = i & 3;
  const int oi = ps[i];
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    if (c >= ncols) break;
    float v = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 t = sp[q][ln][c];
      v += cp == 0 ? t.x : cp == 1 ? t.y : cp == 2 ? t.z : t.w;
    }
    out[(int64_t)c * ldout + row0 + oi] = conv<TOUT>(v);
  }
}

template <typename TIN, typename TOUT>
cudaError_t launch_leaf_apply_inv(const Factor& F, const TIN* in, int64_t ldin, TOUT* out, int64_t ldout, int ncols,
                                  int trans, cudaStream_t s) {
  const int m = F.d.m;
  const int nleaf = 1 << F.d.L;
  const float* Dinv = static_cast<const float*>(F.lu);
  const double Nd = (double)nleaf * m;
  // the scaled Gauss-Jordan tableau T with D^{-1}(step(r), p_c) = T(r, c); p and
  // step in F.perm (see the leaf inverse kernels)
  note_work((sizeof(TIN) + sizeof(TOUT)) * Nd * ncols + 4.0 * Nd * m, 2.0 * m * Nd * ncols);
  if (ncols <= 8 && m == 128 && !trans) {
    if (ncols == 1)
      { leaf_apply_n128_kernel<TIN, TOUT, 1><<<nleaf, 128, 0, s>>>(Dinv, F.perm, F.d.N, in, ldin, out, ldout, ncols); note_launches(1); }
    else if (ncols <= 2)
      { leaf_apply_n128_kernel<TIN, TOUT, 2><<<nleaf, 128, 0, s>>>(Dinv, F.perm, F.d.N, in, ldin, out, ldout, ncols); note_launches(1); }
    else if (ncols <= 4)
      { leaf_apply_n128_kernel<TIN, TOUT, 4><<<nleaf, 128, 0, s>>>(Dinv, F.perm, F.d.N, in, ldin, out, ldout, ncols); note_launches(1); }
    else
      { leaf_apply_n128_kernel<TIN, TOUT, 8><<<nleaf, 128, 0, s>>>(Dinv, F.perm, F.d.N, in, ldin, out, ldout, ncols); note_launches(1); }
  } else if (ncols <= 8) {
    const int th = ((m + 31) / 32) * 32;
    if (ncols == 1)
      { leaf_apply_narrow_kernel<TIN, TOUT, 1><<<nleaf, th, 0, s>>>(m, Dinv, F.perm, F.d.N, in, ldin, out, ldout, ncols, trans); note_launches(1); }
    else if (ncols <= 2)
      { leaf_apply_narrow_kernel<TIN, TOUT, 2><<<nleaf, th, 0, s>>>(m, Dinv, F.perm, F.d.N, in, ldin, out, ldout, ncols, trans); note_launches(1); }
    else if (ncols <= 4)
      { leaf_apply_narrow_kernel<TIN, TOUT, 4><<<nleaf, th, 0, s>>>(m, Dinv, F.perm, F.d.N, in, ldin, out, ldout, ncols, trans); note_launches(1); }
    else
      { leaf_apply_narrow_kernel<TIN, TOUT, 8><<<nleaf, th, 0, s>>>(m, Dinv, F.perm, F.d.N, in, ldin, out, ldout, ncols, trans); note_launches(1); }
  } else {
    dim3 grid(nleaf, (ncols + 63) / 64);
    { leaf_apply_wide_kernel<TIN, TOUT><<<grid, 256, 0, s>>>(m, Dinv, F.perm, F.d.N, in, ldin, out, ldout, ncols, trans); note_launches(1); }
  }
  return cudaGetLastError();
}

template cudaError_t launch_leaf_apply_inv<double, float>(const Factor&, const double*, int64_t, float*, int64_t, int,
                                                          int, cudaStream_t);
template cudaError_t launch_leaf_apply_inv<double, __nv_bfloat16>(const Factor&, const double*, int64_t,
                                                                  __nv_bfloat16*, int64_t, int, int, cudaStream_t);
template cudaError_t launch_leaf_apply_inv<float, float>(const Factor&, const float*, int64_t, float*, int64_t, int,
                                                         int, cudaStream_t);
template cudaError_t launch_leaf_apply_inv<double, double>(const Factor&, const double*, int64_t, double*, int64_t,
                                                           int, int, cudaStream_t);

}  // namespace hodlr
