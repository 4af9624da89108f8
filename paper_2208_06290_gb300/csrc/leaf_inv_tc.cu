// Tensor-core leaf inverse of the low-precision factor (leaves of 65..128
// rows): the first step of Alg. 1 / Alg. 3 (batched leaf factorization) done
// as a blocked Gauss-Jordan inversion with partial pivoting, whose pivots are
// getrf's (so log|det D_b| and its sign are unchanged), with the O(m^3) bulk
// of the elimination on tcgen05.
//
// Layout. One CTA = one warpgroup (4 warps) per leaf, persistent over leaves.
// The leaf's 128 x 128 FP32 tableau lives in TMEM (128 lanes x 128 columns):
// lane r holds row r, and warp w reads and writes lanes 32w .. 32w+31, so each
// thread owns one row. D_b (FP64, column-major) is read row by row (each warp
// load is 32 consecutive rows of one column), converted to FP32 on the integer
// pipe (truncation) and padded with the identity to 128 x 128.
//
// Elimination (rows are never exchanged; step k picks the unused row p_k with
// the largest |t(i, k)|, the lowest row on ties, and the tableau keeps the
// pivot rows unscaled until the end, as in the CUDA-core kernel). The step
// maps every column j != k by M_k = I - g e_{p_k}^T (g_i = t(i,k) / pivot,
// g_{p_k} = 0) and replaces column k by M_k e_{p_k}. For a panel of 32 steps
// k0 .. k0+31 with pivot rows P:
//   * the 32 panel columns are loaded into registers and the 32 steps run on
//     them only (pivot search by a warp max of the |t| bits and a ballot, the
//     four warps' candidates compared through shared memory: one CTA barrier
//     per step); at the end they hold T(:, P), T = M_{k0+31} ... M_{k0};
//   * T - I is zero outside the columns P, so every other column becomes
//     t'(:, j) = T(:, P) t(P, j) + [i not in P] t(i, j): one MMA chain
//     D (TMEM, the tableau's other 96 columns, pivot rows zeroed first)
//     += A B with A = T(:, P) (128 x 32) and B^T = t(P, others) (96 x 32),
//     both staged in shared memory in the K-major core-matrix layout.
// The MMA is kind::tf32 on split operands, x = hi + lo with hi = x with its
// low 13 significand bits cleared and lo = x - hi (exact), as
// A_hi B_hi + A_hi B_lo + A_lo B_hi (relative error about 2^-20 per product,
// near the FP32 arithmetic of the CUDA-core kernel); accumulation is FP32.
// Every row has been a pivot row once at the end; it is scaled by 1 / its
// pivot, and the scaled tableau T satisfies D^{-1}(step(r), p_c) = T(r, c).
// T is written as it is (no permutation: each lane writes its own row,
// coalesced), column-major and, when asked, in the K-major core layout of
// the tensor-core leaf apply, with p (perm[b m + c] = p_c) and its inverse
// (perm[N + b m + r] = step(r)); the consumers gather their inputs by p and
// scatter their outputs by step (or the reverse for D^{-T}). Also written:
// the per-leaf (log|det|, sign) and the status of a zero pivot or a
// non-finite entry.
// The MMA completion wait is bounded; a wait that gives up records
// HODLR_ERR_TIMEOUT, waits (bounded) for the MMA in flight, frees TMEM and
// returns.
#include "tc_common.cuh"

namespace hodlr {
namespace {

constexpr int kLiThreads = 128;
constexpr int kLiCols = 128;             // TMEM columns = tableau columns
constexpr uint32_t kLiSBO = 1024;        // 8-row groups of a K = 32 operand: 8 cores x 128 B

struct LiSmem {
  static constexpr uint32_t kA = 128 * 32 * 4;    // A operand (one part)
  static constexpr uint32_t kB = 96 * 32 * 4;     // B operand (one part)
  static constexpr uint32_t kAhi = 0, kAlo = kA, kBhi = 2 * kA, kBlo = 2 * kA + kB;
  static constexpr uint32_t kOps = 2 * kA + 2 * kB;
  static constexpr int kTLd = 97;                 // [step][column] staging of the pivot rows (in A_lo)
  static constexpr uint32_t kCand = kOps;                         // [2][4][32] floats
  static constexpr uint32_t kKey = kCand + 2 * 4 * 32 * 4;      // uint64 [2][4]: key << 32 | (0xffff - row)
  static constexpr uint32_t kProw = kKey + 64;                  // int [128]: p_k
  static constexpr uint32_t kPiv = kProw + 512;                 // float [128]
  static constexpr uint32_t kRed = kPiv + 512;                  // per-warp log-det partials
  static constexpr uint32_t kBar = kRed + 4 * 32;
  static constexpr uint32_t kBytes = kBar + 64 + 128;           // + alignment slack
  static_assert(32 * kTLd * 4 <= kA, "pivot-row staging fits in A_lo");
};

// x = hi + lo with hi the TF32 part (low 13 significand bits cleared).
__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xffffe000u);
  lo = x - hi;
}

__global__ void __launch_bounds__(kLiThreads, 3) leaf_inv_tc_kernel(int m, int64_t nleaf, const double* __restrict__ D,
                                                                     float* __restrict__ Dinv,
                                                                     float* __restrict__ Dtc, int* __restrict__ perm,
                                                                     double* __restrict__ leaf_ld, DevStatus* st) {
  using S = LiSmem;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  float* s_tr = reinterpret_cast<float*>(smem + S::kAlo);  // pivot rows [step][column], before A_lo is written
  float* s_cand = reinterpret_cast<float*>(smem + S::kCand);
  unsigned long long* s_key = reinterpret_cast<unsigned long long*>(smem + S::kKey);
  int* s_prow = reinterpret_cast<int*>(smem + S::kProw);
  float* s_piv = reinterpret_cast<float*>(smem + S::kPiv);
  double* s_red = reinterpret_cast<double*>(smem + S::kRed);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + S::kBar);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = tid;  // tableau row = TMEM lane

  if (tid == 0) {
    tc::mbar_init(bar, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, kLiCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's lanes

  bool ok = true;
  uint32_t ph = 0;
  bool mma_pending = false;  // thread 0's view
  for (int64_t b = blockIdx.x; b < nleaf && ok; b += gridDim.x) {
    // ---- load row `row` of D_b (identity-padded) into the tableau; the next
    // leaf of this CTA is prefetched into L2 meanwhile
    const double* Db = D + (size_t)b * m * m;
    if (b + gridDim.x < nleaf) {
      const char* nx = reinterpret_cast<const char*>(D + (size_t)(b + gridDim.x) * m * m);
      for (int64_t o = (int64_t)tid * 128; o < (int64_t)m * m * 8; o += 128 * kLiThreads)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(nx + o));
    }
    bool bad = false;
    for (int c0 = 0; c0 < kLiCols; c0 += 32) {
      double x[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int c = c0 + j;
        x[j] = (row < m && c < m) ? Db[(size_t)c * m + row] : (row == c ? 1.0 : 0.0);
      }
      float v[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        bad |= !f64_finite_bits(x[j]);
        v[j] = __uint_as_float(f64_to_f32_trunc_bits(x[j]));
      }
      tc::tmem_st32(tl + c0, v);
    }

    bool used = false;
    int my_step = 0;
    float my_piv = 0.f;
    for (int q = 0; q < kLiCols / 32 && ok; ++q) {
      const int k0 = q * 32;
      float a[32];
      tc::tmem_ld32(tl + k0, a);
      // ---- the panel's 32 steps on its columns, one barrier per step
#pragma unroll
      for (int s = 0; s < 32; ++s) {
        const int buf = s & 1;
        uint32_t ab = __float_as_uint(a[s]) & 0x7fffffffu;
        if (ab > 0x7f800000u) ab = 0x7f800000u;  // NaN ranks as +inf: the order stays total
        const uint32_t key = used ? 0u : ab + 1u;  // 0 = already a pivot row
        const uint32_t wmax = __reduce_max_sync(0xffffffffu, key);
        const int lead = __ffs(__ballot_sync(0xffffffffu, key == wmax)) - 1;  // lowest row of the warp's max
        if (lane == lead) {
          float4* o = reinterpret_cast<float4*>(s_cand + (buf * 4 + warp) * 32);
#pragma unroll
          for (int g = 0; g < 8; ++g) o[g] = make_float4(a[4 * g], a[4 * g + 1], a[4 * g + 2], a[4 * g + 3]);
          s_key[buf * 4 + warp] = ((unsigned long long)wmax << 32) | (unsigned long long)(0xffff - row);
        }
        __syncthreads();
        // largest key, lowest row on ties (rows of lower warps are lower)
        const ulonglong2 k01 = *reinterpret_cast<const ulonglong2*>(s_key + buf * 4);
        const ulonglong2 k23 = *reinterpret_cast<const ulonglong2*>(s_key + buf * 4 + 2);
        const unsigned long long kb = max(max(k01.x, k01.y), max(k23.x, k23.y));
        const int p = 0xffff - (int)(kb & 0xffffull);
        const int pw = p >> 5;
        const float4* prow = reinterpret_cast<const float4*>(s_cand + (buf * 4 + pw) * 32);
        float pr[32];
#pragma unroll
        for (int g = 0; g < 8; ++g) {
          const float4 t = prow[g];
          pr[4 * g] = t.x; pr[4 * g + 1] = t.y; pr[4 * g + 2] = t.z; pr[4 * g + 3] = t.w;
        }
        const float piv = pr[s];
        const float rp = piv != 0.f ? 1.f / piv : 0.f;
        const bool is_p = row == p;
        const float g = is_p ? 0.f : a[s] * rp;
#pragma unroll
        for (int j = 0; j < 32; ++j) a[j] = fmaf(-g, pr[j], a[j]);
        a[s] = is_p ? 1.f : -g;
        if (is_p) {
          used = true;
          my_step = k0 + s;
          my_piv = piv;
        }
        if (tid == 0) {
          s_prow[k0 + s] = p;
          s_piv[k0 + s] = piv;
        }
      }
      // ---- trailing update of the other 96 columns on the tensor cores
      tc::tmem_st32(tl + k0, a);
      const bool piv_here = used && my_step >= k0;  // pivot row of this panel
      const int sl = my_step - k0;
      // (1) pivot rows of this panel: their old values of the other columns
      // into the [step][column] staging, zeros into the tableau
      if (__any_sync(0xffffffffu, piv_here)) {
        for (int c32 = 0; c32 < kLiCols / 32; ++c32) {
          if (c32 == q) continue;
          float v[32];
          tc::tmem_ld32(tl + c32 * 32, v);
          if (piv_here) {
            const int rho0 = c32 < q ? c32 * 32 : c32 * 32 - 32;  // index among the other 96 columns
            float* o = s_tr + sl * S::kTLd + rho0;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              o[j] = v[j];
              v[j] = 0.f;
            }
          }
          tc::tmem_st32(tl + c32 * 32, v);
        }
      }
      __syncthreads();
      // (2) B^T (96 x 32) in the K-major core layout, TF32 hi / lo parts:
      // item (sq, rho) = 16 bytes of steps 4 sq .. 4 sq + 3 of column rho
      {
        uint8_t* bhi = smem + S::kBhi;
        uint8_t* blo = smem + S::kBlo;
        for (int it = tid; it < 96 * 8; it += kLiThreads) {
          const int sq = it / 96, rho = it % 96;
          float h[4], l[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) tf32_split(s_tr[(4 * sq + e) * S::kTLd + rho], h[e], l[e]);
          const uint32_t off = (uint32_t)(rho >> 3) * kLiSBO + (uint32_t)sq * 128 + (uint32_t)(rho & 7) * 16;
          *reinterpret_cast<float4*>(bhi + off) = make_float4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<float4*>(blo + off) = make_float4(l[0], l[1], l[2], l[3]);
        }
      }
      __syncthreads();  // the staging (in A_lo) is read
      // (3) A = T(:, P) (128 x 32), TF32 hi / lo parts, from the panel registers
      {
        uint8_t* ahi = smem + S::kAhi;
        uint8_t* alo = smem + S::kAlo;
        const uint32_t rb = (uint32_t)(row >> 3) * kLiSBO + (uint32_t)(row & 7) * 16;
#pragma unroll
        for (int kc = 0; kc < 8; ++kc) {
          float h[4], l[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) tf32_split(a[4 * kc + e], h[e], l[e]);
          *reinterpret_cast<float4*>(ahi + rb + kc * 128) = make_float4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<float4*>(alo + rb + kc * 128) = make_float4(l[0], l[1], l[2], l[3]);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc::tc_fence_before();
      __syncthreads();
      tc::tc_fence_after();
      if (tid == 0) {
        const uint32_t a_hi = tc::smem_u32(smem + S::kAhi), a_lo = tc::smem_u32(smem + S::kAlo);
        const uint32_t b_hi = tc::smem_u32(smem + S::kBhi), b_lo = tc::smem_u32(smem + S::kBlo);
#pragma unroll
        for (int part = 0; part < 2; ++part) {
          const int c0 = part == 0 ? 0 : k0 + 32;  // tableau columns [c0, c0 + n)
          const int n = part == 0 ? k0 : 96 - k0;
          if (n == 0) continue;
          const uint32_t boff = (uint32_t)((part == 0 ? 0 : k0) >> 3) * kLiSBO;
          const uint32_t idesc = tc::idesc_tf32_f32(128, n);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {  // K = 8 per MMA: two cores along K
            const uint64_t ah = tc::desc_noswz_kmajor(a_hi + ks * 256, 128, kLiSBO);
            const uint64_t al = tc::desc_noswz_kmajor(a_lo + ks * 256, 128, kLiSBO);
            const uint64_t bh = tc::desc_noswz_kmajor(b_hi + boff + ks * 256, 128, kLiSBO);
            const uint64_t bl = tc::desc_noswz_kmajor(b_lo + boff + ks * 256, 128, kLiSBO);
            tc::mma_tf32(tmem + c0, ah, bh, idesc, 1);
            tc::mma_tf32(tmem + c0, ah, bl, idesc, 1);
            tc::mma_tf32(tmem + c0, al, bh, idesc, 1);
          }
        }
        tc::mma_commit(bar);
        mma_pending = true;
      }
      ok = __syncthreads_and(tc::mbar_wait(bar, ph)) != 0;
      if (ok) {
        ph ^= 1;
        mma_pending = false;
      }
      tc::tc_fence_after();
    }
    if (!ok) break;

    // ---- T(r, c) / pivot(step(r)) written row by row (lane r writes row r):
    // column-major (each warp store is 32 consecutive rows of a column) and,
    // for the tensor-core leaf apply, in its K-major core layout (16 bytes of
    // one row per store)
    const float sc = my_piv != 0.f ? 1.f / my_piv : 0.f;
    float* out = Dinv + (size_t)b * m * m;
    for (int c0 = 0; c0 < kLiCols; c0 += 32) {
      float v[32];
      tc::tmem_ld32(tl + c0, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] *= sc;
      if (row < m) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (c0 + j < m) out[(size_t)(c0 + j) * m + row] = v[j];
      }
      if (Dtc) {  // m == 128
        float4* o = reinterpret_cast<float4*>(Dtc + (size_t)b * 128 * 128 + (size_t)(row >> 3) * 1024 +
                                              (size_t)(c0 >> 2) * 32 + (row & 7) * 4);
#pragma unroll
        for (int g = 0; g < 8; ++g) o[g * 8] = make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
      }
    }
    if (row < m) {
      perm[(size_t)b * m + row] = s_prow[row];                      // p_c for c = row
      perm[(size_t)nleaf * m + (size_t)b * m + row] = my_step;      // step(r) for r = row
    }
    // per-step pieces of log|det|: log|pivot|, negative pivots, the first zero
    // pivot, and the inversions of (p_k) (the parity of the row order)
    {
      const int k = tid;
      double la = 0.0;
      int ng = 0, sg = m, inv = 0;
      if (k < m) {
        const float v = s_piv[k];
        la = log(fabs((double)v));
        ng = v < 0.f ? 1 : 0;
        if (v == 0.f) sg = k;
        const int pk = s_prow[k];
        for (int k2 = k + 1; k2 < m; ++k2) inv ^= s_prow[k2] < pk ? 1 : 0;
      }
      ng ^= inv;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        la += __shfl_down_sync(0xffffffffu, la, off);
        ng ^= __shfl_down_sync(0xffffffffu, ng, off);
        sg = min(sg, __shfl_down_sync(0xffffffffu, sg, off));
      }
      if (lane == 0) {
        s_red[warp] = la;
        reinterpret_cast<int*>(s_red + 4)[2 * warp] = ng;
        reinterpret_cast<int*>(s_red + 4)[2 * warp + 1] = sg;
      }
    }
    const bool any_bad = __syncthreads_or(bad) != 0;
    if (tid == 0) {
      const int* rr = reinterpret_cast<const int*>(s_red + 4);
      const double la = s_red[0] + s_red[1] + s_red[2] + s_red[3];
      const int ng = rr[0] ^ rr[2] ^ rr[4] ^ rr[6];
      const int sg = min(min(rr[1], rr[3]), min(rr[5], rr[7]));
      if (any_bad) set_status(st, HODLR_ERR_NONFINITE, b, 0);
      leaf_ld[2 * b] = la;
      leaf_ld[2 * b + 1] = sg < m ? 0.0 : (ng ? -1.0 : 1.0);
      if (sg < m) set_status(st, HODLR_ERR_SINGULAR_LEAF, b, sg);
    }
    __syncthreads();  // the staging, pivot records and partials are reused by the next leaf
  }
  if (tid == 0) {
    if (mma_pending) tc::mbar_wait(bar, ph);
    if (!ok) set_status(st, HODLR_ERR_TIMEOUT, 0, 1);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kLiCols);
}

}  // namespace

bool leaf_inv_tc_supported(const Factor& F) { return g_use_tc && F.d.m > 64 && F.d.m <= 128; }

cudaError_t launch_leaf_inv_tc(const Factor& F, const double* D, float* Dtc, cudaStream_t s) {
  const int m = F.d.m;
  const int64_t nleaf = (int64_t)1 << F.d.L;
  const int bytes = (int)LiSmem::kBytes;
  cudaError_t e = cudaFuncSetAttribute(leaf_inv_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  int64_t grid = (int64_t)sms * 3;  // three CTAs (warpgroups) per SM: 3 x 128 TMEM columns
  if (grid > nleaf) grid = nleaf;
  leaf_inv_tc_kernel<<<(unsigned)grid, kLiThreads, bytes, s>>>(m, nleaf, D, static_cast<float*>(F.lu), Dtc,
                                                               F.perm, F.leaf_ld, F.status);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace hodlr
