// Coupling matrices, one warp per parent, r <= 32. S = I - T_a T_b, its
// Gauss-Jordan inverse and log|det S| are FP64 in every factor (the coupling
// "LU"); the products of the explicit inverse (S^{-1} T_a, T_b S^{-1} T_a,
// T_b S^{-1}) are FP64 for the FP64 and FP32 factors and FP32 (from the FP64
// pieces) for the BF16 factor, whose panels are BF16.
//
// Same quantities as the CTA kernel of level.cu (used for r > 32): with
// K~ = [[I, T_b], [T_a, I]] (Eq. e:k) and the Schur complement
// S = I - T_a T_b,
//   K~^{-1} = [[I + T_b S^{-1} T_a, -T_b S^{-1}], [-S^{-1} T_a, S^{-1}]],
//   det K~ = det S.
// A CTA per parent spends most of its time in barriers at these sizes; a
// warp per parent needs none.
//
// Lane i holds row i of S (padded to 32 x 32 with the identity) in registers.
// Gauss-Jordan with partial pivoting runs without moving rows: at step k the
// pivot row p_k is the unused lane with the largest |s_ik| (lowest lane on
// ties, as LAPACK's first maximum), and the in-place exchange step turns
// row p_k into x_k and column k into y_{p_k}. At the end row p_k, column j of
// the tableau is S^{-1}(k, p_j), which is gathered back into natural order
// through shared memory. The pivots are LU's pivots of S with rows taken in
// the order p_0, p_1, ..., so log|det S| = sum log|pivot| and the sign is the
// parity of the negative pivots and of the inversions of (p_k).
#include <type_traits>

#include "hodlr_internal.cuh"

namespace hodlr {

namespace {
constexpr int kCwWarps = 4;  // parents per CTA
constexpr int kCwLd = 33;    // padded row stride of the per-warp 32 x 32 tiles
constexpr unsigned kFull = 0xffffffffu;
}  // namespace

// Pivot lane of a Gauss-Jordan step: the unused lane with the largest |x|,
// the lowest lane on ties (LAPACK's first maximum), NaN above every number
// (a total order keeps the choice warp-uniform). |x| is compared as the
// integer bits of the FP64 magnitude (the same order for non-NaN values),
// high word then low word, by two warp reductions on the integer pipe:
// the FP64 pipe, the bottleneck of these kernels, is left to the elimination.
__device__ __forceinline__ int pivot_lane(double x, bool used) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
  const unsigned hi = used ? 0u : (unsigned)(bits >> 32) + 1u;  // 0 only for used lanes
  const unsigned lo = used ? 0u : (unsigned)bits;
  const unsigned H = __reduce_max_sync(kFull, hi);
  const unsigned Lo = __reduce_max_sync(kFull, hi == H ? lo : 0u);
  return __ffs(__ballot_sync(kFull, hi == H && lo == Lo)) - 1;  // an unused lane: H >= 1
}

template <bool FULL>
__global__ void __launch_bounds__(32 * kCwWarps) coupling_factor_warp_kernel(int64_t N, int r, int c,
                                                                              const double* __restrict__ P,
                                                                              int64_t cpn_read,
                                                                              double* __restrict__ Kinv,
                                                                              double* __restrict__ node_ld,
                                                                              DevStatus* st, int64_t heap_first,
                                                                              float* __restrict__ Kf) {
  extern __shared__ double cw_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t parents = (int64_t)1 << (c - 1);
  const int64_t j = (int64_t)blockIdx.x * kCwWarps + warp;
  if (j >= parents) return;  // whole warp; only warp-level synchronisation below
  double* Ta = cw_smem + (size_t)warp * 3 * 32 * kCwLd;  // row-major, ld 33
  double* Tb = Ta + 32 * kCwLd;
  double* X = Tb + 32 * kCwLd;
  const int64_t cpn = chunks_per_node(N, c);
  const size_t slot = (size_t)r * r * c;
  const int anc = r * (c - 1);
  const int64_t qa = 2 * j * cpn, qb = (2 * j + 1) * cpn;

  // T_a, T_b: the children's own blocks, chunk partials summed in FP64
#pragma unroll 8
  for (int col = 0; col < 32; ++col) {
    double a = 0.0, b = 0.0;
    if (lane < r && col < r) {
      const double* pa = P + qa * slot + (size_t)(anc + col) * r + lane;
      const double* pb = P + qb * slot + (size_t)(anc + col) * r + lane;
      for (int64_t q = 0; q < cpn_read; ++q) {
        a += pa[q * slot];
        b += pb[q * slot];
      }
    }
    Ta[lane * kCwLd + col] = a;
    Tb[lane * kCwLd + col] = b;
  }
  __syncwarp();

  // row `lane` of S = I - T_a T_b: FP64 products for the FP64 and FP32
  // factors; FP32 products of FP32 copies (in X, free until the tableau is
  // gathered) for the BF16 factor, whose T_a, T_b come from BF16 panels
  double s[32];
  if constexpr (FULL) {
#pragma unroll
    for (int q = 0; q < 32; ++q) s[q] = lane == q ? 1.0 : 0.0;
    for (int t = 0; t < r; ++t) {
      const double a = Ta[lane * kCwLd + t];
#pragma unroll
      for (int q = 0; q < 32; ++q) s[q] = fma(-a, Tb[t * kCwLd + q], s[q]);
    }
  } else {
    float* TaF = reinterpret_cast<float*>(X);
    float* TbF = TaF + 32 * kCwLd;
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      TaF[lane * kCwLd + q] = (float)Ta[lane * kCwLd + q];
      TbF[lane * kCwLd + q] = (float)Tb[lane * kCwLd + q];
    }
    __syncwarp();
    float sf[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) sf[q] = lane == q ? 1.f : 0.f;
    for (int t = 0; t < r; ++t) {
      const float a = TaF[lane * kCwLd + t];
#pragma unroll
      for (int q = 0; q < 32; ++q) sf[q] = fmaf(-a, TbF[t * kCwLd + q], sf[q]);
    }
#pragma unroll
    for (int q = 0; q < 32; ++q) s[q] = (double)sf[q];
    __syncwarp();  // X is the tableau's area below
  }

  bool used = false;
  double mypiv = 1.0;  // lane k: the pivot of step k
  int mypos = lane;   // lane k: the pivot row p_k
  int mystep = lane;  // lane i: the step that took row i as pivot
  int ninv = 0;       // lane k: #{k' > k : p_k' < p_k}
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const int p = pivot_lane(s[k], used);
    const double piv = __shfl_sync(kFull, s[k], p);
    const double rp = piv != 0.0 ? 1.0 / piv : 0.0;
    if (lane < k) ninv += p < mypos ? 1 : 0;
    if (lane == k) {
      mypiv = piv;
      mypos = p;
    }
    const bool isp = lane == p;
    if (isp) {
      used = true;
      mystep = k;
    }
    // row p: s_pq / pivot; other rows: s_iq - (s_ik / pivot) s_pq; column k:
    // 1 / pivot on row p, -s_ik / pivot elsewhere (one FMA per entry)
    const double coef = isp ? rp : -s[k] * rp;
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      if (q == k) continue;
      const double pv = __shfl_sync(kFull, s[q], p);
      s[q] = fma(coef, pv, isp ? 0.0 : s[q]);
    }
    s[k] = coef;
  }

  // log|det S| (FP64, fixed butterfly), sign, first zero pivot
  double la = lane < r ? log(fabs(mypiv)) : 0.0;
  int neg = ((lane < r && mypiv < 0.0) ? 1 : 0) ^ (ninv & 1);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    la += __shfl_xor_sync(kFull, la, off);
    neg ^= __shfl_xor_sync(kFull, neg, off);
  }
  const unsigned zero = __ballot_sync(kFull, lane < r && mypiv == 0.0);
  const int sing = zero ? __ffs(zero) - 1 : -1;

  // S^{-1}(k, i) = tableau(p_k, step of row i)
#pragma unroll
  for (int q = 0; q < 32; ++q) X[lane * kCwLd + q] = s[q];
  __syncwarp();
  double sv[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) sv[i] = X[mypos * kCwLd + __shfl_sync(kFull, mystep, i)];

  __syncwarp();
  // Products of the explicit inverse in TPR (FP64 when FULL, else FP32 from
  // the FP64 S^{-1}, T_a, T_b): FP32 copies of T_a and S^{-1} go to the
  // tableau's area, which the gather above has finished reading.
  using TPR = typename std::conditional<FULL, double, float>::type;
  TPR* TaP;
  TPR* SiP;
  TPR* M1P;
  if constexpr (FULL) {
    TaP = Ta;
    SiP = Ta;  // overwritten with S^{-1} once M1 is formed
    M1P = X;
  } else {
    float* XF = reinterpret_cast<float*>(X);
    TaP = XF;               // [32][33]
    SiP = XF + 32 * kCwLd;  // [32][33]
    M1P = XF;               // overwrites the T_a copy once M1 is formed
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      XF[lane * kCwLd + q] = (float)Ta[lane * kCwLd + q];
      SiP[lane * kCwLd + q] = (float)sv[q];
    }
    __syncwarp();
  }

  // M1 = S^{-1} T_a (row `lane`)
  TPR m1[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) m1[q] = TPR(0);
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const TPR si = (TPR)sv[i];
#pragma unroll
    for (int q = 0; q < 32; ++q) m1[q] = fma(si, TaP[i * kCwLd + q], m1[q]);
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    if constexpr (FULL) Ta[lane * kCwLd + q] = sv[q];  // S^{-1}
    M1P[lane * kCwLd + q] = m1[q];
  }
  __syncwarp();

  const int n = 2 * r;
  double* out = Kinv + (size_t)j * n * n;  // column-major 2r x 2r
  const bool row_ok = lane < r;
  // [21] = -M1, [22] = S^{-1}
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    if (row_ok && q < r) {
      out[(size_t)q * n + r + lane] = -(double)m1[q];
      out[(size_t)(r + q) * n + r + lane] = sv[q];
    }
  }
  // r = 32 and Kf given: the rows of K~^{-1} facing each child in FP32, rows
  // padded to 2r + 4 (the layout the fused tensor-core update stages): row
  // `lane` of the second child is [-M1 | S^{-1}], of the first (below)
  // [I + T_b M1 | -T_b S^{-1}]
  constexpr int kKfLd = 2 * 32 + 4;
  if (Kf) {
    float4* k1 = reinterpret_cast<float4*>(Kf + ((size_t)(2 * j + 1) * 32 + lane) * kKfLd);
#pragma unroll
    for (int q4 = 0; q4 < 8; ++q4) {
      k1[q4] = make_float4((float)-m1[4 * q4], (float)-m1[4 * q4 + 1], (float)-m1[4 * q4 + 2],
                           (float)-m1[4 * q4 + 3]);
      k1[8 + q4] = make_float4((float)sv[4 * q4], (float)sv[4 * q4 + 1], (float)sv[4 * q4 + 2],
                               (float)sv[4 * q4 + 3]);
    }
  }
  // [11] = I + T_b M1, [12] = -T_b S^{-1}
  TPR a11[32], a12[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    a11[q] = TPR(0);
    a12[q] = TPR(0);
  }
  for (int t = 0; t < r; ++t) {
    const TPR tb = (TPR)Tb[lane * kCwLd + t];
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      a11[q] = fma(tb, M1P[t * kCwLd + q], a11[q]);
      a12[q] = fma(tb, SiP[t * kCwLd + q], a12[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    if (row_ok && q < r) {
      out[(size_t)q * n + lane] = (double)a11[q] + (q == lane ? 1.0 : 0.0);
      out[(size_t)(r + q) * n + lane] = -(double)a12[q];
    }
  }
  if (Kf) {
    float4* k0 = reinterpret_cast<float4*>(Kf + ((size_t)(2 * j) * 32 + lane) * kKfLd);
#pragma unroll
    for (int q4 = 0; q4 < 8; ++q4) {
      float e[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) e[u] = (float)a11[4 * q4 + u] + (4 * q4 + u == lane ? 1.f : 0.f);
      k0[q4] = make_float4(e[0], e[1], e[2], e[3]);
      k0[8 + q4] = make_float4((float)-a12[4 * q4], (float)-a12[4 * q4 + 1], (float)-a12[4 * q4 + 2],
                               (float)-a12[4 * q4 + 3]);
    }
  }
  if (lane == 0) {
    node_ld[2 * j] = la;
    node_ld[2 * j + 1] = sing >= 0 ? 0.0 : (neg ? -1.0 : 1.0);
    if (sing >= 0) set_status(st, HODLR_ERR_SINGULAR_COUPLING, heap_first + j, r + sing);
  }
}

// Levels with few parents: the same computation by four warps per parent,
// warp w holding columns 8w .. 8w+7 of every row (lane = row), so that the
// FP64 work of one parent is spread over the SM's four sub-partitions (one
// warp alone runs its FP64 instructions on one of them and, at the top
// levels, is pure latency). Per Gauss-Jordan step the warp owning column k
// finds the pivot and publishes (p, pivot, column k) through shared memory
// (double-buffered by step parity); one barrier per step.
template <bool FULL>
__global__ void __launch_bounds__(128) coupling_factor_cta4_kernel(int64_t N, int r, int c,
                                                                   const double* __restrict__ P, int64_t cpn_read,
                                                                   double* __restrict__ Kinv,
                                                                   double* __restrict__ node_ld, DevStatus* st,
                                                                   int64_t heap_first, float* __restrict__ Kf) {
  using TPR = typename std::conditional<FULL, double, float>::type;
  __shared__ double Ta[32 * kCwLd], Tb[32 * kCwLd], X[32 * kCwLd];
  __shared__ double sh_f[2][32];
  __shared__ double sh_piv[2];
  __shared__ int sh_p[2];
  __shared__ TPR M1s[32 * kCwLd], Sis[32 * kCwLd];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j = blockIdx.x;
  const int64_t cpn = chunks_per_node(N, c);
  const size_t slot = (size_t)r * r * c;
  const int anc = r * (c - 1);
  const int64_t qa = 2 * j * cpn, qb = (2 * j + 1) * cpn;
  const int c0 = warp * 8;  // this warp's columns

  // T_a, T_b (warp w gathers columns 8w .. 8w+7)
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) {
    const int col = c0 + cc;
    double a = 0.0, b = 0.0;
    if (lane < r && col < r) {
      const double* pa = P + qa * slot + (size_t)(anc + col) * r + lane;
      const double* pb = P + qb * slot + (size_t)(anc + col) * r + lane;
      for (int64_t q = 0; q < cpn_read; ++q) {
        a += pa[q * slot];
        b += pb[q * slot];
      }
    }
    Ta[lane * kCwLd + col] = a;
    Tb[lane * kCwLd + col] = b;
    if constexpr (!FULL) {  // FP32 copies for the BF16 factor's S, in M1s / Sis until the products
      M1s[lane * kCwLd + col] = (float)a;
      Sis[lane * kCwLd + col] = (float)b;
    }
  }
  __syncthreads();
  // row `lane`, columns c0.. of S = I - T_a T_b (FP32 products for the BF16
  // factor, as in the one-warp kernel)
  double s[8];
  if constexpr (FULL) {
#pragma unroll
    for (int q = 0; q < 8; ++q) s[q] = lane == c0 + q ? 1.0 : 0.0;
    for (int t = 0; t < r; ++t) {
      const double a = Ta[lane * kCwLd + t];
#pragma unroll
      for (int q = 0; q < 8; ++q) s[q] = fma(-a, Tb[t * kCwLd + c0 + q], s[q]);
    }
  } else {
    float sf[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) sf[q] = lane == c0 + q ? 1.f : 0.f;
    for (int t = 0; t < r; ++t) {
      const float a = M1s[lane * kCwLd + t];
#pragma unroll
      for (int q = 0; q < 8; ++q) sf[q] = fmaf(-a, Sis[t * kCwLd + c0 + q], sf[q]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) s[q] = (double)sf[q];
  }

  bool used = false;
  double mypiv = 1.0;
  int mypos = lane, mystep = lane, ninv = 0;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const int buf = k & 1;
    const int ow = k >> 3, kk = k & 7;
    if (warp == ow) {
      const int idx = pivot_lane(s[kk], used);
      const double pv = __shfl_sync(kFull, s[kk], idx);
      sh_f[buf][lane] = s[kk];
      if (lane == 0) {
        sh_p[buf] = idx;
        sh_piv[buf] = pv;
      }
    }
    __syncthreads();
    const int p = sh_p[buf];
    const double piv = sh_piv[buf];
    const double rp = piv != 0.0 ? 1.0 / piv : 0.0;
    if (lane < k) ninv += p < mypos ? 1 : 0;
    if (lane == k) {
      mypiv = piv;
      mypos = p;
    }
    const bool isp = lane == p;
    if (isp) {
      used = true;
      mystep = k;
    }
    const double coef = isp ? rp : -sh_f[buf][lane] * rp;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const double pvq = __shfl_sync(kFull, s[q], p);
      s[q] = (warp == ow && q == kk) ? coef : fma(coef, pvq, isp ? 0.0 : s[q]);
    }
  }

  double la = lane < r ? log(fabs(mypiv)) : 0.0;
  int neg = ((lane < r && mypiv < 0.0) ? 1 : 0) ^ (ninv & 1);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    la += __shfl_xor_sync(kFull, la, off);
    neg ^= __shfl_xor_sync(kFull, neg, off);
  }
  const unsigned zero = __ballot_sync(kFull, lane < r && mypiv == 0.0);
  const int sing = zero ? __ffs(zero) - 1 : -1;

  // tableau -> X; row k of S^{-1}, columns c0.. : S^{-1}(k, i) = X(p_k, step(i))
#pragma unroll
  for (int q = 0; q < 8; ++q) X[lane * kCwLd + c0 + q] = s[q];
  __syncthreads();
  double sv[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) sv[i] = X[mypos * kCwLd + __shfl_sync(kFull, mystep, i)];
  double svc[8];  // this warp's columns of the row (the array above is only indexed statically)
#pragma unroll
  for (int q = 0; q < 8; ++q) svc[q] = X[mypos * kCwLd + __shfl_sync(kFull, mystep, c0 + q)];
  // M1 = S^{-1} T_a, columns c0..
  TPR m1[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) m1[q] = TPR(0);
#pragma unroll
  for (int i = 0; i < 32; ++i)
#pragma unroll
    for (int q = 0; q < 8; ++q) m1[q] = fma((TPR)sv[i], (TPR)Ta[i * kCwLd + c0 + q], m1[q]);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    M1s[lane * kCwLd + c0 + q] = m1[q];
    Sis[lane * kCwLd + c0 + q] = (TPR)svc[q];
  }
  __syncthreads();
  const int n = 2 * r;
  double* out = Kinv + (size_t)j * n * n;
  const bool row_ok = lane < r;
  constexpr int kKfLd = 2 * 32 + 4;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int col = c0 + q;
    if (row_ok && col < r) {
      out[(size_t)col * n + r + lane] = -(double)m1[q];  // [21]
      out[(size_t)(r + col) * n + r + lane] = svc[q];     // [22]
    }
  }
  if (Kf) {
    float* k1 = Kf + ((size_t)(2 * j + 1) * 32 + lane) * kKfLd;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      k1[c0 + q] = (float)-m1[q];
      k1[32 + c0 + q] = (float)svc[q];
    }
  }
  // [11] = I + T_b M1, [12] = -T_b S^{-1}, columns c0..
  TPR a11[8], a12[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    a11[q] = TPR(0);
    a12[q] = TPR(0);
  }
  for (int t = 0; t < r; ++t) {
    const TPR tb = (TPR)Tb[lane * kCwLd + t];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      a11[q] = fma(tb, M1s[t * kCwLd + c0 + q], a11[q]);
      a12[q] = fma(tb, Sis[t * kCwLd + c0 + q], a12[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int col = c0 + q;
    if (row_ok && col < r) {
      out[(size_t)col * n + lane] = (double)a11[q] + (col == lane ? 1.0 : 0.0);
      out[(size_t)(r + col) * n + lane] = -(double)a12[q];
    }
  }
  if (Kf) {
    float* k0 = Kf + ((size_t)(2 * j) * 32 + lane) * kKfLd;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      k0[c0 + q] = (float)a11[q] + (c0 + q == lane ? 1.f : 0.f);
      k0[32 + c0 + q] = (float)-a12[q];
    }
  }
  if (threadIdx.x == 0) {
    node_ld[2 * j] = la;
    node_ld[2 * j + 1] = sing >= 0 ? 0.0 : (neg ? -1.0 : 1.0);
    if (sing >= 0) set_status(st, HODLR_ERR_SINGULAR_COUPLING, heap_first + j, r + sing);
  }
}

bool coupling_warp_supported(const Factor& F) { return F.d.r <= 32; }

bool coupling_writes_kf32(const Factor& F, int c) {
  return F.prec == HODLR_PREC_BF16 && F.d.r == 32 && F.kf32 != nullptr && g_use_tc &&
         update_tc_supported(F.d.N, F.d.r, c);
}

cudaError_t launch_coupling_factor_warp(const Factor& F, int c, cudaStream_t s) {
  const int r = F.d.r;
  const int n = 2 * r;
  const int64_t parents = (int64_t)1 << (c - 1);
  const size_t sm = (size_t)kCwWarps * 3 * 32 * kCwLd * sizeof(double);
  // FP64 and FP32 factors: the whole inverse in FP64; BF16 factor: S and its
  // inverse in FP64, the products of the explicit inverse in FP32
  const bool full = F.prec != HODLR_PREC_BF16 || g_coupling_fp64;
  if (full)
    cudaFuncSetAttribute(coupling_factor_warp_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  else
    cudaFuncSetAttribute(coupling_factor_warp_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  const double* Pc = F.P;
  const int64_t cpn_read = F.P_reduced ? 1 : chunks_per_node(F.d.N, c);
  float* kf = coupling_writes_kf32(F, c) ? F.kf32 : nullptr;
  if (parents <= 256) {  // few parents: four warps each (latency)
    auto k4 = full ? coupling_factor_cta4_kernel<true> : coupling_factor_cta4_kernel<false>;
    k4<<<(unsigned)parents, 128, 0, s>>>(F.d.N, r, c, Pc, cpn_read, F.K + F.Koff[c] * n * n,
                                         F.node_ld + 2 * F.Koff[c], F.status, parents, kf);
    note_launches(1);
    return cudaGetLastError();
  }
  const int64_t grid = (parents + kCwWarps - 1) / kCwWarps;
  {
    auto kern = full ? coupling_factor_warp_kernel<true> : coupling_factor_warp_kernel<false>;
    kern<<<(unsigned)grid, 32 * kCwWarps, sm, s>>>(
        F.d.N, r, c, F.P, F.P_reduced ? 1 : chunks_per_node(F.d.N, c), F.K + F.Koff[c] * n * n,
        F.node_ld + 2 * F.Koff[c], F.status, parents, coupling_writes_kf32(F, c) ? F.kf32 : nullptr);
    note_launches(1);
  }
  return cudaGetLastError();
}

}  // namespace hodlr
