// Coupling matrices of the BF16 factor: one warp per parent, FP32
// arithmetic, r <= 32 (the FP32 and FP64 factors keep the FP64 CTA kernel).
//
// Same quantities as the FP64 CTA kernel (level.cu): with
// K~ = [[I, T_b], [T_a, I]] (Eq. e:k) and the Schur complement
// S = I - T_a T_b,
//   K~^{-1} = [[I + T_b S^{-1} T_a, -T_b S^{-1}], [-S^{-1} T_a, S^{-1}]],
//   det K~ = det S,
// written in FP64 so that every consumer reads one layout. T_a and T_b are
// products of BF16 panels, so FP32 here adds nothing to their error (the
// paper's single-precision runs do every step in FP32), and FP32 runs at 64x
// the FP64 rate of this GPU.
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
#include "hodlr_internal.cuh"

namespace hodlr {

namespace {
constexpr int kCwWarps = 4;  // parents per CTA
constexpr int kCwLd = 33;    // padded row stride of the per-warp 32 x 32 tiles
constexpr unsigned kFull = 0xffffffffu;
}  // namespace

__global__ void __launch_bounds__(32 * kCwWarps) coupling_factor_warp_kernel(int64_t N, int r, int c,
                                                                              const double* __restrict__ P,
                                                                              int64_t cpn_read,
                                                                              double* __restrict__ Kinv,
                                                                              double* __restrict__ node_ld,
                                                                              DevStatus* st, int64_t heap_first) {
  extern __shared__ float cw_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t parents = (int64_t)1 << (c - 1);
  const int64_t j = (int64_t)blockIdx.x * kCwWarps + warp;
  if (j >= parents) return;  // whole warp; only warp-level synchronisation below
  float* Ta = cw_smem + (size_t)warp * 3 * 32 * kCwLd;  // row-major, ld 33
  float* Tb = Ta + 32 * kCwLd;
  float* X = Tb + 32 * kCwLd;
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
    Ta[lane * kCwLd + col] = (float)a;
    Tb[lane * kCwLd + col] = (float)b;
  }
  __syncwarp();

  // row `lane` of S = I - T_a T_b
  float s[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) s[q] = lane == q ? 1.f : 0.f;
  for (int t = 0; t < r; ++t) {
    const float a = Ta[lane * kCwLd + t];
#pragma unroll
    for (int q = 0; q < 32; ++q) s[q] = fmaf(-a, Tb[t * kCwLd + q], s[q]);
  }

  bool used = false;
  float mypiv = 1.f;  // lane k: the pivot of step k
  int mypos = lane;   // lane k: the pivot row p_k
  int mystep = lane;  // lane i: the step that took row i as pivot
  int ninv = 0;       // lane k: #{k' > k : p_k' < p_k}
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    float v = used ? -1.f : fabsf(s[k]);
    if (v != v) v = __int_as_float(0x7f800000);  // NaN ranks first: a total order keeps the choice warp-uniform
    int idx = lane;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float ov = __shfl_xor_sync(kFull, v, off);
      const int oi = __shfl_xor_sync(kFull, idx, off);
      if (ov > v || (ov == v && oi < idx)) {
        v = ov;
        idx = oi;
      }
    }
    const int p = idx;  // an unused lane: at least one has v >= 0 > -1
    const float piv = __shfl_sync(kFull, s[k], p);
    const float rp = piv != 0.f ? 1.f / piv : 0.f;
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
    const float f = s[k];
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      if (q == k) continue;
      const float w = __shfl_sync(kFull, s[q], p) * rp;
      s[q] = isp ? w : fmaf(-f, w, s[q]);
    }
    s[k] = isp ? rp : -f * rp;
  }

  // log|det S| (FP64, fixed butterfly), sign, first zero pivot
  double la = lane < r ? log(fabs((double)mypiv)) : 0.0;
  int neg = ((lane < r && mypiv < 0.f) ? 1 : 0) ^ (ninv & 1);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    la += __shfl_xor_sync(kFull, la, off);
    neg ^= __shfl_xor_sync(kFull, neg, off);
  }
  const unsigned zero = __ballot_sync(kFull, lane < r && mypiv == 0.f);
  const int sing = zero ? __ffs(zero) - 1 : -1;

  // S^{-1}(k, i) = tableau(p_k, step of row i)
#pragma unroll
  for (int q = 0; q < 32; ++q) X[lane * kCwLd + q] = s[q];
  __syncwarp();
  float sv[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) sv[i] = X[mypos * kCwLd + __shfl_sync(kFull, mystep, i)];

  // M1 = S^{-1} T_a (row `lane`)
  float m1[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) m1[q] = 0.f;
#pragma unroll
  for (int i = 0; i < 32; ++i)
#pragma unroll
    for (int q = 0; q < 32; ++q) m1[q] = fmaf(sv[i], Ta[i * kCwLd + q], m1[q]);
  __syncwarp();
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    Ta[lane * kCwLd + q] = sv[q];  // S^{-1}
    X[lane * kCwLd + q] = m1[q];   // M1
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
      out[(size_t)(r + q) * n + r + lane] = (double)sv[q];
    }
  }
  // [11] = I + T_b M1, [12] = -T_b S^{-1}
  float a11[32], a12[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    a11[q] = 0.f;
    a12[q] = 0.f;
  }
  for (int t = 0; t < r; ++t) {
    const float tb = Tb[lane * kCwLd + t];
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      a11[q] = fmaf(tb, X[t * kCwLd + q], a11[q]);
      a12[q] = fmaf(tb, Ta[t * kCwLd + q], a12[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    if (row_ok && q < r) {
      out[(size_t)q * n + lane] = (double)a11[q] + (q == lane ? 1.0 : 0.0);
      out[(size_t)(r + q) * n + lane] = -(double)a12[q];
    }
  }
  if (lane == 0) {
    node_ld[2 * j] = la;
    node_ld[2 * j + 1] = sing >= 0 ? 0.0 : (neg ? -1.0 : 1.0);
    if (sing >= 0) set_status(st, HODLR_ERR_SINGULAR_COUPLING, heap_first + j, r + sing);
  }
}

bool coupling_warp_supported(const Factor& F) { return F.prec == HODLR_PREC_BF16 && F.d.r <= 32; }

cudaError_t launch_coupling_factor_warp(const Factor& F, int c, cudaStream_t s) {
  const int r = F.d.r;
  const int n = 2 * r;
  const int64_t parents = (int64_t)1 << (c - 1);
  const size_t sm = (size_t)kCwWarps * 3 * 32 * kCwLd * sizeof(float);
  cudaFuncSetAttribute(coupling_factor_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  const int64_t grid = (parents + kCwWarps - 1) / kCwWarps;
  {
    coupling_factor_warp_kernel<<<(unsigned)grid, 32 * kCwWarps, sm, s>>>(
        F.d.N, r, c, F.P, F.P_reduced ? 1 : chunks_per_node(F.d.N, c), F.K + F.Koff[c] * n * n,
        F.node_ld + 2 * F.Koff[c], F.status, parents);
    note_launches(1);
  }
  return cudaGetLastError();
}

}  // namespace hodlr
