// Internal declarations shared by the libhodlr translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include "hodlr.h"

namespace hodlr {

// ---------------------------------------------------------------- status word
// First device-side error wins (atomicCAS on code). Kernels never trap.
struct DevStatus {
  int code;
  int pad;
  long long where;
  long long detail;
};

__device__ __forceinline__ void set_status(DevStatus* st, int code, long long where, long long detail) {
  if (atomicCAS(&st->code, 0, code) == 0) {
    st->where = where;
    st->detail = detail;
  }
}

// ---------------------------------------------------------------- conversions
__device__ __forceinline__ void cvt(double& d, double s) { d = s; }
__device__ __forceinline__ void cvt(float& d, double s) { d = (float)s; }
__device__ __forceinline__ void cvt(float& d, float s) { d = s; }
__device__ __forceinline__ void cvt(double& d, float s) { d = (double)s; }
__device__ __forceinline__ void cvt(float& d, __nv_bfloat16 s) { d = __bfloat162float(s); }
__device__ __forceinline__ void cvt(double& d, __nv_bfloat16 s) { d = (double)__bfloat162float(s); }
__device__ __forceinline__ void cvt(__nv_bfloat16& d, float s) { d = __float2bfloat16_rn(s); }
__device__ __forceinline__ void cvt(__nv_bfloat16& d, double s) { d = __float2bfloat16_rn((float)s); }

template <typename TD, typename TS>
__device__ __forceinline__ TD conv(TS s) {
  TD d;
  cvt(d, s);
  return d;
}

// FP64 -> FP32 on the integer pipe (this GPU's FP64 pipe, which also runs
// the F2F conversion, is narrow): the sign and exponent rebiased and the top
// 23 significand bits kept, i.e. rounding toward zero; magnitudes below
// 2^-126 become a signed zero, finite magnitudes of 2^128 and above become
// infinity, NaN stays NaN.
__device__ __forceinline__ uint32_t f64_to_f32_trunc_bits(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu);
  const uint32_t mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  uint32_t bits = sign | ((uint32_t)(e - 896) << 23) | mant;
  if (e <= 896) bits = sign;
  if (e >= 1151) bits = sign | 0x7F800000u | ((e == 2047 && ((hi & 0xFFFFFu) | lo)) ? 0x400000u : 0u);
  return bits;
}
// isfinite of an FP64 value from its exponent bits (integer pipe).
__device__ __forceinline__ bool f64_finite_bits(double x) {
  return (((uint32_t)__double2hiint(x) >> 20) & 0x7FFu) != 0x7FFu;
}

// Four consecutive elements (16-byte aligned for float / double, 8-byte for
// BF16) loaded in one or two vector accesses and converted; store4 likewise.
template <typename TA>
__device__ __forceinline__ void load4(const __nv_bfloat16* p, TA (&o)[4]) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  o[0] = (TA)__uint_as_float(u.x << 16);
  o[1] = (TA)__uint_as_float(u.x & 0xffff0000u);
  o[2] = (TA)__uint_as_float(u.y << 16);
  o[3] = (TA)__uint_as_float(u.y & 0xffff0000u);
}
template <typename TA>
__device__ __forceinline__ void load4(const float* p, TA (&o)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = (TA)v.x;
  o[1] = (TA)v.y;
  o[2] = (TA)v.z;
  o[3] = (TA)v.w;
}
template <typename TA>
__device__ __forceinline__ void load4(const double* p, TA (&o)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  o[0] = (TA)a.x;
  o[1] = (TA)a.y;
  o[2] = (TA)b.x;
  o[3] = (TA)b.y;
}
template <typename TA>
__device__ __forceinline__ void store4(float* p, const TA (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
}
template <typename TA>
__device__ __forceinline__ void store4(double* p, const TA (&v)[4]) {
  *reinterpret_cast<double2*>(p) = make_double2((double)v[0], (double)v[1]);
  *reinterpret_cast<double2*>(p + 2) = make_double2((double)v[2], (double)v[3]);
}
template <typename TA>
__device__ __forceinline__ void store4(__nv_bfloat16* p, const TA (&v)[4]) {
  __nv_bfloat16 b[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) b[i] = __float2bfloat16_rn((float)v[i]);
  uint2 u;
  u.x = (uint32_t)__bfloat16_as_ushort(b[0]) | ((uint32_t)__bfloat16_as_ushort(b[1]) << 16);
  u.y = (uint32_t)__bfloat16_as_ushort(b[2]) | ((uint32_t)__bfloat16_as_ushort(b[3]) << 16);
  *reinterpret_cast<uint2*>(p) = u;
}

// ---------------------------------------------------------------- tree geometry
// Child level c (1..L): nodes of n_c = N >> c = m * 2^(L-c) rows. Projections
// are split into row chunks of ch(c) rows, n_c halved until it is at most
// kChunkMax (so ch divides n_c, whatever m is); chunk q covers rows
// [q*ch, (q+1)*ch) and belongs to node q / (n_c / ch).
constexpr int64_t kChunkMax = 1024;

__host__ __device__ inline int64_t node_rows(int64_t N, int c) { return N >> c; }
__host__ __device__ inline int64_t chunk_rows(int64_t N, int c) {
  int64_t n = N >> c;
  while (n > kChunkMax) n >>= 1;
  return n;
}
__host__ __device__ inline int64_t num_chunks(int64_t N, int c) { return N / chunk_rows(N, c); }
__host__ __device__ inline int64_t chunks_per_node(int64_t N, int c) {
  return node_rows(N, c) / chunk_rows(N, c);
}

// ---------------------------------------------------------------- factor object
enum class Prec { F64 = 0, F32 = 1, BF16 = 3 };

struct Factor {
  hodlr_desc d;
  hodlr_prec prec;
  cudaStream_t stream;
  // leaf LUs (column-major m x m blocks) in FP64 or FP32, row permutations
  void* lu;          // double* (FP64) or float*
  // LU form: nleaf * m, row i of the factored block is row perm[i] of D_b.
  // Inverse form (low precision, m <= 128): lu holds the scaled Gauss-Jordan
  // tableau T with D_b^{-1}(step(r), p_c) = T(r, c); perm[b m + c] = p_c and
  // perm[N + b m + r] = step(r)
  int* perm;
  // Y_big (N x rL, ld N): double (FP64), float (FP32) or bf16 (BF16)
  void* Y;
  // V_big as used by the level kernels: the caller's V (FP64) or a copy
  const void* Vp;
  int64_t ldvp;
  // coupling LUs: level c (1..L) parents j at Kc[c] + j*(2r)^2 (FP64), perms likewise
  double* K;
  int* Kperm;
  int64_t Koff[26];  // offset (in parents) of child level c's first parent
  // projection partials (FP64): max over levels of num_chunks * r * r*c
  double* P;
  size_t P_elems;
  // BF16 factor: per-parent right-hand sides [W_beta; W_alpha]^T of one level
  // in the tensor cores' operand layout (rhs_bf16_bytes)
  uint8_t* rhs16;
  // BF16 factor: K~^{-1}(rows of alpha, :) in FP32 for every child of one
  // level, rows padded to 2r + 4 (kf32_bytes)
  float* kf32;
  // BF16 factor with m = 128: the leaf stage runs on the tensor cores; the
  // leaf inverse then also writes D_b^{-1} in operand layout into P (P is
  // free until the level loop starts)
  bool leaf_tc = false;
  // set while the factor's level loop has already summed each node's chunk
  // partials into its first slot (top levels), so the coupling kernels read
  // one slot per node
  bool P_reduced = false;
  // log-determinant pieces: leaves (logabs, sign) then parents in Koff order
  double* leaf_ld;
  double* node_ld;
  double* ld_out;    // 2 doubles
  DevStatus* status;
};

size_t factor_workspace_bytes(const hodlr_desc& d, hodlr_prec prec);

// ---------------------------------------------------------------- launch accounting
enum KernelClass {
  KC_LEAF_LU = 0, KC_LEAF_SOLVE, KC_PROJECT, KC_COUPLING, KC_COUPLING_APPLY, KC_UPDATE, KC_REDUCE,
  KC_LEAF_MATVEC, KC_VECTOR, KC_LOGDET, KC_PROJECT_TC, KC_UPDATE_TC, KC_MATVEC, KC_COMPRESS, KC_COUNT
};
// Called by every launcher right after its kernel launch(es): counts them and,
// when profiling is on, records the closing event of the bracket that
// prof_begin opened on the same stream.
void note_launches(int n);
// Algorithmic bytes moved and flops done by the launch(es) of the current
// bracket (the kernel's definition, not its actual traffic); summed per class
// while profiling is on.
void note_work(double bytes, double flops);
struct ProfScope {
  int cls;
  cudaStream_t s;
  void* a;
  ProfScope(int c, cudaStream_t st);
  ~ProfScope();
};

// ---------------------------------------------------------------- kernels (launchers)
// Leaf stage
cudaError_t launch_leaf_lu(const Factor& F, const double* D, cudaStream_t s);
// X_b <- D_b^{-1} X_b (trans = 0) or D_b^{-T} X_b (trans = 1) for all leaves,
// columns [0, ncols); in and out may alias.
template <typename TIN, typename TOUT>
cudaError_t launch_leaf_solve(const Factor& F, const TIN* in, int64_t ldin, TOUT* out, int64_t ldout,
                              int ncols, int trans, cudaStream_t s);

// Level stage. P[q] (r x ncols, ld r) = Bas(rows_q, block)^T R(rows_q, 0:ncols)
// for every chunk q of child level c. Bas is N x (r*L) (ld ldb), block c-1.
template <typename TB, typename TR>
cudaError_t launch_project(int64_t N, int r, int c, const TB* Bas, int64_t ldb, int bas_block,
                           const TR* R, int64_t ldr, int ncols, double* P, int acc_fp64, cudaStream_t s);

// R(rows of node, 0:ncols) += alpha * Bas(rows, block) * W(node') with W(node')
// = Wbase + node' * wstride (r x ncols, ld r), node' = node ^ swap_sibling.
template <typename TB, typename TR>
cudaError_t launch_update(int64_t N, int r, int c, const TB* Bas, int64_t ldb, int bas_block,
                          TR* R, int64_t ldr, int ncols, const double* Wbase, int64_t wstride,
                          int swap_sibling, double alpha, int acc_fp64, cudaStream_t s);

// Coupling (FP64). Factor mode: reduce partials of both children, form K~,
// LU, log|det|, solve for the ancestor columns; W' written to each child's
// first chunk slot. Solve modes reuse the stored LU.
cudaError_t launch_coupling_factor(const Factor& F, int c, cudaStream_t s);
// FP64 warp-per-parent variant (r <= 32)
bool coupling_warp_supported(const Factor& F);
cudaError_t launch_coupling_factor_warp(const Factor& F, int c, cudaStream_t s);
// true when the warp coupling kernel of level c also writes the FP32 rows
// K~^{-1}(rows of alpha, :) the fused tensor-core update stages (F.kf32)
bool coupling_writes_kf32(const Factor& F, int c);
// reduced: the chunk partials of every node were already summed into its
// first slot (launch_reduce_chunks)
cudaError_t launch_coupling_solve(const Factor& F, int c, double* P, int k, int trans, cudaStream_t s,
                                  bool reduced = false);
// Sum the chunk partials of every node into the node's first chunk slot.
cudaError_t launch_reduce_chunks(int64_t N, int r, int c, double* P, int ncols, cudaStream_t s);
// One right-hand side, low-precision panels TB, FP32 vector: the level loop
// of the forward solve in two launches per level (parent sums + coupling
// solve; update of level c fused with the projection of level c - 1).
// parts: solve_k1_parts_elems doubles; W: 2^L * r floats.
size_t solve_k1_parts_elems(const hodlr_desc& d);
template <typename TB>
bool solve_k1_supported(const Factor& F, const TB* Y, const TB* Vp, int64_t ldvp, const float* x);
template <typename TB>
cudaError_t launch_solve_k1_chain(const Factor& F, const TB* Y, const TB* Vp, int64_t ldvp, float* x,
                                  double* parts, float* W, cudaStream_t s);

// Low-precision factors with m <= 128 keep D_b^{-1} (FP32) instead of the LU
// factors; their leaf solves are GEMMs with it.
bool leaf_uses_inverse(const Factor& F);
cudaError_t launch_leaf_inv(const Factor& F, const double* D, cudaStream_t s);
bool leaf_inv_tc_supported(const Factor& F);
cudaError_t launch_leaf_inv_tc(const Factor& F, const double* D, float* Dtc, cudaStream_t s);
template <typename TIN, typename TOUT>
cudaError_t launch_leaf_apply_inv(const Factor& F, const TIN* in, int64_t ldin, TOUT* out, int64_t ldout, int ncols,
                                  int trans, cudaStream_t s);

// Coupling application with any slot width (gradient sweeps).
cudaError_t launch_coupling_apply_any(const Factor& F, int c, double* P, int64_t sw, int nrhs, int first_is_beta,
                                      int trans, cudaStream_t s);
// Gradient helpers (grad.cu)
cudaError_t launch_leaf_identity(int64_t N, int m, double* E, cudaStream_t s);
template <typename TB>
cudaError_t launch_leaf_outer(int64_t N, int m, int K, const double* A, int64_t lda, const TB* B, int64_t ldb,
                              double alpha, double beta, const double* Tadd, double* out, cudaStream_t s);
cudaError_t launch_coupling_h(const Factor& F, int c, double* H, double* HT, cudaStream_t s);

// One-right-hand-side matvec in three launches (matvec1.cu).
size_t matvec1_scratch_elems(const hodlr_desc& d);
cudaError_t launch_matvec1(const hodlr_desc& d, const double* D, const double* U, const double* V, const double* x,
                           double* y, double* scratch, cudaStream_t s);

// Leaf stage of the matvec: Y_b = D_b X_b (FP64).
cudaError_t launch_leaf_matvec(const hodlr_desc& d, const double* D, const double* X, int64_t ldx,
                               double* Y, int64_t ldy, int k, cudaStream_t s);

// Vectors
template <typename TD, typename TS>
cudaError_t launch_copy_cols(int64_t N, int k, const TS* src, int64_t lds, TD* dst, int64_t ldd, cudaStream_t s);
cudaError_t launch_axpby_cols(int64_t N, int k, double a, const double* x, int64_t ldx, double b, double* y,
                              int64_t ldy, cudaStream_t s);  // y = a x + b y
// out[j] = sum_i x(i,j)*y(i,j) for j < k (deterministic two-stage), scratch >= dot_scratch_elems(N,k)
size_t dot_scratch_elems(int64_t N, int k);
cudaError_t launch_dots(int64_t N, int k, const double* x, int64_t ldx, const double* y, int64_t ldy,
                        double* out, double* scratch, cudaStream_t s);
// out[j] = sum_i X(i, j) * w(i) for j < k (X N x k, ld ldx) -> multi-dot with one vector
cudaError_t launch_multidot(int64_t N, int k, const double* X, int64_t ldx, const double* w, double* out,
                            double* scratch, cudaStream_t s);
// w -= X h  (X N x k, h k device vector)
cudaError_t launch_gemv_sub(int64_t N, int k, const double* X, int64_t ldx, const double* h, double* w,
                            cudaStream_t s);
cudaError_t launch_bdots(int64_t N, int k, int nq, const double* V, const double* w, double* out, double* scratch,
                         cudaStream_t s);
cudaError_t launch_bgemv(int64_t N, int k, int nq, const double* V, const double* coef, double alpha, double* y,
                         int64_t ldy, cudaStream_t s);
cudaError_t launch_scale_inv_norm(int64_t N, int k, const double* w, const double* nrm2, double* out,
                                  cudaStream_t s);
cudaError_t launch_logdet_reduce(const Factor& F, cudaStream_t s);

// Tensor-core (tcgen05 + TMA) projection of the BF16 factor; supported when
// r is 32 or 64 and the level's row chunks are multiples of 64 rows.
bool project_tc_supported(int64_t N, int r, int c);
cudaError_t launch_project_tc(int64_t N, int r, int L, int c, const __nv_bfloat16* Vp, int64_t ldv,
                              const __nv_bfloat16* Y, double* P, DevStatus* st, cudaStream_t s,
                              uint8_t* rhs16 = nullptr);
cudaError_t launch_project_tc32(int64_t N, int r, int L, int c, const float* Vp, int64_t ldv, const float* Y,
                                double* P, DevStatus* st, cudaStream_t s);
// Coupling solve fused into the tensor-core ancestor update (BF16 factor):
// uses the raw projections in each node's first slot, the coupling inverses
// and the BF16 right-hand-side staging area rhs16 (rhs_bf16_bytes).
bool update_tc_supported(int64_t N, int r, int c);
size_t rhs_bf16_bytes(const hodlr_desc& d);
size_t kf32_bytes(const hodlr_desc& d);
cudaError_t launch_update_coupled_tc(const Factor& F, int c, cudaStream_t s, bool rhs_ready = false);
// Tensor-core (kind::tf32) leaf stage Y = D_b^{-1} U of the BF16 factor
// (m = 128, r L a multiple of 32; U 16-byte aligned with even ldu).
bool leaf_apply_tc_supported(const Factor& F);
cudaError_t launch_leaf_apply_tc(const Factor& F, const double* U, int64_t ldu, cudaStream_t s);
// Set by hodlr_tc_enable (process-wide; default on).
hodlr_status check_desc_ext(const hodlr_desc* d);
extern bool g_use_tc;
extern bool g_coupling_fp64;  // BF16 factor: form S = I - T_a T_b and the inverse's products in FP64

}  // namespace hodlr
