// Tensor-core (tcgen05) projection kernel of the BF16 factorization: for every
// row chunk q of child level c, P[q] = V(rows_q, block c-1)^T Y(rows_q, 0:rc)
// (Alg. 3 projections T and W of Eq. e:node1), with BF16 operands staged by
// TMA and FP32 accumulation in tensor memory.
//
// Formulation: D[m][n] = sum_k Y(row0+k, m) V(row0+k, vcol+n), i.e. the MMA's
// A operand is a 128-column tile of Y (K = rows, contiguous in memory: K-major)
// and B is the r-column V block (also K-major); M = 128 columns of Y, N = r,
// K = 64 rows per pipeline stage (4 MMAs of K = 16).
#include <cudaTypedefs.h>

#include "tc_common.cuh"

namespace hodlr {

namespace {

constexpr int kBK = 64;       // rows per stage
constexpr int kBM = 128;      // Y columns per tile
constexpr int kStages = 4;
constexpr uint32_t kABytes = kBM * kBK * 2;

template <int RN>
struct ProjSmem {
  static constexpr uint32_t kBBytes = RN * kBK * 2;
  static constexpr uint32_t kStageBytes = kABytes + kBBytes;
  static constexpr uint32_t kBarOff = kStages * kStageBytes;
  static constexpr uint32_t kBytes = kBarOff + 256 + 1024;  // + barriers, + alignment slack
};

}  // namespace

// Persistent: CTA i handles work items i, i + gridDim.x, ... (item = chunk q,
// column tile mt). Warp 0 lane 0 issues TMA loads, warp 1 lane 0 issues the
// MMAs, all four warps drain TMEM (warp w owns TMEM lanes 32w..32w+31 =
// columns of the tile) and write the FP64 partial.
template <int RN>
__global__ void __launch_bounds__(128) project_tc_kernel(const __grid_constant__ CUtensorMap mapY,
                                                         const __grid_constant__ CUtensorMap mapV, int64_t ch,
                                                         int64_t nchunks, int vcol, int rc, double* __restrict__ P,
                                                         DevStatus* st, int level) {
  using S = ProjSmem<RN>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S::kBarOff);
  uint64_t* empty = full + kStages;
  uint64_t* done = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr uint32_t kTmemCols = RN < 32 ? 32 : RN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(done, 1);
    tc::fence_mbar_init();
    tc::prefetch_tmap(&mapY);
    tc::prefetch_tmap(&mapV);
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, kTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int mtiles = (rc + kBM - 1) / kBM;
  const int64_t items = nchunks * mtiles;
  const int nk = (int)(ch / kBK);
  uint32_t kt_global = 0;  // stage-use counter shared by producer and MMA issuer (same sequence)
  uint32_t item_count = 0;
  bool ok = true;
  for (int64_t it = blockIdx.x; it < items; it += gridDim.x, ++item_count) {
    const int64_t q = it / mtiles;
    const int mt = (int)(it % mtiles);
    const int64_t row0 = q * ch;
    const int col0 = mt * kBM;
    if (warp == 0 && lane == 0) {
      for (int kt = 0; kt < nk; ++kt) {
        const uint32_t g = kt_global + kt;
        const int s = g % kStages;
        if (g >= (uint32_t)kStages && !tc::mbar_wait(&empty[s], ((g / kStages) - 1) & 1)) { ok = false; break; }
        uint8_t* a = smem + s * S::kStageBytes;
        tc::mbar_expect_tx(&full[s], S::kStageBytes);
        tc::tma_load_2d(a, &mapY, (int32_t)(row0 + kt * kBK), col0, &full[s]);
        tc::tma_load_2d(a + kABytes, &mapV, (int32_t)(row0 + kt * kBK), vcol, &full[s]);
      }
    } else if (warp == 1 && lane == 0) {
      constexpr uint32_t idesc = tc::idesc_bf16_f32(kBM, RN);
      for (int kt = 0; kt < nk; ++kt) {
        const uint32_t g = kt_global + kt;
        const int s = g % kStages;
        if (!tc::mbar_wait(&full[s], (g / kStages) & 1)) { ok = false; break; }
        tc::tc_fence_after();
        const uint32_t a = tc::smem_u32(smem + s * S::kStageBytes);
        const uint64_t ad = tc::desc_sw128_kmajor(a);
        const uint64_t bd = tc::desc_sw128_kmajor(a + kABytes);
#pragma unroll
        for (int kk = 0; kk < kBK / 16; ++kk)
          tc::mma_bf16(tmem, ad + 2 * kk, bd + 2 * kk, idesc, (kt | kk) != 0);
        tc::mma_commit(&empty[s]);
      }
      tc::mma_commit(done);
    }
    kt_global += nk;
    // epilogue: wait for the accumulator, drain TMEM, write the FP64 partial.
    // ok is made block-uniform first: tcgen05.ld is warp-collective.
    if (!tc::mbar_wait(done, item_count & 1)) ok = false;
    ok = __syncthreads_and(ok) != 0;
    tc::tc_fence_after();
    if (ok) {
      const int m = col0 + warp * 32 + lane;
      double* Pq = P + (size_t)q * RN * rc;
#pragma unroll
      for (int cc = 0; cc < (RN + 31) / 32; ++cc) {
        float v[32];
        tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + cc * 32, v);
        if (m < rc) {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (cc * 32 + j < RN) Pq[(size_t)m * RN + cc * 32 + j] = (double)v[j];
        }
      }
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (!__syncthreads_and(ok)) break;
  }
  // the producer's loads have all landed once the last full[] phases completed
  if (warp == 0 && lane == 0) {
    for (int s = 0; s < kStages && (uint32_t)s < kt_global; ++s) {
      const uint32_t last = kt_global - 1 - ((kt_global - 1 - s) % kStages);
      if (!tc::mbar_wait(&full[last % kStages], (last / kStages) & 1)) ok = false;
    }
  }
  if (!ok && threadIdx.x == 0) set_status(st, HODLR_ERR_TIMEOUT, level, 0);
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2-D BF16 tensor map over a column-major rows x cols matrix (leading
// dimension ld elements), box = box_rows (inner) x box_cols, 128-byte swizzle.
bool make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows,
              int box_cols) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)box_rows, (cuuint32_t)box_cols};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 148;
  }
  return n;
}

template <int RN>
cudaError_t project_tc_go(const __nv_bfloat16* Vp, int64_t ldv, const __nv_bfloat16* Y, int64_t N, int rL, int c,
                          int rc, double* P, DevStatus* st, cudaStream_t s) {
  using S = ProjSmem<RN>;
  CUtensorMap mY, mV;
  if (!make_map(&mY, Y, N, rL, N, kBK, kBM)) return cudaErrorInvalidValue;
  if (!make_map(&mV, Vp, N, rL, ldv, kBK, RN)) return cudaErrorInvalidValue;
  const int64_t ch = chunk_rows(N, c);
  const int64_t nch = num_chunks(N, c);
  const int64_t items = nch * ((rc + kBM - 1) / kBM);
  const int per_sm = (int)((227 * 1024) / S::kBytes);
  int64_t grid = (int64_t)sm_count() * (per_sm < 1 ? 1 : per_sm);
  if (grid > items) grid = items;
  cudaFuncSetAttribute(project_tc_kernel<RN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kBytes);
  { project_tc_kernel<RN><<<(unsigned)grid, 128, S::kBytes, s>>>(mY, mV, ch, nch, (c - 1) * RN, rc, P, st, c); note_launches(1); }
  return cudaGetLastError();
}

}  // namespace

bool project_tc_supported(int64_t N, int r, int c) {
  return (r == 32 || r == 64) && chunk_rows(N, c) % kBK == 0 && encode_fn() != nullptr;
}

cudaError_t launch_project_tc(int64_t N, int r, int L, int c, const __nv_bfloat16* Vp, int64_t ldv,
                              const __nv_bfloat16* Y, double* P, DevStatus* st, cudaStream_t s) {
  ProfScope prof_(KC_PROJECT_TC, s);
  const int rc = r * c;
  note_work(2.0 * (double)N * r + 2.0 * (double)N * rc + 8.0 * num_chunks(N, c) * r * rc, 2.0 * N * r * (double)rc);
  if (r == 32) return project_tc_go<32>(Vp, ldv, Y, N, r * L, c, rc, P, st, s);
  return project_tc_go<64>(Vp, ldv, Y, N, r * L, c, rc, P, st, s);
}


// ===========================================================================
// Coupling solve fused into the tensor-core ancestor update of the BF16 factor
// (Eq. e:node1 and Eq. e:node2, Alg. 3). With Rhs = [W_beta; W_alpha] the raw
// projections of the two children of a parent (2r x anc, rows 0..r-1 from the
// second child, as the right-hand side of K~ [w_first; w_second]) and K~^{-1}
// the parent's coupling inverse,
//   W'_alpha = K~^{-1}(rows of alpha, :) Rhs,
//   Y(rows, 0:anc) -= Y_own W'_alpha = (Y_own K~^{-1}(rows of alpha, :)) Rhs.
//
// Step 1 (rhs_bf16_kernel, once per level): Rhs^T of every parent rounded to
// BF16 and stored in the K-major core-matrix layout of a tcgen05 B operand
// (8-row x 16-byte cores, LBO = 128 B between cores along K, SBO = 2r/8 * 128 B
// between 8-row groups), one contiguous block per kFuNC ancestor columns, so
// that one bulk copy stages it.
// Step 2 (update_coupled_tc_kernel): per 128-row tile of a node, TMA brings the
// own block Y_own (128 x r); Z = Y_own K~^{-1}(alpha rows, :) (128 x 2r) is
// formed on the CUDA cores in FP32 and rounded to BF16 into the A layout; per
// chunk of kFuNC ancestor columns a bulk copy brings Rhs^T and TMA the old Y
// tile, one tcgen05.mma kind::f16 chain (K = 2r) accumulates Z Rhs in TMEM,
// and the epilogue subtracts it from the staged tile, which TMA stores back.
namespace {

constexpr int kFuNC = 128;   // ancestor columns per MMA chunk (N of the MMA)
constexpr int kFuBox = 32;   // columns per TMA box of Y (box = 128 rows x 32 columns)

template <int RK>
struct FusedSmem {
  static constexpr int K2 = 2 * RK;
  static constexpr uint32_t kABytes = 128 * K2 * 2;       // Z, K-major cores
  static constexpr uint32_t kBBytes = kFuNC * K2 * 2;     // Rhs^T chunk
  static constexpr int kKLd = K2 + 4;                     // padded row: 4-way instead of 32-way store conflicts
  static constexpr uint32_t kKBytes = RK * kKLd * 4;      // K~^{-1}(alpha rows, :), FP32
  static constexpr uint32_t kOwnBytes = 128 * RK * 2;     // Y_own tile [k][m]
  static constexpr uint32_t kYBytes = 128 * kFuNC * 2;    // old / new Y tile [j][m]
  static constexpr uint32_t kBarOff = kABytes + kBBytes + kKBytes + kOwnBytes + kYBytes;
  static constexpr uint32_t kBytes = kBarOff + 64 + 128;  // 3 mbarriers + TMEM slot, + alignment slack
};

// Rhs^T of every parent of child level c into the B layout above. Thread per
// 16-byte core row (8 consecutive K entries of one ancestor column); threads
// with consecutive (nn & 7) write one 128-byte core matrix together.
template <int RK>
__global__ void rhs_bf16_kernel(int c, const double* __restrict__ P, int64_t pstride, int anc,
                                uint8_t* __restrict__ out) {
  constexpr int K2 = 2 * RK;
  constexpr int KG = K2 / 8;
  constexpr uint32_t kSBO = KG * 128;
  const int64_t parents = (int64_t)1 << (c - 1);
  const int64_t per_parent = (int64_t)anc * KG;
  const int64_t total = parents * per_parent;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / per_parent;
    const int64_t w = e % per_parent;
    const int lo = (int)(w & 7);
    const int64_t g = w >> 3;              // (nn >> 3) * KG + kg
    const int kg = (int)(g % KG);
    const int nn = (int)((g / KG) * 8 + lo);
    // rows 0..r-1: second child 2j+1; rows r..2r-1: first child 2j
    const int k0 = kg * 8;
    const double* src = k0 < RK ? P + (2 * j + 1) * pstride + (int64_t)nn * RK + k0
                                : P + (2 * j) * pstride + (int64_t)nn * RK + (k0 - RK);
    const double2 a = *reinterpret_cast<const double2*>(src);
    const double2 b = *reinterpret_cast<const double2*>(src + 2);
    const double2 cc = *reinterpret_cast<const double2*>(src + 4);
    const double2 d = *reinterpret_cast<const double2*>(src + 6);
    auto pack = [](double x, double y) {
      return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn((float)x)) |
             ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn((float)y)) << 16);
    };
    const int chunk = nn / kFuNC, nl = nn % kFuNC;
    uint8_t* dst = out + (size_t)j * anc * K2 * 2 + (size_t)chunk * kFuNC * K2 * 2 + (size_t)(nl >> 3) * kSBO +
                   (size_t)kg * 128 + (size_t)(nl & 7) * 16;
    *reinterpret_cast<uint4*>(dst) = make_uint4(pack(a.x, a.y), pack(b.x, b.y), pack(cc.x, cc.y), pack(d.x, d.y));
  }
}

__device__ __forceinline__ void bulk_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   tc::smem_u32(dst)),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(tc::smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int32_t x, int32_t y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(tc::smem_u32(src))
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// 2-D BF16 tensor map without swizzle over the column-major N x cols matrix Y
// (ld N): box = 128 rows x kFuBox columns, stored in shared memory as
// [column][row] (column j of the box at j * 256 bytes).
bool make_map_plain(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {128, (cuuint32_t)kFuBox};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

template <int RK>
__global__ void __launch_bounds__(256, RK == 32 ? 2 : 1) update_coupled_tc_kernel(const __grid_constant__ CUtensorMap mapY, int64_t N,
                                                                int c, const uint8_t* __restrict__ rhs,
                                                                const double* __restrict__ Kinv, int anc,
                                                                DevStatus* st) {
  using S = FusedSmem<RK>;
  constexpr int K2 = 2 * RK;
  constexpr uint32_t kSBO = (K2 / 8) * 128;
  constexpr uint32_t kTmemCols = kFuNC;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  uint8_t* sA = smem;
  uint8_t* sB = sA + S::kABytes;
  float* sK = reinterpret_cast<float*>(sB + S::kBBytes);
  __nv_bfloat16* sOwn = reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<uint8_t*>(sK) + S::kKBytes);
  __nv_bfloat16* sY = reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<uint8_t*>(sOwn) + S::kOwnBytes);
  uint64_t* bar_own = reinterpret_cast<uint64_t*>(smem + S::kBarOff);
  uint64_t* bar_ld = bar_own + 1;
  uint64_t* bar_mma = bar_own + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_own + 3);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    tc::mbar_init(bar_own, 1);
    tc::mbar_init(bar_ld, 1);
    tc::mbar_init(bar_mma, 1);
    tc::fence_mbar_init();
    tc::prefetch_tmap(&mapY);
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, kTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int64_t n = N >> c;
  const int64_t tiles = N / 128;
  const int nchunks = (anc + kFuNC - 1) / kFuNC;
  bool ok = true;
  uint32_t ph_own = 0, ph_ld = 0, ph_mma = 0;
  // copies / MMAs issued by thread 0 and not yet waited for (thread 0's view)
  bool own_pending = false, ld_pending = false, mma_pending = false;
  for (int64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
    const int64_t row0 = t * 128;
    const int64_t node = row0 / n;
    const int64_t parent = node >> 1;
    const int first = (node & 1) == 0;
    const uint8_t* rhs_j = rhs + (size_t)parent * anc * K2 * 2;
    if (tid == 0) {
      // the previous tile's last store must have left sY before it is refilled
      bulk_wait_read0();
      tc::mbar_expect_tx(bar_own, S::kOwnBytes);
#pragma unroll
      for (int b = 0; b < RK / kFuBox; ++b)
        tc::tma_load_2d(sOwn + b * 128 * kFuBox, &mapY, (int32_t)row0, (c - 1) * RK + b * kFuBox, bar_own);
      const int nc = anc < kFuNC ? anc : kFuNC;
      tc::mbar_expect_tx(bar_ld, (uint32_t)nc * K2 * 2 + (uint32_t)nc * 128 * 2);
      bulk_load_1d(sB, rhs_j, (uint32_t)nc * K2 * 2, bar_ld);
      for (int b = 0; b < nc / kFuBox; ++b) tc::tma_load_2d(sY + b * 128 * kFuBox, &mapY, (int32_t)row0, b * kFuBox, bar_ld);
      own_pending = ld_pending = true;
    }
    // K~^{-1}(alpha rows, :) -> sK[k][q]  (FP64 column-major 2r x 2r)
    const double* Kj = Kinv + (size_t)parent * K2 * K2;
    const int rowoff = first ? 0 : RK;
    for (int e = tid; e < RK * K2; e += blockDim.x) {
      const int k = e % RK, q = e / RK;
      sK[k * S::kKLd + q] = (float)Kj[(size_t)q * K2 + rowoff + k];
    }
    __syncthreads();
    ok = __syncthreads_and(tc::mbar_wait(bar_own, ph_own)) != 0;
    if (!ok) break;
    ph_own ^= 1;
    own_pending = false;
    // Z = Y_own K~^{-1}(alpha rows, :): thread pair per row, each half of 2r
    {
      const int m = tid & 127, half = tid >> 7;
      float yv[RK];
#pragma unroll
      for (int k = 0; k < RK; ++k) yv[k] = __bfloat162float(sOwn[k * 128 + m]);
#pragma unroll
      for (int g = 0; g < RK / 8; ++g) {  // 8 output columns -> one 16-byte core row
        const int q0 = half * RK + g * 8;
        float z[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) z[u] = 0.f;
#pragma unroll
        for (int k = 0; k < RK; ++k) {
          const float4 k0 = *reinterpret_cast<const float4*>(sK + k * S::kKLd + q0);
          const float4 k1 = *reinterpret_cast<const float4*>(sK + k * S::kKLd + q0 + 4);
          z[0] = fmaf(yv[k], k0.x, z[0]);
          z[1] = fmaf(yv[k], k0.y, z[1]);
          z[2] = fmaf(yv[k], k0.z, z[2]);
          z[3] = fmaf(yv[k], k0.w, z[3]);
          z[4] = fmaf(yv[k], k1.x, z[4]);
          z[5] = fmaf(yv[k], k1.y, z[5]);
          z[6] = fmaf(yv[k], k1.z, z[6]);
          z[7] = fmaf(yv[k], k1.w, z[7]);
        }
        uint32_t pk[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          pk[u] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(z[2 * u])) |
                  ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(z[2 * u + 1])) << 16);
        const int kg = q0 / 8;
        *reinterpret_cast<uint4*>(sA + kg * 128 + (m >> 3) * kSBO + (m & 7) * 16) =
            make_uint4(pk[0], pk[1], pk[2], pk[3]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int ch = 0; ch < nchunks && ok; ++ch) {
      const int col0 = ch * kFuNC;
      const int nc = (anc - col0) < kFuNC ? (anc - col0) : kFuNC;  // multiple of 32 (anc = r (c-1))
      if (ch > 0 && tid == 0) {
        bulk_wait_read0();
        tc::mbar_expect_tx(bar_ld, (uint32_t)nc * K2 * 2 + (uint32_t)nc * 128 * 2);
        bulk_load_1d(sB, rhs_j + (size_t)col0 * K2 * 2, (uint32_t)nc * K2 * 2, bar_ld);
        for (int b = 0; b < nc / kFuBox; ++b)
          tc::tma_load_2d(sY + b * 128 * kFuBox, &mapY, (int32_t)row0, col0 + b * kFuBox, bar_ld);
        ld_pending = true;
      }
      tc::tc_fence_before();
      ok = __syncthreads_and(tc::mbar_wait(bar_ld, ph_ld)) != 0;  // also orders the Z writes before the MMA
      if (!ok) break;
      ph_ld ^= 1;
      ld_pending = false;
      tc::tc_fence_after();
      if (tid == 0) {
        const uint32_t idesc = tc::idesc_bf16_f32(128, nc);
        const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
#pragma unroll
        for (int ks = 0; ks < K2 / 16; ++ks)
          tc::mma_bf16(tmem, tc::desc_noswz_kmajor(a0 + ks * 256, 128, kSBO),
                       tc::desc_noswz_kmajor(b0 + ks * 256, 128, kSBO), idesc, ks != 0);
        tc::mma_commit(bar_mma);
        mma_pending = true;
      }
      ok = __syncthreads_and(tc::mbar_wait(bar_mma, ph_mma)) != 0;  // block-uniform before warp-collective loads
      if (!ok) break;
      ph_mma ^= 1;
      mma_pending = false;
      tc::tc_fence_after();
      // warps w and w+4 share TMEM lanes 32 (w % 4) .. +31 and split the columns
      const int m = (warp & 3) * 32 + lane;
      for (int cb = (warp >> 2) * 32; cb < nc; cb += 64) {
        float v[32];
        tc::tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + cb, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          __nv_bfloat16* p = sY + (cb + j) * 128 + m;
          *p = __float2bfloat16_rn(__bfloat162float(*p) - v[j]);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc::tc_fence_before();
      __syncthreads();
      tc::tc_fence_after();
      if (tid == 0) {
        for (int b = 0; b < nc / kFuBox; ++b)
          tma_store_2d(&mapY, sY + b * 128 * kFuBox, (int32_t)row0, col0 + b * kFuBox);
        bulk_commit();
      }
    }
  }
  if (tid == 0) {
    // a wait that gave up leaves its copies / MMAs in flight: let them land
    // (bounded) before the shared memory and TMEM are released
    if (own_pending) tc::mbar_wait(bar_own, ph_own);
    if (ld_pending) tc::mbar_wait(bar_ld, ph_ld);
    if (mma_pending) tc::mbar_wait(bar_mma, ph_mma);
    bulk_wait0();
    if (!ok) set_status(st, HODLR_ERR_TIMEOUT, c, 2);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

bool update_tc_supported(int64_t N, int r, int c) {
  return (r == 32 || r == 64) && ((N >> c) % 128) == 0 && encode_fn() != nullptr;
}

size_t rhs_bf16_bytes(const hodlr_desc& d) {
  // max over child levels c of 2^(c-1) parents x (r (c-1)) x 2r BF16
  size_t best = 0;
  for (int c = 2; c <= d.L; ++c) {
    const size_t b = ((size_t)1 << (c - 1)) * (size_t)d.r * (c - 1) * 2 * d.r * 2;
    if (b > best) best = b;
  }
  return best;
}

cudaError_t launch_update_coupled_tc(const Factor& F, int c, cudaStream_t s) {
  const int64_t N = F.d.N;
  const int r = F.d.r;
  const int anc = r * (c - 1);
  if (anc <= 0) return cudaSuccess;
  const int64_t cpn = chunks_per_node(N, c);
  const int64_t pstride = cpn * (int64_t)r * r * c;  // node -> its first chunk's slot (reduced)
  const int64_t parents = (int64_t)1 << (c - 1);
  {
    ProfScope prof_(KC_COUPLING_APPLY, s);
    note_work(8.0 * (double)(1ll << c) * r * anc + 2.0 * (double)parents * anc * 2 * r, 0.0);
    const int64_t total = parents * (int64_t)anc * (2 * r / 8);
    int64_t grid = (total + 255) / 256;
    if (grid > 16 * (int64_t)sm_count()) grid = 16 * (int64_t)sm_count();
    if (r == 32) {
      rhs_bf16_kernel<32><<<(unsigned)grid, 256, 0, s>>>(c, F.P, pstride, anc, F.rhs16);
    } else {
      rhs_bf16_kernel<64><<<(unsigned)grid, 256, 0, s>>>(c, F.P, pstride, anc, F.rhs16);
    }
    note_launches(1);
  }
  ProfScope prof_(KC_UPDATE_TC, s);
  note_work(2.0 * (double)N * r + 4.0 * (double)N * anc + 4.0 * (double)parents * anc * r +
                32.0 * (double)parents * r * r,
            4.0 * N * r * (double)anc + 4.0 * N * r * (double)r);
  CUtensorMap mY;
  __nv_bfloat16* Y = static_cast<__nv_bfloat16*>(F.Y);
  if (!make_map_plain(&mY, Y, N, (int64_t)r * F.d.L, N)) return cudaErrorInvalidValue;
  const double* Kc = F.K + F.Koff[c] * 4 * r * r;
  const int64_t tiles = N / 128;
  if (r == 32) {
    using S = FusedSmem<32>;
    const int per_sm = (int)((227 * 1024) / S::kBytes);
    int64_t grid = (int64_t)sm_count() * (per_sm < 1 ? 1 : per_sm);
    if (grid > tiles) grid = tiles;
    cudaFuncSetAttribute(update_coupled_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kBytes);
    { update_coupled_tc_kernel<32><<<(unsigned)grid, 256, S::kBytes, s>>>(mY, N, c, F.rhs16, Kc, anc, F.status); note_launches(1); }
  } else {
    using S = FusedSmem<64>;
    const int per_sm = (int)((227 * 1024) / S::kBytes);
    int64_t grid = (int64_t)sm_count() * (per_sm < 1 ? 1 : per_sm);
    if (grid > tiles) grid = tiles;
    cudaFuncSetAttribute(update_coupled_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kBytes);
    { update_coupled_tc_kernel<64><<<(unsigned)grid, 256, S::kBytes, s>>>(mY, N, c, F.rhs16, Kc, anc, F.status); note_launches(1); }
  }
  return cudaGetLastError();
}

}  // namespace hodlr

namespace hodlr {

// ===========================================================================
// Tensor-core leaf stage of the BF16 factor (Alg. 3, first step; Eq. e:u):
// Y(I_b, :) = D_b^{-1} U_big(I_b, :) for every leaf b of m = 128 rows, with
// tcgen05.mma kind::tf32 (FP32 operands read as TF32, FP32 accumulation):
// M = 128 rows of the leaf, N = kLaNC columns of U per MMA chain, K = 128.
//   A = D_b^{-1}: written by the leaf inverse in the K-major core-matrix
//       layout (8-row x 16-byte cores, LBO = 128 B along K, SBO = 4096 B
//       between 8-row groups), 64 KB per leaf, staged by one bulk copy;
//   B = U(I_b, cols)^T: U is column-major, i.e. K-contiguous per column; each
//       thread converts 4 consecutive FP64 rows of one column to FP32 and
//       stores one 16-byte core row;
//   D (TMEM, FP32) -> BF16 into a [column][row] tile, stored by TMA.
// FP64 -> FP32 for the TF32 operand: the FP64 sign and exponent are rebiased
// and the top 23 significand bits kept (truncation; the MMA uses the top 10),
// on the integer pipe; magnitudes below 2^-126 become zero.
namespace {

constexpr int kLaNC = 64;  // columns of U per MMA chain

struct LeafTcSmem {
  static constexpr uint32_t kABytes = 128 * 128 * 4;
  static constexpr uint32_t kBBytes = kLaNC * 128 * 4;
  static constexpr uint32_t kYBytes = 128 * kLaNC * 2;
  static constexpr uint32_t kBarOff = kABytes + kBBytes + kYBytes;
  static constexpr uint32_t kBytes = kBarOff + 64 + 128;
};

__device__ __forceinline__ uint32_t f64_to_f32_trunc_bits(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu);
  const uint32_t mant = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  uint32_t bits = sign | ((uint32_t)(e - 896) << 23) | mant;
  if (e <= 896) bits = sign;                                                 // tiny -> signed zero
  if (e >= 1151) bits = sign | 0x7F800000u | ((hi & 0xFFFFFu) | lo ? 0x400000u : 0u);  // inf / NaN
  return bits;
}

__host__ __device__ constexpr uint32_t idesc_tf32_f32(int M, int N) {
  return (1u << 4)                     // D format: F32
         | (2u << 7)                   // A format: TF32
         | (2u << 10)                  // B format: TF32
         | ((uint32_t)(N >> 3) << 17)  // N / 8
         | ((uint32_t)(M >> 4) << 24); // M / 16
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

}  // namespace

__global__ void __launch_bounds__(256, 2) leaf_apply_tc_kernel(const __grid_constant__ CUtensorMap mapY,
                                                               int64_t nleaf, int rL,
                                                               const float* __restrict__ Acore,
                                                               const double* __restrict__ U, int64_t ldu,
                                                               DevStatus* st) {
  using S = LeafTcSmem;
  constexpr uint32_t kSBO = 4096;  // 32 cores along K x 128 B
  constexpr uint32_t kTmemCols = kLaNC;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  uint8_t* sA = smem;
  uint8_t* sB = sA + S::kABytes;
  __nv_bfloat16* sY = reinterpret_cast<__nv_bfloat16*>(sB + S::kBBytes);
  uint64_t* bar_a = reinterpret_cast<uint64_t*>(smem + S::kBarOff);
  uint64_t* bar_mma = bar_a + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_a + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    tc::mbar_init(bar_a, 1);
    tc::mbar_init(bar_mma, 1);
    tc::fence_mbar_init();
    tc::prefetch_tmap(&mapY);
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, kTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int nchunks = rL / kLaNC + (rL % kLaNC ? 1 : 0);
  bool ok = true;
  uint32_t ph_a = 0, ph_mma = 0;
  bool a_pending = false, mma_pending = false;  // thread 0's view
  for (int64_t b = blockIdx.x; b < nleaf && ok; b += gridDim.x) {
    const int64_t row0 = b * 128;
    if (tid == 0) {
      tc::mbar_expect_tx(bar_a, S::kABytes);
      bulk_load_1d(sA, Acore + (size_t)b * 128 * 128, S::kABytes, bar_a);
      a_pending = true;
    }
    for (int ch = 0; ch < nchunks && ok; ++ch) {
      const int col0 = ch * kLaNC;
      const int nc = (rL - col0) < kLaNC ? (rL - col0) : kLaNC;  // multiple of 32
      // B: nc columns x 128 rows; item = (8-column group, k quad, column in group)
      {
        constexpr int kItems = kLaNC * 32;  // 16-byte core rows of a full chunk
        constexpr int kPer = kItems / 256;
        double2 v0[kPer], v1[kPer];
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
          const int it = tid + u * 256;
          const int jl = it & 7, kq = (it >> 3) & 31, jg = it >> 8;
          const int j = jg * 8 + jl;
          if (j < nc) {
            const double* src = U + (int64_t)(col0 + j) * ldu + row0 + kq * 4;
            v0[u] = *reinterpret_cast<const double2*>(src);
            v1[u] = *reinterpret_cast<const double2*>(src + 2);
          }
        }
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
          const int it = tid + u * 256;
          const int jl = it & 7, kq = (it >> 3) & 31, jg = it >> 8;
          if (jg * 8 + jl < nc)
            *reinterpret_cast<uint4*>(sB + jg * kSBO + kq * 128 + jl * 16) =
                make_uint4(f64_to_f32_trunc_bits(v0[u].x), f64_to_f32_trunc_bits(v0[u].y),
                           f64_to_f32_trunc_bits(v1[u].x), f64_to_f32_trunc_bits(v1[u].y));
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc::tc_fence_before();
      if (ch == 0) {
        ok = __syncthreads_and(tc::mbar_wait(bar_a, ph_a)) != 0;
        if (!ok) break;
        ph_a ^= 1;
        a_pending = false;
      } else {
        __syncthreads();
      }
      tc::tc_fence_after();
      if (tid == 0) {
        const uint32_t idesc = idesc_tf32_f32(128, nc);
        const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
#pragma unroll
        for (int ks = 0; ks < 16; ++ks)  // K = 8 per MMA: two cores along K
          mma_tf32(tmem, tc::desc_noswz_kmajor(a0 + ks * 256, 128, kSBO),
                   tc::desc_noswz_kmajor(b0 + ks * 256, 128, kSBO), idesc, ks != 0);
        tc::mma_commit(bar_mma);
        mma_pending = true;
        bulk_wait_read0();  // the previous chunk's store has left sY
      }
      ok = __syncthreads_and(tc::mbar_wait(bar_mma, ph_mma)) != 0;
      if (!ok) break;
      ph_mma ^= 1;
      mma_pending = false;
      tc::tc_fence_after();
      // warps w and w+4 share TMEM lanes 32 (w % 4) .. +31 and split the columns
      const int m = (warp & 3) * 32 + lane;
      for (int cb = (warp >> 2) * 32; cb < nc; cb += 64) {
        float v[32];
        tc::tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + cb, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) sY[(cb + j) * 128 + m] = __float2bfloat16_rn(v[j]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc::tc_fence_before();
      __syncthreads();
      tc::tc_fence_after();
      if (tid == 0) {
        for (int bx = 0; bx < nc / kFuBox; ++bx)
          tma_store_2d(&mapY, sY + bx * 128 * kFuBox, (int32_t)row0, col0 + bx * kFuBox);
        bulk_commit();
      }
    }
  }
  if (tid == 0) {
    if (a_pending) tc::mbar_wait(bar_a, ph_a);
    if (mma_pending) tc::mbar_wait(bar_mma, ph_mma);
    bulk_wait0();
    if (!ok) set_status(st, HODLR_ERR_TIMEOUT, 0, 3);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

bool leaf_apply_tc_supported(const Factor& F) {
  return g_use_tc && F.prec == HODLR_PREC_BF16 && F.d.m == 128 && (F.d.r * F.d.L) % 32 == 0 &&
         encode_fn() != nullptr;
}

cudaError_t launch_leaf_apply_tc(const Factor& F, const double* U, int64_t ldu, cudaStream_t s) {
  ProfScope prof_(KC_LEAF_SOLVE, s);
  const int64_t N = F.d.N;
  const int rL = F.d.r * F.d.L;
  const int64_t nleaf = (int64_t)1 << F.d.L;
  note_work(8.0 * (double)N * rL + 2.0 * (double)N * rL + 4.0 * (double)nleaf * 128 * 128,
            2.0 * (double)N * 128 * rL);
  CUtensorMap mY;
  if (!make_map_plain(&mY, F.Y, N, rL, N)) return cudaErrorInvalidValue;
  using S = LeafTcSmem;
  const int per_sm = (int)((227 * 1024) / (S::kBytes + 1024));
  int64_t grid = (int64_t)sm_count() * (per_sm < 1 ? 1 : per_sm);
  if (grid > nleaf) grid = nleaf;
  cudaFuncSetAttribute(leaf_apply_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kBytes);
  {
    leaf_apply_tc_kernel<<<(unsigned)grid, 256, S::kBytes, s>>>(mY, nleaf, rL, reinterpret_cast<const float*>(F.P),
                                                                 U, ldu, F.status);
    note_launches(1);
  }
  return cudaGetLastError();
}

}  // namespace hodlr
