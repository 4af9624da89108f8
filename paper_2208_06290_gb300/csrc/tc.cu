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

constexpr int kBK = 64;       // rows per stage (BF16; 32 for FP32 tiles: 128 bytes of each column either way)
constexpr int kBM = 128;      // Y columns per tile
constexpr uint32_t kABytes = kBM * 128;  // 128 columns x 128 bytes of rows
constexpr int kPjThreads = 192;          // 4 epilogue warps, producer, MMA issuer

// Stage ring: 5 x 20 KB (r = 32) or 4 x 24 KB (r = 64), two CTAs per SM.
template <int RN>
struct ProjSmem {
  static constexpr int kNS = RN <= 32 ? 5 : 4;
  static constexpr uint32_t kBBytes = RN * 128;
  static constexpr uint32_t kStageBytes = kABytes + kBBytes;
  static constexpr uint32_t kBarOff = kNS * kStageBytes;
  static constexpr uint32_t kBytes = kBarOff + 256 + 1024;  // + barriers, TMEM slot, flag; + alignment slack
  static_assert(8 * (2 * kNS + 5) + 8 <= 256, "barrier area");
  static_assert(2 * (kBytes + 1024) <= 228 * 1024, "two CTAs per SM");
};


__device__ __forceinline__ bool wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  const uint32_t a = tc::smem_u32(bar);
  const long long t0 = clock64();
  for (uint32_t it = 0; it < tc::kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 15) == 15) {
      if (*abort_flag) return false;
      if (clock64() - t0 > tc::kSpinCycles) {
        *abort_flag = 1;
        return false;
      }
    }
  }
  *abort_flag = 1;
  return false;
}

__device__ __forceinline__ void named_bar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// AND of pred over the `count` threads of named barrier `id` (all of them
// take the same branch afterwards).
__device__ __forceinline__ bool named_bar_and(int id, int count, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n barrier.cta.red.and.pred q, %2, %3, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id), "r"(count)
      : "memory");
  return r != 0;
}

// Lane 0 waits, the warp learns the outcome (warp-uniform).
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  int r = 1;
  if ((threadIdx.x & 31) == 0) r = wait_or_abort(bar, parity, abort_flag) ? 1 : 0;
  return __shfl_sync(0xffffffffu, r, 0) != 0;
}

}  // namespace

// Persistent and warp-specialized (192 threads); CTA i handles work items
// i, i + gridDim.x, ... (item = chunk q, column tile mt):
//   warp 4, lane 0 (producer): TMA loads of the Y tile and the V block into a
//     ring of stages, running ahead across items;
//   warp 5, lane 0 (MMA issuer): one tcgen05.mma chain per item (K = the
//     chunk's rows) into one of two TMEM accumulators;
//   warps 0-3 (epilogue; warp w reads TMEM lanes 32w..32w+31 = columns of the
//     tile): drain an accumulator and write the FP64 partial while the MMAs of
//     the next item run into the other one.
// Hand-offs are mbarriers; every wait is bounded and also gives up when
// another thread has raised the CTA's abort flag; the copies and MMAs in
// flight are let land (bounded) before the TMEM is freed.
// With rhs16 (levels where every node is one chunk, ahead of the fused
// update): the ancestor columns m < anc of a node's projection are written
// straight into the BF16 right-hand-side operand of its parent (the layout
// of rhs_bf16_kernel: rows 0..r-1 from the second child, r..2r-1 from the
// first), and only the own block (the coupling's T) into P in FP64.
// T = __nv_bfloat16 (BF16 factor, kind::f16, 64 rows per stage) or float
// (TF32 factor: FP32 tiles read by kind::tf32, 32 rows per stage); both give
// 128-byte swizzled rows, 4 MMAs of 32 bytes of K per stage.
template <int RN, typename T = __nv_bfloat16>
__global__ void __launch_bounds__(kPjThreads) project_tc_kernel(const __grid_constant__ CUtensorMap mapY,
                                                                const __grid_constant__ CUtensorMap mapV, int64_t ch,
                                                                int64_t nchunks, int vcol, int rc,
                                                                double* __restrict__ P, DevStatus* st, int level,
                                                                uint8_t* __restrict__ rhs16, int anc) {
  using S = ProjSmem<RN>;
  constexpr int NS = S::kNS;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S::kBarOff);  // [NS] TMA transaction count
  uint64_t* empty = full + NS;                                       // [NS] MMA commit
  uint64_t* acc_full = empty + NS;                                   // [2]  MMA commit
  uint64_t* acc_empty = acc_full + 2;                                // [2]  128 epilogue threads
  uint64_t* drain = acc_empty + 2;                                   //      MMA commit at exit
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr uint32_t kAcc = RN < 32 ? 32 : RN;  // TMEM columns of one accumulator
  constexpr uint32_t kTmemCols = 2 * kAcc;

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      tc::mbar_init(&acc_full[a], 1);
      tc::mbar_init(&acc_empty[a], 128);
    }
    tc::mbar_init(drain, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
    tc::prefetch_tmap(&mapY);
    tc::prefetch_tmap(&mapV);
  }
  if (warp == 5) tc::tmem_alloc(tmem_slot, kTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  constexpr int kRows = 128 / (int)sizeof(T);  // rows per stage
  constexpr bool kTF32 = sizeof(T) == 4;
  const int mtiles = (rc + kBM - 1) / kBM;
  const int64_t items = nchunks * mtiles;
  const int nk = (int)(ch / kRows);

  if (warp == 4) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      uint32_t g = 0;  // stage uses issued
      bool ok = true;
      for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x) {
        const int64_t row0 = (it / mtiles) * ch;
        const int col0 = (int)(it % mtiles) * kBM;
        for (int kt = 0; kt < nk; ++kt, ++g) {
          const int s = g % NS;
          if (g >= (uint32_t)NS && !(ok = wait_or_abort(&empty[s], ((g / NS) - 1) & 1, abort_flag))) break;
          uint8_t* a = smem + s * S::kStageBytes;
          tc::mbar_expect_tx(&full[s], S::kStageBytes);
          tc::tma_load_2d(a, &mapY, (int32_t)(row0 + kt * kRows), col0, &full[s]);
          tc::tma_load_2d(a + kABytes, &mapV, (int32_t)(row0 + kt * kRows), vcol, &full[s]);
        }
      }
      // let the last copies land before the CTA can exit (bounded)
      for (uint32_t q = 0; q < (uint32_t)NS && q < g; ++q) {
        const uint32_t u = g - 1 - q;
        tc::mbar_wait(&full[u % NS], (u / NS) & 1);
      }
    }
  } else if (warp == 5) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = kTF32 ? tc::idesc_tf32_f32(kBM, RN) : tc::idesc_bf16_f32(kBM, RN);
      uint32_t g = 0, i = 0;
      bool ok = true, issued = false;
      for (int64_t it = blockIdx.x; it < items && ok; it += gridDim.x, ++i) {
        const uint32_t a = i & 1;
        if (i >= 2 && !(ok = wait_or_abort(&acc_empty[a], ((i >> 1) - 1) & 1, abort_flag))) break;
        tc::tc_fence_after();
        for (int kt = 0; kt < nk; ++kt, ++g) {
          const int s = g % NS;
          if (!(ok = wait_or_abort(&full[s], (g / NS) & 1, abort_flag))) break;
          tc::tc_fence_after();
          const uint32_t sa = tc::smem_u32(smem + s * S::kStageBytes);
          const uint64_t ad = tc::desc_sw128_kmajor(sa);
          const uint64_t bd = tc::desc_sw128_kmajor(sa + kABytes);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {  // 32 bytes of K each (16 BF16 / 8 TF32)
            if constexpr (kTF32)
              tc::mma_tf32(tmem + a * kAcc, ad + 2 * kk, bd + 2 * kk, idesc, (kt | kk) != 0);
            else
              tc::mma_bf16(tmem + a * kAcc, ad + 2 * kk, bd + 2 * kk, idesc, (kt | kk) != 0);
          }
          issued = true;
          tc::mma_commit(&empty[s]);
        }
        if (!ok) break;
        tc::mma_commit(&acc_full[a]);
      }
      // every MMA issued has finished before the TMEM is freed (bounded)
      if (issued) {
        tc::mma_commit(drain);
        tc::mbar_wait(drain, 0);
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    uint32_t i = 0;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x, ++i) {
      const int64_t q = it / mtiles;
      const int col0 = (int)(it % mtiles) * kBM;
      const uint32_t a = i & 1;
      if (!warp_wait(&acc_full[a], (i >> 1) & 1, abort_flag)) break;  // warp-uniform: tcgen05.ld is collective
      tc::tc_fence_after();
      const int m = col0 + warp * 32 + lane;
      double* Pq = P + (size_t)q * RN * rc;
      constexpr int K2 = 2 * RN;
      constexpr uint32_t kSBOr = (K2 / 8) * 128;
#pragma unroll
      for (int cc = 0; cc < (RN + 31) / 32; ++cc) {
        float v[32];
        tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + a * kAcc + cc * 32, v);
        if (!kTF32 && rhs16 && m < anc) {
          // row k = koff + n of the parent's [W_beta; W_alpha]^T, column m
          const int koff = (q & 1) ? 0 : RN;
          constexpr int kNC = 64;  // ancestor columns per block of the operand (the fused update's chunk)
          uint8_t* base = rhs16 + (size_t)(q >> 1) * anc * K2 * 2 + (size_t)(m / kNC) * kNC * K2 * 2 +
                          (size_t)((m % kNC) >> 3) * kSBOr + (size_t)(m & 7) * 16;
#pragma unroll
          for (int kg = 0; kg < 4; ++kg) {
            uint32_t pk[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
              pk[u] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[kg * 8 + 2 * u])) |
                      ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[kg * 8 + 2 * u + 1])) << 16);
            *reinterpret_cast<uint4*>(base + (size_t)((koff + cc * 32) / 8 + kg) * 128) =
                make_uint4(pk[0], pk[1], pk[2], pk[3]);
          }
        } else if (m < rc) {
          // 16-byte stores of the thread's 32 consecutive doubles
          double2* dst = reinterpret_cast<double2*>(Pq + (size_t)m * RN + cc * 32);
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (cc * 32 + 2 * j < RN) dst[j] = make_double2((double)v[2 * j], (double)v[2 * j + 1]);
        }
      }
      tc::tc_fence_before();
      tc::mbar_arrive(&acc_empty[a]);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (tid == 0 && *abort_flag) set_status(st, HODLR_ERR_TIMEOUT, level, 0);
  if (warp == 5) tc::tmem_dealloc(tmem, kTmemCols);
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
              int box_cols, bool fp32 = false) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  cuuint64_t strides[1] = {(cuuint64_t)ld * (fp32 ? 4 : 2)};
  cuuint32_t box[2] = {(cuuint32_t)box_rows, (cuuint32_t)box_cols};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
            const_cast<void*>(base), dims, strides, box, estr,
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

template <int RN, typename T>
cudaError_t project_tc_go(const T* Vp, int64_t ldv, const T* Y, int64_t N, int rL, int c,
                          int rc, double* P, DevStatus* st, cudaStream_t s, uint8_t* rhs16) {
  using S = ProjSmem<RN>;
  constexpr bool f32 = sizeof(T) == 4;
  constexpr int kRows = 128 / (int)sizeof(T);
  CUtensorMap mY, mV;
  // only the r c columns the level projects: the column tiles past them are
  // out of bounds for the copy engine (filled with zeros, not read)
  if (!make_map(&mY, Y, N, rc, N, kRows, kBM, f32)) return cudaErrorInvalidValue;
  if (!make_map(&mV, Vp, N, rL, ldv, kRows, RN, f32)) return cudaErrorInvalidValue;
  const int64_t ch = chunk_rows(N, c);
  const int64_t nch = num_chunks(N, c);
  const int64_t items = nch * ((rc + kBM - 1) / kBM);
  const int per_sm = (int)((227 * 1024) / S::kBytes);
  int64_t grid = (int64_t)sm_count() * (per_sm < 1 ? 1 : per_sm);
  if (grid > items) grid = items;
  cudaFuncSetAttribute(project_tc_kernel<RN, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kBytes);
  { project_tc_kernel<RN, T><<<(unsigned)grid, kPjThreads, S::kBytes, s>>>(mY, mV, ch, nch, (c - 1) * RN, rc, P, st, c,
                                                                      rhs16, RN * (c - 1)); note_launches(1); }
  return cudaGetLastError();
}

}  // namespace

bool project_tc_supported(int64_t N, int r, int c) {
  return (r == 32 || r == 64) && chunk_rows(N, c) % kBK == 0 && encode_fn() != nullptr;
}

cudaError_t launch_project_tc(int64_t N, int r, int L, int c, const __nv_bfloat16* Vp, int64_t ldv,
                              const __nv_bfloat16* Y, double* P, DevStatus* st, cudaStream_t s, uint8_t* rhs16) {
  ProfScope prof_(KC_PROJECT_TC, s);
  const int rc = r * c;
  const double anc = (double)r * (c - 1);
  note_work(2.0 * (double)N * r + 2.0 * (double)N * rc +
                (rhs16 ? 8.0 * num_chunks(N, c) * r * r + 2.0 * num_chunks(N, c) * r * anc
                       : 8.0 * num_chunks(N, c) * r * rc),
            2.0 * N * r * (double)rc);
  if (r == 32) return project_tc_go<32, __nv_bfloat16>(Vp, ldv, Y, N, r * L, c, rc, P, st, s, rhs16);
  return project_tc_go<64, __nv_bfloat16>(Vp, ldv, Y, N, r * L, c, rc, P, st, s, rhs16);
}

// TF32 factor: FP32 panels, projections on kind::tf32
cudaError_t launch_project_tc32(int64_t N, int r, int L, int c, const float* Vp, int64_t ldv, const float* Y,
                                double* P, DevStatus* st, cudaStream_t s) {
  ProfScope prof_(KC_PROJECT_TC, s);
  const int rc = r * c;
  note_work(4.0 * (double)N * r + 4.0 * (double)N * rc + 8.0 * num_chunks(N, c) * r * rc, 2.0 * N * r * (double)rc);
  if (r == 32) return project_tc_go<32, float>(Vp, ldv, Y, N, r * L, c, rc, P, st, s, nullptr);
  return project_tc_go<64, float>(Vp, ldv, Y, N, r * L, c, rc, P, st, s, nullptr);
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
// Step 2 (update_coupled_tc_kernel): per 128-row tile of a node, the own block
// Y_own (128 x r) and K~^{-1}(rows of alpha, :) (FP32 rows staged per child by
// the coupling kernel or kf32_kernel) are rounded to BF16 operands and
// Z = Y_own K~^{-1}(alpha rows, :) (128 x 2r) is formed by one tcgen05.mma
// chain (K = r) in TMEM, then rounded to BF16 into the A layout; per chunk of
// kFuNC ancestor columns one tcgen05.mma kind::f16 chain (K = 2r) accumulates
// Z Rhs in TMEM, and the epilogue subtracts it from the old Y tile, staged and
// stored by TMA. The roles and their pipeline are described at the kernel.
namespace {

constexpr int kFuNC = 64;    // ancestor columns per MMA chunk (N of the MMA; the projection's rhs16 epilogue uses the same)
constexpr int kFuBox = 32;   // columns per TMA box of Y (box = 128 rows x 32 columns)

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

// Y(x.., y..) += tile, element-wise in the L2 (BF16 add, round to nearest).
__device__ __forceinline__ void tma_reduce_add_2d(const CUtensorMap* map, const void* src, int32_t x, int32_t y) {
  asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(tc::smem_u32(src))
               : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
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

// Pipelined, warp-specialized form of step 2 (320 threads, persistent over
// 128-row tiles; every CTA walks tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// and chunks of kFuNC ancestor columns inside each tile in the same order):
//   warp 4, lane 0 (producer): TMA / bulk copies: per tile the own block
//     Y_own (128 x r) and the FP32 rows K~^{-1}(rows of alpha, :)
//     (precomputed per node, see kf32_kernel); per chunk the parent's Rhs^T
//     chunk into a ring of stages;
//   warps 0-3 (Z warps, thread per row): Y_own and K~^{-1}(alpha rows, :)^T
//     into BF16 K-major operands; after the Z product, Z from TMEM rounded to
//     BF16 into the A operand;
//   warp 5, lane 0 (MMA issuer): per tile the Z product (K = r) into TMEM
//     columns 128.., per chunk one tcgen05.mma chain (K = 2r) into one of two
//     TMEM accumulators;
//   warps 6-9 (epilogue, TMEM lane quarter = warp % 4): the accumulator,
//     negated and rounded to BF16, into one of two [column][row] tiles, which
//     one thread adds to Y by a TMA reduction (cp.reduce.async.bulk.tensor
//     .add: the L2 forms Y + (-Z Rhs) and rounds it to BF16), so the old Y
//     never passes through the SM.
// Hand-offs are mbarriers (full / empty pairs). Every wait is bounded and also
// gives up when another thread has raised the CTA's abort flag; on the way out
// thread 0 of each role lets its own copies and MMAs land (bounded) before the
// TMEM is freed.
namespace {

// Rhs^T stages, Z (A operand) and output buffers: four stages, one A buffer,
// one own-block buffer and two output tiles keep r = 32 at two CTAs per SM
// (109 KB of shared memory each).
template <int RK> constexpr int fu_stages() { return 4; }
template <int RK> constexpr int fu_abufs() { return 1; }
template <int RK> constexpr int fu_obufs() { return 1; }  // own-block / K~ rows buffers
constexpr int kFuOut = 2;                                  // output tiles (TMA reductions in flight)
constexpr int kFuThreads = 320;  // 10 warps

template <int RK>
struct FusedSmem {
  static constexpr int K2 = 2 * RK;
  static constexpr int kKLd = K2 + 4;                     // padded FP32 row of K~^{-1}(alpha rows, :)
  static constexpr uint32_t kOwnBytes = 128 * RK * 2;     // Y_own tile [k][m]
  static constexpr uint32_t kKfBytes = RK * kKLd * 4;
  static constexpr uint32_t kABytes = 128 * K2 * 2;       // Z, K-major cores
  static constexpr uint32_t kBBytes = kFuNC * K2 * 2;     // Rhs^T chunk
  static constexpr uint32_t kYBytes = 128 * kFuNC * 2;    // output tile -Z Rhs [j][m]
  static constexpr int NS = fu_stages<RK>();
  static constexpr int NA = fu_abufs<RK>();
  static constexpr int NO = fu_obufs<RK>();
  static constexpr uint32_t kAoBytes = 128 * RK * 2;      // Y_own, K-major cores (A of the Z product)
  static constexpr uint32_t kKbBytes = K2 * RK * 2;       // K~^{-1}(alpha rows, :)^T, K-major cores (its B)
  static constexpr uint32_t kOwnOff = 0;
  static constexpr uint32_t kKfOff = kOwnOff + NO * kOwnBytes;
  static constexpr uint32_t kAoOff = kKfOff + NO * kKfBytes;
  static constexpr uint32_t kKbOff = kAoOff + kAoBytes;
  static constexpr uint32_t kAOff = kKbOff + kKbBytes;
  static constexpr uint32_t kBOff = kAOff + NA * kABytes;
  static constexpr uint32_t kYOff = kBOff + NS * kBBytes;
  static constexpr uint32_t kBarOff = kYOff + kFuOut * kYBytes;
  static constexpr uint32_t kBytes = kBarOff + 256 + 128;  // barriers, TMEM slot, flag, + alignment slack
  static_assert(8 * (14 + 2 * NS) + 16 <= 256, "barrier area");
  static_assert(kBytes <= 227 * 1024, "shared memory per CTA");
};

// K~^{-1}(rows of alpha, :) in FP32 for every child alpha of level c,
// rows padded to 2r + 4 floats (the layout the fused update stages).
template <int RK>
__global__ void kf32_kernel(int c, const double* __restrict__ Kinv, float* __restrict__ Kf) {
  constexpr int K2 = 2 * RK, LD = K2 + 4;
  const int64_t nodes = (int64_t)1 << c;
  const int64_t total = nodes * RK * K2;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t node = e / (RK * K2);
    const int w = (int)(e % (RK * K2));
    const int q = w / RK, k = w % RK;  // k fastest: coalesced reads of a Kinv column
    const double* Kj = Kinv + (size_t)(node >> 1) * K2 * K2;
    const int rowoff = (node & 1) ? RK : 0;
    Kf[(size_t)node * RK * LD + (size_t)k * LD + q] = (float)Kj[(size_t)q * K2 + rowoff + k];
  }
}

}  // namespace

template <int RK>
__global__ void __launch_bounds__(kFuThreads, RK == 32 ? 2 : 1) update_coupled_tc_kernel(const __grid_constant__ CUtensorMap mapY,
                                                                          int64_t N, int c,
                                                                          const uint8_t* __restrict__ rhs,
                                                                          const float* __restrict__ Kf, int anc,
                                                                          DevStatus* st) {
  using S = FusedSmem<RK>;
  constexpr int NA = S::NA;
  constexpr int K2 = 2 * RK;
  constexpr uint32_t kSBO = (K2 / 8) * 128;
  constexpr uint32_t kTmemCols = 256;          // two chunk accumulators (2 x kFuNC) + the Z product (2r)
  constexpr uint32_t kZCol = 2 * kFuNC;
  constexpr uint32_t kSBOr = (RK / 8) * 128;   // 8-row group stride of the K = r operands
  constexpr int NO = S::NO;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  __nv_bfloat16* sOwn = reinterpret_cast<__nv_bfloat16*>(smem + S::kOwnOff);  // [NO][RK][128]
  float* sKf = reinterpret_cast<float*>(smem + S::kKfOff);                     // [NO][RK][kKLd]
  uint8_t* sAo = smem + S::kAoOff;
  uint8_t* sKb = smem + S::kKbOff;
  uint8_t* sA = smem + S::kAOff;                                               // [NA]
  uint8_t* sB = smem + S::kBOff;                                               // [stages]
  __nv_bfloat16* sY = reinterpret_cast<__nv_bfloat16*>(smem + S::kYOff);      // [kFuOut][kFuNC][128]
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S::kBarOff);
  uint64_t* own_full = bars;                        // [2]
  uint64_t* own_empty = bars + 2;                   // [2]   count 128 (Z threads)
  uint64_t* a_full = bars + 4;                      // [2]   count 128 (Z threads)
  uint64_t* a_empty = bars + 6;                     // [2]   MMA commit
  uint64_t* acc_full = bars + 8;                    // [2]   MMA commit
  uint64_t* acc_empty = bars + 10;                  // [2]   count 128 (epilogue threads)
  uint64_t* zin_full = bars + 12;                   //       count 128 (Z threads: A_own and B staged)
  uint64_t* z_done = bars + 13;                     //       MMA commit of the Z product
  uint64_t* ld_full = bars + 14;                    // [stages]
  uint64_t* b_empty = bars + 14 + S::NS;        // [stages] MMA commit
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 14 + 2 * S::NS);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 15 + 2 * S::NS);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&own_full[i], 1);
      tc::mbar_init(&own_empty[i], 128);
      tc::mbar_init(&a_full[i], 128);
      tc::mbar_init(&a_empty[i], 1);
      tc::mbar_init(&acc_full[i], 1);
      tc::mbar_init(&acc_empty[i], 128);
    }
    tc::mbar_init(zin_full, 128);
    tc::mbar_init(z_done, 1);
    for (int i = 0; i < S::NS; ++i) {
      tc::mbar_init(&ld_full[i], 1);
      tc::mbar_init(&b_empty[i], 1);
    }
    *abort_flag = 0;
    tc::fence_mbar_init();
    tc::prefetch_tmap(&mapY);
  }
  if (warp == 5) tc::tmem_alloc(tmem_slot, kTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int64_t n = N >> c;
  const int64_t tiles = N / 128;
  const int nch = (anc + kFuNC - 1) / kFuNC;

  if (warp == 4) {
    // ---------------------------------------------------------------- producer
    // the whole warp walks the schedule and waits; lane 0 issues the copies
    uint32_t g = 0, it = 0;
    int pend_own = 0, pend_ld = 0;  // copies issued (the drain below waits for their landing)
    bool ok = true;
    for (int64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++it) {
      const int64_t row0 = t * 128;
      const int64_t node = row0 / n;
      const int tb = it % NO;
      if (it >= (uint32_t)NO && !(ok = warp_wait(&own_empty[tb], ((it / NO) - 1) & 1, abort_flag))) break;
      if (lane == 0) {
        tc::mbar_expect_tx(&own_full[tb], S::kOwnBytes + S::kKfBytes);
#pragma unroll
        for (int b = 0; b < RK / kFuBox; ++b)
          tc::tma_load_2d(sOwn + (size_t)tb * 128 * RK + b * 128 * kFuBox, &mapY, (int32_t)row0,
                          (c - 1) * RK + b * kFuBox, &own_full[tb]);
        bulk_load_1d(sKf + (size_t)tb * RK * S::kKLd, Kf + (size_t)node * RK * S::kKLd, S::kKfBytes,
                     &own_full[tb]);
      }
      pend_own = it + 1;
      const uint8_t* rhs_j = rhs + (size_t)(node >> 1) * anc * K2 * 2;
      for (int ch = 0; ch < nch; ++ch, ++g) {
        const int col0 = ch * kFuNC;
        const int nc = (anc - col0) < kFuNC ? (anc - col0) : kFuNC;
        const int s = g % S::NS;
        if (g >= (uint32_t)S::NS && !(ok = warp_wait(&b_empty[s], ((g / S::NS) - 1) & 1, abort_flag))) break;
        if (lane == 0) {
          tc::mbar_expect_tx(&ld_full[s], (uint32_t)nc * K2 * 2);
          bulk_load_1d(sB + (size_t)s * S::kBBytes, rhs_j + (size_t)col0 * K2 * 2, (uint32_t)nc * K2 * 2,
                       &ld_full[s]);
        }
        pend_ld = g + 1;
        __syncwarp();
      }
    }
    // let the last copies land before the CTA can exit (bounded)
    if (lane == 0) {
      for (int q = 0; q < NO && q < pend_own; ++q) {
        const uint32_t last = pend_own - 1 - q;
        tc::mbar_wait(&own_full[last % NO], (last / NO) & 1);
      }
      for (int q = 0; q < S::NS && q < pend_ld; ++q) {
        const uint32_t gg = pend_ld - 1 - q;
        tc::mbar_wait(&ld_full[gg % S::NS], (gg / S::NS) & 1);
      }
    }
    __syncwarp();
  } else if (warp == 5) {
    // ---------------------------------------------------------------- MMA issuer
    // the whole warp walks the schedule and waits; lane 0 issues and commits
    uint32_t g = 0, it = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++it) {
      // Z = Y_own K~^{-1}(alpha rows, :): M = 128, N = 2r, K = r, into TMEM columns kZCol..
      if (!(ok = warp_wait(zin_full, it & 1, abort_flag))) break;
      tc::tc_fence_after();
      if (lane == 0) {
        const uint32_t idesc = tc::idesc_bf16_f32(128, K2);
        const uint32_t a0 = tc::smem_u32(sAo), b0 = tc::smem_u32(sKb);
#pragma unroll
        for (int ks = 0; ks < RK / 16; ++ks)
          tc::mma_bf16(tmem + kZCol, tc::desc_noswz_kmajor(a0 + ks * 256, 128, kSBOr),
                       tc::desc_noswz_kmajor(b0 + ks * 256, 128, kSBOr), idesc, ks != 0);
        tc::mma_commit(z_done);
      }
      __syncwarp();
      const int ab = it % NA;
      if (!(ok = warp_wait(&a_full[ab], (it / NA) & 1, abort_flag))) break;
      tc::tc_fence_after();
      for (int ch = 0; ch < nch; ++ch, ++g) {
        const int col0 = ch * kFuNC;
        const int nc = (anc - col0) < kFuNC ? (anc - col0) : kFuNC;
        const int s = g % S::NS, a = g & 1;
        if (!(ok = warp_wait(&ld_full[s], (g / S::NS) & 1, abort_flag))) break;
        if (g >= 2 && !(ok = warp_wait(&acc_empty[a], ((g >> 1) - 1) & 1, abort_flag))) break;
        tc::tc_fence_after();
        if (lane == 0) {
          const uint32_t idesc = tc::idesc_bf16_f32(128, nc);
          const uint32_t a0 = tc::smem_u32(sA + (size_t)ab * S::kABytes), b0 = tc::smem_u32(sB + (size_t)s * S::kBBytes);
#pragma unroll
          for (int ks = 0; ks < K2 / 16; ++ks)
            tc::mma_bf16(tmem + a * kFuNC, tc::desc_noswz_kmajor(a0 + ks * 256, 128, kSBO),
                         tc::desc_noswz_kmajor(b0 + ks * 256, 128, kSBO), idesc, ks != 0);
          tc::mma_commit(&acc_full[a]);
          tc::mma_commit(&b_empty[s]);
        }
        __syncwarp();
      }
      if (!ok) break;
      if (lane == 0) tc::mma_commit(&a_empty[ab]);  // sA[ab] may be refilled once this tile's MMAs are done
      __syncwarp();
    }
    // drain: the last commit covers every MMA issued (bounded)
    if (lane == 0 && g > 0) tc::mbar_wait(&acc_full[(g - 1) & 1], ((g - 1) >> 1) & 1);
    __syncwarp();
  } else if (warp < 4) {
    // ---------------------------------------------------------------- Z warps
    // stage Y_own and K~^{-1}(alpha rows, :)^T as BF16 K-major operands, let
    // the MMA issuer form Z in TMEM, then round Z to BF16 into the A operand
    const int m = tid;  // 0..127: tile row, and TMEM lane (warp % 4 = lane quarter)
    uint32_t it = 0;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x, ++it) {
      const int tb = it % NO;
      if (!wait_or_abort(&own_full[tb], (it / NO) & 1, abort_flag)) break;
      if (it >= 1 && !wait_or_abort(z_done, (it - 1) & 1, abort_flag)) break;  // previous Z product consumed sAo / sKb
      const __nv_bfloat16* own = sOwn + (size_t)tb * 128 * RK;
      const float* kf = sKf + (size_t)tb * RK * S::kKLd;
#pragma unroll
      for (int kg = 0; kg < RK / 8; ++kg) {  // row m of Y_own -> A cores
        uint32_t pk[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          pk[u] = (uint32_t)__bfloat16_as_ushort(own[(kg * 8 + 2 * u) * 128 + m]) |
                  ((uint32_t)__bfloat16_as_ushort(own[(kg * 8 + 2 * u + 1) * 128 + m]) << 16);
        *reinterpret_cast<uint4*>(sAo + (m >> 3) * kSBOr + kg * 128 + (m & 7) * 16) =
            make_uint4(pk[0], pk[1], pk[2], pk[3]);
      }
      for (int e = m; e < K2 * (RK / 8); e += 128) {  // (q, k-group) of K~^{-1}(alpha rows, :)^T -> B cores
        const int q = e % K2, kg = e / K2;
        uint32_t pk[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
          pk[u] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(kf[(kg * 8 + 2 * u) * S::kKLd + q])) |
                  ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(kf[(kg * 8 + 2 * u + 1) * S::kKLd + q]))
                   << 16);
        *reinterpret_cast<uint4*>(sKb + (q >> 3) * kSBOr + kg * 128 + (q & 7) * 16) =
            make_uint4(pk[0], pk[1], pk[2], pk[3]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc::mbar_arrive(&own_empty[tb]);
      tc::mbar_arrive(zin_full);
      const int ab = it % NA;
      bool w = wait_or_abort(z_done, it & 1, abort_flag);
      if (w && it >= (uint32_t)NA) w = wait_or_abort(&a_empty[ab], ((it / NA) - 1) & 1, abort_flag);
      if (!__all_sync(0xffffffffu, w)) break;  // warp-uniform before the warp-collective TMEM loads
      tc::tc_fence_after();
      uint8_t* sAt = sA + (size_t)ab * S::kABytes;
#pragma unroll
      for (int cb = 0; cb < K2; cb += 32) {
        float v[32];
        tc::tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + kZCol + cb, v);
#pragma unroll
        for (int g8 = 0; g8 < 4; ++g8) {
          uint32_t pk[4];
#pragma unroll
          for (int u = 0; u < 4; ++u)
            pk[u] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[g8 * 8 + 2 * u])) |
                    ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v[g8 * 8 + 2 * u + 1])) << 16);
          *reinterpret_cast<uint4*>(sAt + ((cb >> 3) + g8) * 128 + (m >> 3) * kSBO + (m & 7) * 16) =
              make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
      }
      tc::tc_fence_before();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc::mbar_arrive(&a_full[ab]);
    }
  } else if (warp >= 6) {
    // ---------------------------------------------------------------- epilogue
    const int q4 = warp & 3;                 // TMEM lane quarter
    const int row = q4 * 32 + lane;          // tile row
    const bool storer = warp == 6 && lane == 0;
    uint32_t g = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
      const int64_t row0 = t * 128;
      for (int ch = 0; ch < nch; ++ch, ++g) {
        const int col0 = ch * kFuNC;
        const int nc = (anc - col0) < kFuNC ? (anc - col0) : kFuNC;
        const int a = g & 1, ob = (int)(g % kFuOut);
        const bool w = wait_or_abort(&acc_full[a], (g >> 1) & 1, abort_flag);
        // uniform over the epilogue warps; also orders the storer's read-wait
        // for this output tile before the writes below
        if (!(ok = named_bar_and(1, 128, w))) break;
        tc::tc_fence_after();
        __nv_bfloat16* ys = sY + (size_t)ob * 128 * kFuNC;
        for (int cb = 0; cb < nc; cb += 32) {
          float v[32];
          tc::tmem_ld32(tmem + ((uint32_t)(q4 * 32) << 16) + a * kFuNC + cb, v);
#pragma unroll
          for (int j = 0; j < 32; ++j) ys[(cb + j) * 128 + row] = __float2bfloat16_rn(-v[j]);
        }
        tc::tc_fence_before();
        tc::mbar_arrive(&acc_empty[a]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        named_bar_sync(1, 128);
        if (storer) {
          for (int b = 0; b < nc / kFuBox; ++b)
            tma_reduce_add_2d(&mapY, ys + b * 128 * kFuBox, (int32_t)row0, col0 + b * kFuBox);
          bulk_commit();
          bulk_wait_read1();  // the previous chunk's reduction has read the other output tile
        }
      }
    }
    if (storer) bulk_wait0();
  }
  tc::tc_fence_before();
  __syncthreads();
  if (tid == 0 && *abort_flag) set_status(st, HODLR_ERR_TIMEOUT, c, 2);
  if (warp == 5) tc::tmem_dealloc(tmem, kTmemCols);
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

size_t kf32_bytes(const hodlr_desc& d) {
  // 2^L children (the deepest level) x r x (2r + 4) FP32
  return ((size_t)1 << d.L) * (size_t)d.r * (2 * d.r + 4) * 4;
}

cudaError_t launch_update_coupled_tc(const Factor& F, int c, cudaStream_t s, bool rhs_ready) {
  const int64_t N = F.d.N;
  const int r = F.d.r;
  const int anc = r * (c - 1);
  if (anc <= 0) return cudaSuccess;
  const int64_t cpn = chunks_per_node(N, c);
  const int64_t pstride = cpn * (int64_t)r * r * c;  // node -> its first chunk's slot (reduced)
  const int64_t parents = (int64_t)1 << (c - 1);
  const double* Kc = F.K + F.Koff[c] * 4 * r * r;
  {
    ProfScope prof_(KC_COUPLING_APPLY, s);
    note_work((rhs_ready ? 0.0 : 8.0 * (double)(1ll << c) * r * anc + 2.0 * (double)parents * anc * 2 * r) +
                  8.0 * parents * 4.0 * r * r + 4.0 * (1ll << c) * r * (2.0 * r + 4),
              0.0);
    const int64_t total = parents * (int64_t)anc * (2 * r / 8);
    int64_t grid = (total + 255) / 256;
    if (grid > 16 * (int64_t)sm_count()) grid = 16 * (int64_t)sm_count();
    const int64_t kt = ((int64_t)1 << c) * r * 2 * r;
    int64_t gk = (kt + 255) / 256;
    if (gk > 16 * (int64_t)sm_count()) gk = 16 * (int64_t)sm_count();
    if (r == 32) {
      if (!rhs_ready) {  // else the projection wrote it
        rhs_bf16_kernel<32><<<(unsigned)grid, 256, 0, s>>>(c, F.P, pstride, anc, F.rhs16);
        note_launches(1);
      }
      if (!coupling_writes_kf32(F, c)) {
        kf32_kernel<32><<<(unsigned)gk, 256, 0, s>>>(c, Kc, F.kf32);
        note_launches(1);
      }
    } else {
      if (!rhs_ready) {
        rhs_bf16_kernel<64><<<(unsigned)grid, 256, 0, s>>>(c, F.P, pstride, anc, F.rhs16);
        note_launches(1);
      }
      kf32_kernel<64><<<(unsigned)gk, 256, 0, s>>>(c, Kc, F.kf32);
      note_launches(1);
    }
  }
  ProfScope prof_(KC_UPDATE_TC, s);
  note_work(2.0 * (double)N * r + 4.0 * (double)N * anc + 4.0 * (double)parents * anc * r +
                4.0 * (double)(1ll << c) * r * (2.0 * r + 4),
            4.0 * N * r * (double)anc + 4.0 * N * r * (double)r);
  CUtensorMap mY;
  __nv_bfloat16* Y = static_cast<__nv_bfloat16*>(F.Y);
  if (!make_map_plain(&mY, Y, N, (int64_t)r * F.d.L, N)) return cudaErrorInvalidValue;
  const int64_t tiles = N / 128;
  if (r == 32) {
    using S = FusedSmem<32>;
    const int per_sm = (int)((227 * 1024) / (S::kBytes + 1024));
    int64_t grid = (int64_t)sm_count() * (per_sm < 1 ? 1 : per_sm);
    if (grid > tiles) grid = tiles;
    cudaFuncSetAttribute(update_coupled_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kBytes);
    { update_coupled_tc_kernel<32><<<(unsigned)grid, kFuThreads, S::kBytes, s>>>(mY, N, c, F.rhs16, F.kf32, anc, F.status); note_launches(1); }
  } else {
    using S = FusedSmem<64>;
    const int per_sm = (int)((227 * 1024) / (S::kBytes + 1024));
    int64_t grid = (int64_t)sm_count() * (per_sm < 1 ? 1 : per_sm);
    if (grid > tiles) grid = tiles;
    cudaFuncSetAttribute(update_coupled_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kBytes);
    { update_coupled_tc_kernel<64><<<(unsigned)grid, kFuThreads, S::kBytes, s>>>(mY, N, c, F.rhs16, F.kf32, anc, F.status); note_launches(1); }
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
//   A = the leaf's Gauss-Jordan tableau T (D_b^{-1} with permuted rows and
//       columns), written by the leaf inverse in the K-major core-matrix
//       layout (8-row x 16-byte cores, LBO = 128 B along K, SBO = 4096 B
//       between 8-row groups), 64 KB per leaf, staged by one bulk copy;
//   B(c, :) = U(p_c, cols): FP64 tiles of U staged by TMA, gathered by p and
//       converted in shared memory into the 128-byte swizzled K-major layout;
//   D (TMEM, FP32) -> BF16, row r to row step(r) of a [column][row] tile,
//       stored by TMA.
// FP64 -> FP32 for the TF32 operand: the FP64 sign and exponent are rebiased
// and the top 23 significand bits kept (truncation; the MMA uses the top 10),
// on the integer pipe; magnitudes below 2^-126 become zero.
namespace {

constexpr int kLaNC = 32;       // columns of U per chunk (N of the MMA)
constexpr int kLaStages = 3;    // FP64 U tiles in flight
constexpr int kLaThreads = 320; // 4 converter warps, 4 epilogue warps, producer, MMA issuer

struct LeafTcSmem {
  static constexpr uint32_t kABytes = 128 * 128 * 4;      // D_b^{-1} tableau, K-major cores
  static constexpr uint32_t kUBytes = 128 * kLaNC * 8;    // FP64 U tile [column][row]
  static constexpr uint32_t kBBytes = kLaNC * 128 * 4;    // TF32 operand, K-major, 128-byte swizzle
  static constexpr uint32_t kYBytes = 128 * kLaNC * 2;    // BF16 Y tile [column][row]
  static constexpr uint32_t kUOff = kABytes;
  static constexpr uint32_t kBOff = kUOff + kLaStages * kUBytes;
  static constexpr uint32_t kYOff = kBOff + 2 * kBBytes;
  static constexpr uint32_t kBarOff = kYOff + 2 * kYBytes;
  static constexpr uint32_t kBytes = kBarOff + 256 + 1024;  // barriers, TMEM slot, flag; + alignment slack
  static_assert(kBOff % 1024 == 0, "swizzled operand atoms are 1024-byte aligned");
  static_assert(8 * (2 * kLaStages + 11) + 8 <= 256, "barrier area");
  static_assert(kBytes <= 227 * 1024, "shared memory per CTA");
};

// FP64 tensor map over the column-major N x cols matrix U (ld elements):
// box = 128 rows x kLaNC columns, no swizzle ([column][row] in shared memory).
bool make_map_u64(CUtensorMap* map, const double* base, int64_t rows, int64_t cols, int64_t ld) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 8};
  cuuint32_t box[2] = {128, (cuuint32_t)kLaNC};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

}  // namespace

// Persistent, warp-specialized (320 threads, one CTA per SM); every role walks
// the same sequence of (leaf, chunk) pairs:
//   warp 8, lane 0 (producer): TMA loads of the FP64 U tiles (128 rows x 32
//     columns) into a ring of kLaStages stages, running ahead across leaves;
//   warps 0-3 (converters): U tile -> B operand of the chunk (double
//     buffered): thread (warp w, lane q) forms rows 4q..4q+3 of B for columns
//     w, w + 4, ...: B(c, j) = U(p_c, j) read from the staged tile, FP64 ->
//     FP32 on the integer pipe, one 16-byte store in the 128-byte swizzled
//     K-major layout (the 8 lanes of one 128-byte row hit 8 distinct chunks);
//   warp 9, lane 0 (MMA issuer): per leaf the bulk copy of A (and an L2
//     prefetch of the CTA's next A), per chunk 16 tcgen05.mma kind::tf32 (K =
//     8 each) into one of two TMEM accumulators (M = 128, N = 32);
//   warps 4-7 (epilogue, TMEM lane quarter = warp % 4): accumulator -> BF16
//     rows scattered by step into a [column][row] tile (double buffered),
//     stored by TMA.
// Hand-offs are mbarriers; every wait is bounded and also gives up when
// another thread has raised the CTA's abort flag; copies and MMAs in flight
// are let land (bounded) before the TMEM is freed and the CTA exits.
__global__ void __launch_bounds__(kLaThreads, 1) leaf_apply_tc_kernel(const __grid_constant__ CUtensorMap mapY,
                                                                      const __grid_constant__ CUtensorMap mapU,
                                                                      int64_t nleaf, int rL,
                                                                      const float* __restrict__ Acore,
                                                                      const int* __restrict__ perm,
                                                                      DevStatus* st) {
  using S = LeafTcSmem;
  constexpr uint32_t kSBO = 4096;  // A: 32 cores along K x 128 B per 8-row group
  constexpr uint32_t kTmemCols = 2 * kLaNC;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  const double* sU = reinterpret_cast<const double*>(smem + S::kUOff);
  uint8_t* sB = smem + S::kBOff;
  __nv_bfloat16* sY = reinterpret_cast<__nv_bfloat16*>(smem + S::kYOff);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S::kBarOff);
  uint64_t* u_full = bars;                        // [stages] TMA transaction count
  uint64_t* u_empty = bars + kLaStages;           // [stages] 128 converter threads
  uint64_t* b_full = bars + 2 * kLaStages;        // [2]      128 converter threads
  uint64_t* b_empty = b_full + 2;                 // [2]      MMA commit
  uint64_t* acc_full = b_full + 4;                // [2]      MMA commit
  uint64_t* acc_empty = b_full + 6;               // [2]      128 epilogue threads
  uint64_t* a_full = b_full + 8;                  //          TMA transaction count
  uint64_t* a_empty = b_full + 9;                 //          MMA commit (the leaf's MMAs are done)
  uint64_t* drain = b_full + 10;                  //          MMA commit at exit
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(b_full + 11);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < kLaStages; ++s) {
      tc::mbar_init(&u_full[s], 1);
      tc::mbar_init(&u_empty[s], 128);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&b_full[i], 128);
      tc::mbar_init(&b_empty[i], 1);
      tc::mbar_init(&acc_full[i], 1);
      tc::mbar_init(&acc_empty[i], 128);
    }
    tc::mbar_init(a_full, 1);
    tc::mbar_init(a_empty, 1);
    tc::mbar_init(drain, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
    tc::prefetch_tmap(&mapY);
    tc::prefetch_tmap(&mapU);
  }
  if (warp == 9) tc::tmem_alloc(tmem_slot, kTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int nch = rL / kLaNC;

  if (warp == 8) {
    // ---------------------------------------------------------------- producer
    if (lane == 0) {
      uint32_t g = 0;  // chunks issued
      bool ok = true;
      for (int64_t b = blockIdx.x; b < nleaf && ok; b += gridDim.x) {
        for (int ch = 0; ch < nch; ++ch, ++g) {
          const int s = (int)(g % kLaStages);
          if (g >= (uint32_t)kLaStages &&
              !(ok = wait_or_abort(&u_empty[s], ((g / kLaStages) - 1) & 1, abort_flag)))
            break;
          tc::mbar_expect_tx(&u_full[s], S::kUBytes);
          tc::tma_load_2d(smem + S::kUOff + s * S::kUBytes, &mapU, (int32_t)(b * 128), ch * kLaNC, &u_full[s]);
        }
      }
      // let the last copies land before the CTA can exit (bounded)
      for (uint32_t q = 0; q < (uint32_t)kLaStages && q < g; ++q) {
        const uint32_t u = g - 1 - q;
        tc::mbar_wait(&u_full[u % kLaStages], (u / kLaStages) & 1);
      }
    }
  } else if (warp == 9) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_tf32_f32(128, kLaNC);
      const uint32_t a0 = tc::smem_u32(sA);
      uint32_t g = 0, i = 0;
      bool ok = true, issued = false, a_pending = false;
      for (int64_t b = blockIdx.x; b < nleaf && ok; b += gridDim.x, ++i) {
        // A of this leaf once the previous leaf's MMAs have read the buffer
        if (i >= 1 && !(ok = wait_or_abort(a_empty, (i - 1) & 1, abort_flag))) break;
        tc::mbar_expect_tx(a_full, S::kABytes);
        bulk_load_1d(sA, Acore + (size_t)b * 128 * 128, S::kABytes, a_full);
        a_pending = true;
        if (b + gridDim.x < nleaf) bulk_prefetch_l2(Acore + (size_t)(b + gridDim.x) * 128 * 128, S::kABytes);
        if (!(ok = wait_or_abort(a_full, i & 1, abort_flag))) break;
        a_pending = false;
        tc::tc_fence_after();
        for (int ch = 0; ch < nch; ++ch, ++g) {
          const uint32_t bb = g & 1;
          if (!(ok = wait_or_abort(&b_full[bb], (g >> 1) & 1, abort_flag))) break;
          if (g >= 2 && !(ok = wait_or_abort(&acc_empty[bb], ((g >> 1) - 1) & 1, abort_flag))) break;
          tc::tc_fence_after();
          const uint32_t b0 = tc::smem_u32(sB + bb * S::kBBytes);
#pragma unroll
          for (int ks = 0; ks < 16; ++ks)  // K = 8 per MMA; B: 4 swizzle atoms of 32 K, 32 bytes per MMA
            tc::mma_tf32(tmem + bb * kLaNC, tc::desc_noswz_kmajor(a0 + ks * 256, 128, kSBO),
                         tc::desc_sw128_kmajor(b0 + (ks >> 2) * 4096) + 2 * (ks & 3), idesc, ks != 0);
          issued = true;
          tc::mma_commit(&b_empty[bb]);
          tc::mma_commit(&acc_full[bb]);
        }
        if (!ok) break;
        tc::mma_commit(a_empty);
      }
      if (a_pending) tc::mbar_wait(a_full, i & 1);  // the copy into sA lands before the CTA exits
      if (issued) {                                 // every MMA issued has finished (bounded)
        tc::mma_commit(drain);
        tc::mbar_wait(drain, 0);
      }
    }
  } else if (warp < 4) {
    // ---------------------------------------------------------------- converters
    // lane q forms rows 4q..4q+3 of B: swizzle atom q / 8, 16-byte chunk q % 8
    const int at = lane >> 3, cq = lane & 7;
    uint32_t g = 0;
    bool ok = true;
    for (int64_t b = blockIdx.x; b < nleaf && ok; b += gridDim.x) {
      const int4 pq = *reinterpret_cast<const int4*>(perm + (size_t)b * 128 + 4 * lane);  // p_{4q} .. p_{4q+3}
      for (int ch = 0; ch < nch; ++ch, ++g) {
        const int s = (int)(g % kLaStages);
        const uint32_t bb = g & 1;
        if (!(ok = warp_wait(&u_full[s], (g / kLaStages) & 1, abort_flag))) break;
        if (g >= 2 && !(ok = warp_wait(&b_empty[bb], ((g >> 1) - 1) & 1, abort_flag))) break;
        const double* u = sU + (size_t)s * 128 * kLaNC;
        uint8_t* bt = sB + bb * S::kBBytes;
#pragma unroll
        for (int jj = 0; jj < kLaNC / 4; ++jj) {
          const int j = warp + 4 * jj;
          const double* uc = u + j * 128;
          *reinterpret_cast<uint4*>(bt + at * 4096 + (j >> 3) * 1024 + (j & 7) * 128 + ((cq ^ (j & 7)) << 4)) =
              make_uint4(f64_to_f32_trunc_bits(uc[pq.x]), f64_to_f32_trunc_bits(uc[pq.y]),
                         f64_to_f32_trunc_bits(uc[pq.z]), f64_to_f32_trunc_bits(uc[pq.w]));
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc::mbar_arrive(&b_full[bb]);
        tc::mbar_arrive(&u_empty[s]);
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue
    const int q4 = warp & 3;
    const int row = q4 * 32 + lane;  // row r of the leaf product = TMEM lane
    const bool storer = warp == 4 && lane == 0;
    uint32_t g = 0;
    bool ok = true;
    for (int64_t b = blockIdx.x; b < nleaf && ok; b += gridDim.x) {
      const int my_out = perm[(size_t)nleaf * 128 + (size_t)b * 128 + row];  // step(r): row of Y
      for (int ch = 0; ch < nch; ++ch, ++g) {
        const uint32_t ab = g & 1;
        const bool w = warp_wait(&acc_full[ab], (g >> 1) & 1, abort_flag);
        // uniform over the epilogue warps; also orders the storer's read-wait
        // for this Y buffer before the writes below
        if (!(ok = named_bar_and(1, 128, w))) break;
        tc::tc_fence_after();
        float v[32];
        tc::tmem_ld32(tmem + ((uint32_t)(q4 * 32) << 16) + ab * kLaNC, v);
        tc::tc_fence_before();
        tc::mbar_arrive(&acc_empty[ab]);
        __nv_bfloat16* yt = sY + (size_t)ab * 128 * kLaNC;
#pragma unroll
        for (int j = 0; j < kLaNC; ++j) yt[j * 128 + my_out] = __float2bfloat16_rn(v[j]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        named_bar_sync(1, 128);
        if (storer) {
          tma_store_2d(&mapY, yt, (int32_t)(b * 128), ch * kLaNC);
          bulk_commit();
          bulk_wait_read1();  // the previous chunk's store has read the other buffer
        }
      }
    }
    if (storer) bulk_wait0();
  }
  tc::tc_fence_before();
  __syncthreads();
  if (tid == 0 && *abort_flag) set_status(st, HODLR_ERR_TIMEOUT, 0, 3);
  if (warp == 9) tc::tmem_dealloc(tmem, kTmemCols);
}

bool leaf_apply_tc_supported(const Factor& F) {
  return g_use_tc && F.prec == HODLR_PREC_BF16 && F.d.m == 128 && (F.d.r * F.d.L) % kLaNC == 0 &&
         encode_fn() != nullptr;
}

cudaError_t launch_leaf_apply_tc(const Factor& F, const double* U, int64_t ldu, cudaStream_t s) {
  ProfScope prof_(KC_LEAF_SOLVE, s);
  const int64_t N = F.d.N;
  const int rL = F.d.r * F.d.L;
  const int64_t nleaf = (int64_t)1 << F.d.L;
  note_work(8.0 * (double)N * rL + 2.0 * (double)N * rL + 4.0 * (double)nleaf * 128 * 128,
            2.0 * (double)N * 128 * rL);
  CUtensorMap mY, mU;
  if (!make_map_plain(&mY, F.Y, N, rL, N)) return cudaErrorInvalidValue;
  if (!make_map_u64(&mU, U, N, rL, ldu)) return cudaErrorInvalidValue;
  using S = LeafTcSmem;
  int64_t grid = sm_count();  // one CTA per SM
  if (grid > nleaf) grid = nleaf;
  cudaFuncSetAttribute(leaf_apply_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::kBytes);
  {
    leaf_apply_tc_kernel<<<(unsigned)grid, kLaThreads, S::kBytes, s>>>(
        mY, mU, nleaf, rL, reinterpret_cast<const float*>(F.P), F.perm, F.status);
    note_launches(1);
  }
  return cudaGetLastError();
}

}  // namespace hodlr
