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
// Tensor-core ancestor update of the BF16 factor (Eq. e:node2):
//   Y(rows, 0:anc) -= Y(rows, own block) * W'(node),  W' FP64 r x anc (ld r).
// Tile = 128 rows of one node (M = 128), N = up to 256 ancestor columns per
// MMA, K = r. Y's own block is column-major, i.e. M-contiguous for this
// product, so the CTA's threads transpose it into the K-major canonical
// layout without swizzle (8-row x 16-byte core matrices, LBO = 128 B between
// cores along K, SBO = r/8 * 128 B between 8-row groups); W' is converted to
// BF16 into the same layout (N rows). The FP32 accumulator in TMEM is then
// subtracted from the old BF16 values, 32 columns per tcgen05.ld.
namespace {

constexpr int kUpdNC = 256;  // ancestor columns per MMA chunk

template <int RK>
struct UpdSmem {
  static constexpr uint32_t kABytes = 128 * RK * 2;
  static constexpr uint32_t kBBytes = kUpdNC * RK * 2;
  // padded so that at most two CTAs (2 x 256 TMEM columns) share an SM
  static constexpr uint32_t kBytes = (kABytes + kBBytes + 192) > 100 * 1024 ? (kABytes + kBBytes + 192) : 100 * 1024;
};

}  // namespace

template <int RK>
__global__ void __launch_bounds__(256) update_tc_kernel(int64_t N, int c, __nv_bfloat16* __restrict__ Y,
                                                        const double* __restrict__ Wbase, int64_t wstride, int anc,
                                                        DevStatus* st) {
  using S = UpdSmem<RK>;
  extern __shared__ __align__(128) uint8_t smem_raw[];
  uint8_t* sA = smem_raw;
  uint8_t* sB = smem_raw + S::kABytes;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sB + S::kBBytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr uint32_t kSBO = (RK / 8) * 128;
  constexpr uint32_t kTmemCols = kUpdNC;

  if (tid == 0) {
    tc::mbar_init(bar, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, kTmemCols);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int64_t n = N >> c;
  const int64_t tiles = N / 128;
  const int rk = RK;
  bool ok = true;
  uint32_t phase = 0;
  for (int64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
    const int64_t row0 = t * 128;
    const int64_t node = row0 / n;
    const double* W = Wbase + node * wstride;
    const __nv_bfloat16* Yown = Y + (int64_t)(c - 1) * rk * N + row0;
    // A: 128 rows x RK of the own block, K-major cores
    for (int e = tid; e < 128 * (RK / 8); e += blockDim.x) {
      const int m = e & 127, kg = e >> 7;
      uint32_t pk[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const __nv_bfloat16 lo = Yown[(int64_t)(kg * 8 + 2 * q) * N + m];
        const __nv_bfloat16 hi = Yown[(int64_t)(kg * 8 + 2 * q + 1) * N + m];
        pk[q] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
      }
      *reinterpret_cast<uint4*>(sA + kg * 128 + (m >> 3) * kSBO + (m & 7) * 16) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
    for (int col0 = 0; col0 < anc && ok; col0 += kUpdNC) {
      const int nc = (anc - col0) < kUpdNC ? (anc - col0) : kUpdNC;  // multiple of 16 (anc = r (c-1))
      // B: nc rows (ancestor columns) x RK, K-major cores, from FP64 W'
      for (int e = tid; e < nc * (RK / 8); e += blockDim.x) {
        const int nn = e % nc, kg = e / nc;
        const double* w = W + (int64_t)(col0 + nn) * rk + kg * 8;
        uint32_t pk[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const __nv_bfloat16 lo = __float2bfloat16_rn((float)w[2 * q]);
          const __nv_bfloat16 hi = __float2bfloat16_rn((float)w[2 * q + 1]);
          pk[q] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
        }
        *reinterpret_cast<uint4*>(sB + kg * 128 + (nn >> 3) * kSBO + (nn & 7) * 16) =
            make_uint4(pk[0], pk[1], pk[2], pk[3]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc::tc_fence_before();
      __syncthreads();
      tc::tc_fence_after();
      if (tid == 0) {
        const uint32_t idesc = tc::idesc_bf16_f32(128, nc);
        const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
#pragma unroll
        for (int ks = 0; ks < RK / 16; ++ks)
          tc::mma_bf16(tmem, tc::desc_noswz_kmajor(a0 + ks * 256, 128, kSBO),
                       tc::desc_noswz_kmajor(b0 + ks * 256, 128, kSBO), idesc, ks != 0);
        tc::mma_commit(bar);
      }
      ok = __syncthreads_and(tc::mbar_wait(bar, phase)) != 0;  // block-uniform before warp-collective loads
      phase ^= 1;
      tc::tc_fence_after();
      if (ok) {
        // warps w and w+4 share TMEM lanes 32 (w % 4) .. +31 and split the columns
        const int m = (warp & 3) * 32 + lane;
        __nv_bfloat16* yrow = Y + row0 + m;
        for (int cb = (warp >> 2) * 32; cb < nc; cb += 64) {
          float v[32];
          tc::tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + cb, v);
          float old[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) old[j] = __bfloat162float(yrow[(int64_t)(col0 + cb + j) * N]);
#pragma unroll
          for (int j = 0; j < 32; ++j) yrow[(int64_t)(col0 + cb + j) * N] = __float2bfloat16_rn(old[j] - v[j]);
        }
      }
      tc::tc_fence_before();
      __syncthreads();
      tc::tc_fence_after();
    }
  }
  if (!ok && tid == 0) set_status(st, HODLR_ERR_TIMEOUT, c, 1);
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

bool update_tc_supported(int64_t N, int r, int c) {
  return (r == 32 || r == 64) && ((N >> c) % 128) == 0;
}

cudaError_t launch_update_tc(int64_t N, int r, int c, __nv_bfloat16* Y, const double* Wbase, int64_t wstride,
                             DevStatus* st, cudaStream_t s) {
  ProfScope prof_(KC_UPDATE_TC, s);
  const int anc = r * (c - 1);
  if (anc <= 0) return cudaSuccess;
  note_work(2.0 * (double)N * r + 4.0 * (double)N * anc + 8.0 * (double)(1ll << c) * r * anc,
            2.0 * N * r * (double)anc);
  const int64_t tiles = N / 128;
  int64_t grid = 2 * (int64_t)sm_count();
  if (grid > tiles) grid = tiles;
  if (r == 32) {
    cudaFuncSetAttribute(update_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)UpdSmem<32>::kBytes);
    { update_tc_kernel<32><<<(unsigned)grid, 256, UpdSmem<32>::kBytes, s>>>(N, c, Y, Wbase, wstride, anc, st); note_launches(1); }
  } else {
    cudaFuncSetAttribute(update_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)UpdSmem<64>::kBytes);
    { update_tc_kernel<64><<<(unsigned)grid, 256, UpdSmem<64>::kBytes, s>>>(N, c, Y, Wbase, wstride, anc, st); note_launches(1); }
  }
  return cudaGetLastError();
}

}  // namespace hodlr
