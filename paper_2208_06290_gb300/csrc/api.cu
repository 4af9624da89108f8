// C ABI of libhodlr: argument checks, workspace layout and the host-side
// sequencing of the level-by-level factorization (Alg. 1 / Alg. 3) and solves
// (Alg. 2 / Alg. 4), the FP64 matvec and the refined solvers.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "hodlr_internal.cuh"

namespace hodlr {

cudaError_t launch_coupling_factor_apply(const Factor& F, int c, cudaStream_t s);

bool g_use_tc = true;
bool g_coupling_fp64 = false;

// ---------------------------------------------------------------- launch accounting
namespace {
std::atomic<long long> g_launches{0};
std::atomic<bool> g_prof{false};
thread_local int t_bracket = 0;
thread_local double t_bytes = 0.0, t_flops = 0.0;
struct PendingBracket {
  int cls;
  cudaEvent_t a, b;
  int n;
  double bytes, flops;
};
std::mutex g_mu;
std::vector<PendingBracket> g_pending;
std::vector<cudaEvent_t> g_pool;
double g_ms[KC_COUNT];
long long g_n[KC_COUNT];
double g_bytes[KC_COUNT], g_flops[KC_COUNT];
const char* kClassName[KC_COUNT] = {"leaf_lu", "leaf_solve", "project", "coupling", "coupling_apply",
                                    "update", "reduce_chunks", "leaf_matvec", "vector", "logdet",
                                    "project_tc", "update_tc", "matvec", "compress"};

cudaEvent_t pool_get() {
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

void note_launches(int n) {
  g_launches += n;
  t_bracket += n;
}

void note_work(double bytes, double flops) {
  t_bytes += bytes;
  t_flops += flops;
}

ProfScope::ProfScope(int c, cudaStream_t st) : cls(c), s(st), a(nullptr) {
  if (!g_prof.load(std::memory_order_relaxed)) return;
  t_bracket = 0;
  t_bytes = 0.0;
  t_flops = 0.0;
  cudaEvent_t e = pool_get();
  if (e && cudaEventRecord(e, s) == cudaSuccess) a = e;
}

ProfScope::~ProfScope() {
  if (!a) return;
  cudaEvent_t e0 = static_cast<cudaEvent_t>(a);
  if (t_bracket == 0) {
    std::lock_guard<std::mutex> g(g_mu);
    g_pool.push_back(e0);
    return;
  }
  cudaEvent_t e1 = pool_get();
  if (!e1 || cudaEventRecord(e1, s) != cudaSuccess) return;
  std::lock_guard<std::mutex> g(g_mu);
  g_pending.push_back({cls, e0, e1, t_bracket, t_bytes, t_flops});
}

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t status, ld_out, leaf_ld, node_ld, lu, perm, Y, Vp, K, P, rhs16, kf32, total;
};

size_t panel_elem_bytes(hodlr_prec p) {
  switch (p) {
    case HODLR_PREC_FP64: return 8;
    case HODLR_PREC_FP32:
    case HODLR_PREC_TF32: return 4;
    default: return 2;
  }
}

size_t max_partial_elems(const hodlr_desc& d, int ncols_per_level_factor, int k) {
  // factor: slot r x (r c) at level c; solve/matvec: slot r x k
  size_t best = 0;
  for (int c = 1; c <= d.L; ++c) {
    const size_t cols = ncols_per_level_factor ? (size_t)d.r * c : (size_t)k;
    const size_t e = (size_t)num_chunks(d.N, c) * d.r * cols;
    if (e > best) best = e;
  }
  return best;
}

// inplace (FP64 only): the leaf LUs overwrite the caller's D and Y_big its U
// (ldu = N), so neither is part of the workspace.
Layout factor_layout(const hodlr_desc& d, hodlr_prec prec, bool inplace = false) {
  Layout l{};
  const size_t nleaf = (size_t)1 << d.L;
  const size_t N = (size_t)d.N;
  const size_t rL = (size_t)d.r * d.L;
  const size_t tl = prec == HODLR_PREC_FP64 ? 8 : 4;
  const size_t tp = panel_elem_bytes(prec);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += align_up(bytes); return o; };
  l.status = take(sizeof(DevStatus));
  l.ld_out = take(2 * sizeof(double));
  l.leaf_ld = take(nleaf * 2 * sizeof(double));
  l.node_ld = take((nleaf - 1) * 2 * sizeof(double) + 16);
  l.lu = inplace ? 0 : take(nleaf * d.m * d.m * tl);
  l.perm = take(2 * N * sizeof(int));  // LU: row permutations; inverse form: p and step (see leaf_inv*.cu)
  l.Y = inplace ? 0 : take(N * rL * tp);
  l.Vp = prec == HODLR_PREC_FP64 ? 0 : take(N * rL * tp);
  l.K = take((nleaf - 1) * 4 * (size_t)d.r * d.r * sizeof(double) + 16);
  {
    // P also holds the tensor-core copy of the leaf inverses before the level loop
    const size_t pb = max_partial_elems(d, 1, 0) * sizeof(double);
    const size_t tcb = (prec == HODLR_PREC_BF16 && d.m == 128) ? nleaf * (size_t)d.m * d.m * 4 : 0;
    l.P = take(pb > tcb ? pb : tcb);
  }
  l.rhs16 = prec == HODLR_PREC_BF16 ? take(rhs_bf16_bytes(d)) : 0;
  l.kf32 = prec == HODLR_PREC_BF16 ? take(kf32_bytes(d)) : 0;
  l.total = off;
  return l;
}

hodlr_status check_desc(const hodlr_desc* d) {
  if (!d) return HODLR_ERR_ARG;
  if (d->L < 1 || d->L > 24 || d->m < 1 || d->m > 256 || d->r < 1 || d->r > 64 || d->r > d->m) return HODLR_ERR_ARG;
  if (d->reserved != 0) return HODLR_ERR_ARG;
  if (d->N != ((int64_t)d->m << d->L)) return HODLR_ERR_ARG;
  if (d->ldu < d->N || d->ldv < d->N) return HODLR_ERR_ARG;
  return HODLR_OK;
}

bool prec_ok(hodlr_prec p) {
  return p == HODLR_PREC_FP64 || p == HODLR_PREC_FP32 || p == HODLR_PREC_TF32 || p == HODLR_PREC_BF16;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

#define HODLR_CUDA(...)                            \
  do {                                             \
    cudaError_t e_ = (__VA_ARGS__);                \
    if (e_ != cudaSuccess) return HODLR_ERR_CUDA;  \
  } while (0)

template <typename TP>
hodlr_status factor_levels(Factor& F, cudaStream_t s) {
  const hodlr_desc& d = F.d;
  TP* Y = static_cast<TP*>(F.Y);
  const TP* Vp = static_cast<const TP*>(F.Vp);
  for (int c = d.L; c >= 1; --c) {
    const int rc = d.r * c;
    const int anc = d.r * (c - 1);
    // levels where every node is one row chunk and the fused tensor-core update
    // follows: the projection writes the ancestor columns straight into the
    // update's BF16 right-hand-side operand
    bool rhs_ready = false;
    if constexpr (std::is_same<TP, __nv_bfloat16>::value) {
      rhs_ready = g_use_tc && anc > 0 && project_tc_supported(d.N, d.r, c) && update_tc_supported(d.N, d.r, c) &&
                  chunks_per_node(d.N, c) == 1;
      if (g_use_tc && project_tc_supported(d.N, d.r, c))
        HODLR_CUDA(launch_project_tc(d.N, d.r, d.L, c, Vp, F.ldvp, Y, F.P, F.status, s,
                                     rhs_ready ? F.rhs16 : nullptr));
      else
        HODLR_CUDA(launch_project<TP, TP>(d.N, d.r, c, Vp, F.ldvp, c - 1, Y, d.N, rc, F.P, 0, s));
    } else if constexpr (std::is_same<TP, float>::value) {
      if (F.prec == HODLR_PREC_TF32 && g_use_tc && project_tc_supported(d.N, d.r, c))
        HODLR_CUDA(launch_project_tc32(d.N, d.r, d.L, c, Vp, F.ldvp, Y, F.P, F.status, s));
      else
        HODLR_CUDA(launch_project<TP, TP>(d.N, d.r, c, Vp, F.ldvp, c - 1, Y, d.N, rc, F.P, 0, s));
    } else {
      HODLR_CUDA(launch_project<TP, TP>(d.N, d.r, c, Vp, F.ldvp, c - 1, Y, d.N, rc, F.P, 0, s));
    }
    F.P_reduced = chunks_per_node(d.N, c) > 1;
    if (F.P_reduced) HODLR_CUDA(launch_reduce_chunks(d.N, d.r, c, F.P, rc, s));
    HODLR_CUDA(launch_coupling_factor(F, c, s));
    if (anc > 0) {
      const int64_t wstride = chunks_per_node(d.N, c) * (int64_t)d.r * rc;
      bool done = false;
      if constexpr (std::is_same<TP, __nv_bfloat16>::value) {
        if (g_use_tc && update_tc_supported(d.N, d.r, c)) {
          // W' = K~^{-1} [W_beta; W_alpha] applied inside the update
          HODLR_CUDA(launch_update_coupled_tc(F, c, s, rhs_ready));
          done = true;
        }
      }
      if (!done) {
        HODLR_CUDA(launch_coupling_factor_apply(F, c, s));
        HODLR_CUDA(launch_update<TP, TP>(d.N, d.r, c, Y, d.N, c - 1, Y, d.N, anc, F.P, wstride, 0, -1.0, 0, s));
      }
    }
    F.P_reduced = false;
  }
  return HODLR_OK;
}

size_t solve_partials_bytes(const hodlr_desc& d, int k) {
  return align_up(max_partial_elems(d, 0, k) * sizeof(double));
}

// In-place solve on x (N x k, ld ldx) in type TX with the factor's panels TP.
template <typename TP, typename TX>
hodlr_status solve_core(const Factor& F, TX* x, int64_t ldx, int k, double* Ps, int trans, cudaStream_t s,
                        double* parts = nullptr) {
  const hodlr_desc& d = F.d;
  const TP* Y = static_cast<const TP*>(F.Y);
  const TP* Vp = static_cast<const TP*>(F.Vp);
  if (!trans) {
    HODLR_CUDA((launch_leaf_solve<TX, TX>(F, x, ldx, x, ldx, k, 0, s)));
    if constexpr (std::is_same<TX, float>::value && !std::is_same<TP, double>::value) {
      // one column: two launches per level (projection parts in `parts`, W in Ps)
      if (k == 1 && parts && solve_k1_supported<TP>(F, Y, Vp, F.ldvp, x)) {
        HODLR_CUDA(launch_solve_k1_chain<TP>(F, Y, Vp, F.ldvp, x, parts, reinterpret_cast<float*>(Ps), s));
        return HODLR_OK;
      }
    }
    for (int c = d.L; c >= 1; --c) {
      HODLR_CUDA((launch_project<TP, TX>(d.N, d.r, c, Vp, F.ldvp, c - 1, x, ldx, k, Ps, 0, s)));
      const bool red = chunks_per_node(d.N, c) >= 8;  // many partials per node: sum them in parallel first
      if (red) HODLR_CUDA(launch_reduce_chunks(d.N, d.r, c, Ps, k, s));
      HODLR_CUDA(launch_coupling_solve(F, c, Ps, k, 0, s, red));
      const int64_t wstride = chunks_per_node(d.N, c) * (int64_t)d.r * k;
      HODLR_CUDA((launch_update<TP, TX>(d.N, d.r, c, Y, d.N, c - 1, x, ldx, k, Ps, wstride, 0, -1.0, 0, s)));
    }
  } else {
    for (int c = 1; c <= d.L; ++c) {
      HODLR_CUDA((launch_project<TP, TX>(d.N, d.r, c, Y, d.N, c - 1, x, ldx, k, Ps, 0, s)));
      const bool red = chunks_per_node(d.N, c) >= 8;
      if (red) HODLR_CUDA(launch_reduce_chunks(d.N, d.r, c, Ps, k, s));
      HODLR_CUDA(launch_coupling_solve(F, c, Ps, k, 1, s, red));
      const int64_t wstride = chunks_per_node(d.N, c) * (int64_t)d.r * k;
      HODLR_CUDA((launch_update<TP, TX>(d.N, d.r, c, Vp, F.ldvp, c - 1, x, ldx, k, Ps, wstride, 1, -1.0, 0, s)));
    }
    HODLR_CUDA((launch_leaf_solve<TX, TX>(F, x, ldx, x, ldx, k, 1, s)));
  }
  return HODLR_OK;
}

hodlr_status solve_any(const Factor& F, double* B, int64_t ldb, int k, void* work, int trans, cudaStream_t s) {
  const hodlr_desc& d = F.d;
  double* Ps = static_cast<double*>(work);
  if (F.prec == HODLR_PREC_FP64) return solve_core<double, double>(F, B, ldb, k, Ps, trans, s);
  float* xw = reinterpret_cast<float*>(static_cast<char*>(work) + solve_partials_bytes(d, k));
  double* parts = k == 1 ? reinterpret_cast<double*>(static_cast<char*>(work) + solve_partials_bytes(d, k) +
                                                    align_up((size_t)d.N * k * sizeof(float)))
                        : nullptr;
  HODLR_CUDA((launch_copy_cols<float, double>(d.N, k, B, ldb, xw, d.N, s)));
  hodlr_status st = F.prec != HODLR_PREC_BF16  // FP32 panels (FP32 and TF32 factors)
                        ? solve_core<float, float>(F, xw, d.N, k, Ps, trans, s, parts)
                        : solve_core<__nv_bfloat16, float>(F, xw, d.N, k, Ps, trans, s, parts);
  if (st != HODLR_OK) return st;
  HODLR_CUDA((launch_copy_cols<double, float>(d.N, k, xw, d.N, B, ldb, s)));
  return HODLR_OK;
}

size_t solve_ws_bytes(const Factor& F, int k) {
  size_t b = solve_partials_bytes(F.d, k);
  if (F.prec != HODLR_PREC_FP64) b += align_up((size_t)F.d.N * k * sizeof(float));
  // one right-hand side, low precision: the parts of the projections
  if (F.prec != HODLR_PREC_FP64 && k == 1) b += align_up(solve_k1_parts_elems(F.d) * sizeof(double));
  return b;
}

// Minimum matvec scratch (per-level partials); with k = 1 a workspace of
// matvec_ws_bytes also enables the four-launch path of matvec1.cu.
size_t matvec_min_bytes(const hodlr_desc& d, int k) { return solve_partials_bytes(d, k); }
size_t matvec_fast_bytes(const hodlr_desc& d) { return align_up(matvec1_scratch_elems(d) * sizeof(double)); }
size_t matvec_ws_bytes(const hodlr_desc& d, int k) {
  const size_t a = matvec_min_bytes(d, k);
  return k == 1 ? std::max(a, matvec_fast_bytes(d)) : a;
}

hodlr_status matvec_core(const hodlr_desc& d, const double* D, const double* U, const double* V, const double* X,
                         int64_t ldx, double* Y, int64_t ldy, int k, void* work, cudaStream_t s,
                         size_t work_bytes = 0) {
  double* Ps = static_cast<double*>(work);
  if (k == 1 && work_bytes >= matvec_fast_bytes(d)) {
    HODLR_CUDA(launch_matvec1(d, D, U, V, X, Y, Ps, s));
    return HODLR_OK;
  }
  HODLR_CUDA(launch_leaf_matvec(d, D, X, ldx, Y, ldy, k, s));
  for (int c = 1; c <= d.L; ++c) {
    HODLR_CUDA((launch_project<double, double>(d.N, d.r, c, V, d.ldv, c - 1, X, ldx, k, Ps, 1, s)));
    HODLR_CUDA(launch_reduce_chunks(d.N, d.r, c, Ps, k, s));
    const int64_t wstride = chunks_per_node(d.N, c) * (int64_t)d.r * k;
    HODLR_CUDA((launch_update<double, double>(d.N, d.r, c, U, d.ldu, c - 1, Y, ldy, k, Ps, wstride, 1, 1.0, 1, s)));
  }
  return HODLR_OK;
}

bool valid_factor(const Factor* F) { return F != nullptr; }

}  // namespace

size_t factor_workspace_bytes(const hodlr_desc& d, hodlr_prec prec) { return factor_layout(d, prec).total; }

// Entry points for the allocation-free matvec (noalloc.cu).
hodlr_status matvec_core_ext(const hodlr_desc& d, const double* D, const double* U, const double* V, const double* X,
                             int64_t ldx, double* Y, int64_t ldy, int k, void* work, cudaStream_t s,
                             size_t work_bytes) {
  return matvec_core(d, D, U, V, X, ldx, Y, ldy, k, work, s, work_bytes);
}
size_t matvec_scratch_bytes(const hodlr_desc& d, int k) { return matvec_min_bytes(d, k); }
hodlr_status check_desc_ext(const hodlr_desc* d) { return check_desc(d); }

}  // namespace hodlr

using namespace hodlr;

struct hodlr_factor_s : public hodlr::Factor {};

extern "C" {

const char* hodlr_strerror(hodlr_status s) {
  switch (s) {
    case HODLR_OK: return "ok";
    case HODLR_ERR_ARG: return "invalid argument";
    case HODLR_ERR_WORKSPACE: return "workspace too small or misaligned";
    case HODLR_ERR_CUDA: return "CUDA runtime error";
    case HODLR_ERR_SINGULAR_LEAF: return "singular leaf block";
    case HODLR_ERR_SINGULAR_COUPLING: return "singular coupling matrix";
    case HODLR_ERR_NONFINITE: return "non-finite input";
    case HODLR_ERR_NOT_CONVERGED: return "iteration did not converge";
    case HODLR_ERR_TIMEOUT: return "device-side wait timed out";
    case HODLR_ERR_SCRATCH_LIMIT: return "problem exceeds the fixed scratch of the allocation-free entry point";
  }
  return "unknown status";
}

hodlr_status hodlr_factor_workspace_size(const hodlr_desc* desc, hodlr_prec prec, size_t* bytes) {
  hodlr_status st = check_desc(desc);
  if (st != HODLR_OK) return st;
  if (!prec_ok(prec) || !bytes) return HODLR_ERR_ARG;
  *bytes = factor_layout(*desc, prec).total;
  return HODLR_OK;
}

static hodlr_status factor_entry(const hodlr_desc* desc, const double* D, const double* U, const double* V,
                                 hodlr_prec prec, bool inplace, void* workspace, size_t workspace_bytes,
                                 hodlr_stream_t stream, hodlr_factor_t* out) {
  hodlr_status st = check_desc(desc);
  if (st != HODLR_OK) return st;
  if (!prec_ok(prec) || !D || !U || !V || !out) return HODLR_ERR_ARG;
  if (!aligned(D, 8) || !aligned(U, 8) || !aligned(V, 8)) return HODLR_ERR_ARG;
  if (inplace && (prec != HODLR_PREC_FP64 || desc->ldu != desc->N || U == V)) return HODLR_ERR_ARG;
  const Layout lay = factor_layout(*desc, prec, inplace);
  if (!workspace || !aligned(workspace, kAlign) || workspace_bytes < lay.total) return HODLR_ERR_WORKSPACE;
  hodlr_factor_s* F = new (std::nothrow) hodlr_factor_s();
  if (!F) return HODLR_ERR_ARG;
  char* w = static_cast<char*>(workspace);
  const hodlr_desc& d = *desc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  F->d = d;
  F->prec = prec;
  F->stream = s;
  F->status = reinterpret_cast<DevStatus*>(w + lay.status);
  F->ld_out = reinterpret_cast<double*>(w + lay.ld_out);
  F->leaf_ld = reinterpret_cast<double*>(w + lay.leaf_ld);
  F->node_ld = reinterpret_cast<double*>(w + lay.node_ld);
  F->lu = inplace ? static_cast<void*>(const_cast<double*>(D)) : static_cast<void*>(w + lay.lu);
  F->perm = reinterpret_cast<int*>(w + lay.perm);
  F->Y = inplace ? static_cast<void*>(const_cast<double*>(U)) : static_cast<void*>(w + lay.Y);
  F->K = reinterpret_cast<double*>(w + lay.K);
  F->P = reinterpret_cast<double*>(w + lay.P);
  F->P_elems = max_partial_elems(d, 1, 0);
  F->rhs16 = prec == HODLR_PREC_BF16 ? reinterpret_cast<uint8_t*>(w + lay.rhs16) : nullptr;
  F->kf32 = prec == HODLR_PREC_BF16 ? reinterpret_cast<float*>(w + lay.kf32) : nullptr;
  for (int c = 0; c < 26; ++c) F->Koff[c] = 0;
  for (int c = 1; c <= d.L; ++c) F->Koff[c] = ((int64_t)1 << (c - 1)) - 1;
  if (prec == HODLR_PREC_FP64) {
    F->Vp = V;
    F->ldvp = d.ldv;
  } else {
    F->Vp = w + lay.Vp;
    F->ldvp = d.N;
  }
  auto fail = [&](hodlr_status e) { delete F; return e; };
  if (cudaMemsetAsync(F->status, 0, sizeof(DevStatus), s) != cudaSuccess) return fail(HODLR_ERR_CUDA);
  F->leaf_tc = leaf_apply_tc_supported(*F) && aligned(U, 16) && d.ldu % 2 == 0;
  const int rL = d.r * d.L;
  if (launch_leaf_lu(*F, D, s) != cudaSuccess) return fail(HODLR_ERR_CUDA);
  hodlr_status r = HODLR_OK;
  if (prec == HODLR_PREC_FP64) {
    if (launch_leaf_solve<double, double>(*F, U, d.ldu, static_cast<double*>(F->Y), d.N, rL, 0, s) != cudaSuccess)
      return fail(HODLR_ERR_CUDA);
    r = factor_levels<double>(*F, s);
  } else if (prec == HODLR_PREC_FP32 || prec == HODLR_PREC_TF32) {
    if (launch_copy_cols<float, double>(d.N, rL, V, d.ldv, static_cast<float*>(const_cast<void*>(F->Vp)), d.N, s) !=
        cudaSuccess)
      return fail(HODLR_ERR_CUDA);
    if (launch_leaf_solve<double, float>(*F, U, d.ldu, static_cast<float*>(F->Y), d.N, rL, 0, s) != cudaSuccess)
      return fail(HODLR_ERR_CUDA);
    r = factor_levels<float>(*F, s);
  } else {
    if (launch_copy_cols<__nv_bfloat16, double>(d.N, rL, V, d.ldv,
                                                static_cast<__nv_bfloat16*>(const_cast<void*>(F->Vp)), d.N,
                                                s) != cudaSuccess)
      return fail(HODLR_ERR_CUDA);
    const cudaError_t e =
        F->leaf_tc ? launch_leaf_apply_tc(*F, U, d.ldu, s)
                   : launch_leaf_solve<double, __nv_bfloat16>(*F, U, d.ldu, static_cast<__nv_bfloat16*>(F->Y), d.N,
                                                              rL, 0, s);
    if (e != cudaSuccess) return fail(HODLR_ERR_CUDA);
    r = factor_levels<__nv_bfloat16>(*F, s);
  }
  if (r != HODLR_OK) return fail(r);
  *out = F;
  return HODLR_OK;
}

hodlr_status hodlr_factor(const hodlr_desc* desc, const double* D, const double* U, const double* V,
                          hodlr_prec prec, void* workspace, size_t workspace_bytes, hodlr_stream_t stream,
                          hodlr_factor_t* out) {
  return factor_entry(desc, D, U, V, prec, false, workspace, workspace_bytes, stream, out);
}

hodlr_status hodlr_factor_inplace_workspace_size(const hodlr_desc* desc, size_t* bytes) {
  hodlr_status st = check_desc(desc);
  if (st != HODLR_OK) return st;
  if (!bytes || desc->ldu != desc->N) return HODLR_ERR_ARG;
  *bytes = factor_layout(*desc, HODLR_PREC_FP64, true).total;
  return HODLR_OK;
}

hodlr_status hodlr_factor_inplace(const hodlr_desc* desc, double* D, double* U, const double* V, void* workspace,
                                  size_t workspace_bytes, hodlr_stream_t stream, hodlr_factor_t* out) {
  return factor_entry(desc, D, U, V, HODLR_PREC_FP64, true, workspace, workspace_bytes, stream, out);
}

hodlr_status hodlr_factor_status(hodlr_factor_t f, int64_t* where, int64_t* detail) {
  if (!valid_factor(f)) return HODLR_ERR_ARG;
  DevStatus h{};
  if (cudaStreamSynchronize(f->stream) != cudaSuccess) return HODLR_ERR_CUDA;
  if (cudaMemcpy(&h, f->status, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return HODLR_ERR_CUDA;
  if (where) *where = h.where;
  if (detail) *detail = h.detail;
  return static_cast<hodlr_status>(h.code);
}

void hodlr_free(hodlr_factor_t f) { delete f; }

hodlr_status hodlr_solve_workspace_size(hodlr_factor_t f, int32_t k, size_t* bytes) {
  if (!valid_factor(f) || k < 1 || !bytes) return HODLR_ERR_ARG;
  *bytes = solve_ws_bytes(*f, k);
  return HODLR_OK;
}

static hodlr_status solve_entry(hodlr_factor_t f, double* B, int64_t ldb, int32_t k, void* work, size_t bytes,
                                hodlr_stream_t stream, int trans) {
  if (!valid_factor(f) || !B || k < 1 || ldb < f->d.N || !aligned(B, 8)) return HODLR_ERR_ARG;
  if (!work || !aligned(work, kAlign) || bytes < solve_ws_bytes(*f, k)) return HODLR_ERR_WORKSPACE;
  return solve_any(*f, B, ldb, k, work, trans, reinterpret_cast<cudaStream_t>(stream));
}

hodlr_status hodlr_solve(hodlr_factor_t f, double* B, int64_t ldb, int32_t k, void* workspace,
                         size_t workspace_bytes, hodlr_stream_t stream) {
  return solve_entry(f, B, ldb, k, workspace, workspace_bytes, stream, 0);
}

hodlr_status hodlr_solve_adjoint(hodlr_factor_t f, double* B, int64_t ldb, int32_t k, void* workspace,
                                 size_t workspace_bytes, hodlr_stream_t stream) {
  return solve_entry(f, B, ldb, k, workspace, workspace_bytes, stream, 1);
}

hodlr_status hodlr_logdet(hodlr_factor_t f, hodlr_stream_t stream, double* sign, double* logabsdet) {
  if (!valid_factor(f) || !sign || !logabsdet) return HODLR_ERR_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (launch_logdet_reduce(*f, s) != cudaSuccess) return HODLR_ERR_CUDA;
  double h[2];
  if (cudaMemcpyAsync(h, f->ld_out, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return HODLR_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return HODLR_ERR_CUDA;
  *sign = h[0];
  *logabsdet = h[1];
  DevStatus st{};
  if (cudaMemcpy(&st, f->status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return HODLR_ERR_CUDA;
  return static_cast<hodlr_status>(st.code);
}

hodlr_status hodlr_matvec_workspace_size(const hodlr_desc* desc, int32_t k, size_t* bytes) {
  hodlr_status st = check_desc(desc);
  if (st != HODLR_OK) return st;
  if (k < 1 || !bytes) return HODLR_ERR_ARG;
  *bytes = matvec_ws_bytes(*desc, k);
  return HODLR_OK;
}

hodlr_status hodlr_matvec(const hodlr_desc* desc, const double* D, const double* U, const double* V,
                          const double* X, int64_t ldx, double* Y, int64_t ldy, int32_t k, void* workspace,
                          size_t workspace_bytes, hodlr_stream_t stream) {
  hodlr_status st = check_desc(desc);
  if (st != HODLR_OK) return st;
  if (!D || !U || !V || !X || !Y || k < 1 || ldx < desc->N || ldy < desc->N) return HODLR_ERR_ARG;
  if (X == Y) return HODLR_ERR_ARG;
  if (!workspace || !aligned(workspace, kAlign) || workspace_bytes < matvec_min_bytes(*desc, k))
    return HODLR_ERR_WORKSPACE;
  return matvec_core(*desc, D, U, V, X, ldx, Y, ldy, k, workspace, reinterpret_cast<cudaStream_t>(stream),
                     workspace_bytes);
}

// ------------------------------------------------------------ refined solvers
namespace {

// Workspace of the refined solvers. FGMRES (restart > 0) keeps, for the k
// right-hand sides in lockstep, the Arnoldi basis V (restart + 1 vectors per
// column), the preconditioned vectors Z and their FP64 products W = A Z
// (restart each), stored so that the q-th vectors of all columns form one
// N x k block (column q * k + j, ld N).
struct RefineLayout {
  size_t R, solve, mv, dots, scal, V, Z, W, w, Xb, total;
};

RefineLayout refine_layout(const Factor& F, int k, int restart) {
  RefineLayout l{};
  const size_t N = (size_t)F.d.N;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += align_up(bytes); return o; };
  const size_t kk = (size_t)k;
  const size_t m = (size_t)restart;
  l.R = take(N * kk * sizeof(double));
  l.solve = take(solve_ws_bytes(F, k));
  l.mv = take(matvec_ws_bytes(F.d, k));
  l.dots = take(dot_scratch_elems(F.d.N, (int)((m + 1) * kk)) * sizeof(double));
  l.scal = take(((2 * (m + 1) + 3 + m) * kk + 8) * sizeof(double));
  if (restart > 0) {
    l.V = take(N * (m + 1) * kk * sizeof(double));
    l.Z = take(N * m * kk * sizeof(double));
    l.W = take(N * m * kk * sizeof(double));
    l.w = take(N * kk * sizeof(double));
    l.Xb = take(N * kk * sizeof(double));  // refinement's best iterate, FGMRES's starting point
  }
  l.total = off;
  return l;
}

hodlr_status col_norms2(int64_t N, int k, const double* x, int64_t ldx, double* dev_out, double* scratch,
                        double* host_out, cudaStream_t s) {
  HODLR_CUDA(launch_dots(N, k, x, ldx, x, ldx, dev_out, scratch, s));
  HODLR_CUDA(cudaMemcpyAsync(host_out, dev_out, (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, s));
  HODLR_CUDA(cudaStreamSynchronize(s));
  return HODLR_OK;
}

// Flexible GMRES(restart), right-preconditioned by the factor, on k columns in
// lockstep: every inner iteration applies the preconditioner to the k new
// basis vectors in one k-column solve and the FP64 operator in one k-column
// matvec; classical Gram-Schmidt twice, per column, with batched dot products;
// one host synchronization per iteration reads the k columns' Hessenberg
// entries (Givens rotations on the host). A column whose residual estimate
// reaches 0.5 tol stops extending its basis (its later vectors are computed
// but never used). After each cycle x += Z y and r -= (A Z) y from the stored
// FP64 products (no further matvec); a column that has converged takes y = 0.
// X holds the initial guess on entry (start_from_x) or is set to f^{-1} B.
hodlr_status gmres_core(const Factor& F, const double* D, const double* U, const double* V, const double* B,
                        int64_t ldb, double* X, int64_t ldx, int k, double tol, int restart, int max_iter,
                        bool start_from_x, char* w, const RefineLayout& lay, cudaStream_t s, int* iters_out,
                        double* relres_out) {
  const hodlr_desc& d = F.d;
  const int64_t N = d.N;
  const int m = restart;
  double* R = reinterpret_cast<double*>(w + lay.R);
  void* sw = w + lay.solve;
  void* mw = w + lay.mv;
  double* scratch = reinterpret_cast<double*>(w + lay.dots);
  double* scal = reinterpret_cast<double*>(w + lay.scal);
  double* dev_h1 = scal;                          // (m + 1) k
  double* dev_h2 = dev_h1 + (size_t)(m + 1) * k;  // (m + 1) k
  double* dev_hn = dev_h2 + (size_t)(m + 1) * k;  // k
  double* dev_nr = dev_hn + k;                    // k
  double* dev_nb = dev_nr + k;                    // k
  double* dev_coef = dev_nb + k;                  // m k
  double* Vb = reinterpret_cast<double*>(w + lay.V);
  double* Zb = reinterpret_cast<double*>(w + lay.Z);
  double* Wb = reinterpret_cast<double*>(w + lay.W);
  double* wv = reinterpret_cast<double*>(w + lay.w);
  hodlr_status st;
  if (!start_from_x) {
    HODLR_CUDA(launch_copy_cols<double, double>(N, k, B, ldb, X, ldx, s));
    if ((st = solve_any(F, X, ldx, k, sw, 0, s)) != HODLR_OK) return st;
  }
  std::vector<double> nb(k), nr(k), hh((size_t)(2 * (m + 1) + 1) * k), coef((size_t)m * k);
  std::vector<double> H((size_t)k * (m + 1) * m), g((size_t)k * (m + 1)), cs((size_t)k * m), sn((size_t)k * m),
      y(m);
  std::vector<int> nsteps(k), done(k);
  // |A z_i| per column and inner step (the raw Hessenberg column's norm), and
  // a running bound on |r (recursive) - (b - A x)| / |b| from the rounding of
  // x += Z y and r -= (A Z) y (about eps sum_i |y_i| |A z_i| per cycle)
  std::vector<double> hnorm((size_t)k * m), drift(k, 0.0);
  if ((st = col_norms2(N, k, B, ldb, dev_nb, scratch, nb.data(), s)) != HODLR_OK) return st;
  for (int j = 0; j < k; ++j) nb[j] = std::sqrt(nb[j]) > 0.0 ? std::sqrt(nb[j]) : 1.0;
  // r = B - A X (FP64 matvec) once; later cycles update it from W
  if ((st = matvec_core(d, D, U, V, X, ldx, R, N, k, mw, s, matvec_ws_bytes(d, k))) != HODLR_OK) return st;
  HODLR_CUDA(launch_axpby_cols(N, k, 1.0, B, ldb, -1.0, R, N, s));
  int total_it = 0;
  double worst = INFINITY;
  for (;;) {
    if ((st = col_norms2(N, k, R, N, dev_nr, scratch, nr.data(), s)) != HODLR_OK) return st;
    // a column that looks converged while its drift bound could hide tol is
    // checked against the true residual: r = b - A x (one FP64 matvec for all
    // columns), which also restarts every column from its true residual
    bool verify = false;
    for (int j = 0; j < k; ++j)
      verify |= std::sqrt(nr[j]) / nb[j] <= tol && drift[j] > 0.01 * tol;
    if (verify) {
      if ((st = matvec_core(d, D, U, V, X, ldx, R, N, k, mw, s, matvec_ws_bytes(d, k))) != HODLR_OK) return st;
      HODLR_CUDA(launch_axpby_cols(N, k, 1.0, B, ldb, -1.0, R, N, s));
      if ((st = col_norms2(N, k, R, N, dev_nr, scratch, nr.data(), s)) != HODLR_OK) return st;
      std::fill(drift.begin(), drift.end(), 0.0);
    }
    worst = 0.0;
    bool any = false;
    for (int j = 0; j < k; ++j) {
      const double rel = std::sqrt(nr[j]) / nb[j];
      worst = std::isnan(rel) ? INFINITY : std::max(worst, rel);
      done[j] = rel > tol ? 0 : 1;
      any |= !done[j];
      nsteps[j] = 0;
      std::fill(g.begin() + (size_t)j * (m + 1), g.begin() + (size_t)(j + 1) * (m + 1), 0.0);
      g[(size_t)j * (m + 1)] = std::sqrt(nr[j]);
    }
    if (!any || total_it >= max_iter) break;
    HODLR_CUDA(launch_scale_inv_norm(N, k, R, dev_nr, Vb, s));  // v_0 = r / |r|
    int nq = 0;
    for (int i = 0; i < m && total_it < max_iter; ++i) {
      double* Vi = Vb + (size_t)i * k * N;
      double* Zi = Zb + (size_t)i * k * N;
      double* Wi = Wb + (size_t)i * k * N;
      HODLR_CUDA(launch_copy_cols<double, double>(N, k, Vi, N, Zi, N, s));
      if ((st = solve_any(F, Zi, N, k, sw, 0, s)) != HODLR_OK) return st;  // z = M^{-1} v
      if ((st = matvec_core(d, D, U, V, Zi, N, Wi, N, k, mw, s, matvec_ws_bytes(d, k))) != HODLR_OK) return st;
      HODLR_CUDA(launch_copy_cols<double, double>(N, k, Wi, N, wv, N, s));
      // classical Gram-Schmidt, twice
      HODLR_CUDA(launch_bdots(N, k, i + 1, Vb, wv, dev_h1, scratch, s));
      HODLR_CUDA(launch_bgemv(N, k, i + 1, Vb, dev_h1, -1.0, wv, N, s));
      HODLR_CUDA(launch_bdots(N, k, i + 1, Vb, wv, dev_h2, scratch, s));
      HODLR_CUDA(launch_bgemv(N, k, i + 1, Vb, dev_h2, -1.0, wv, N, s));
      HODLR_CUDA(launch_dots(N, k, wv, N, wv, N, dev_hn, scratch, s));
      HODLR_CUDA(launch_scale_inv_norm(N, k, wv, dev_hn, Vb + (size_t)(i + 1) * k * N, s));
      HODLR_CUDA(cudaMemcpyAsync(hh.data(), dev_h1, hh.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
      HODLR_CUDA(cudaStreamSynchronize(s));
      ++total_it;
      nq = i + 1;
      bool all = true;
      for (int j = 0; j < k; ++j) {
        if (done[j]) continue;
        double* Hi = H.data() + ((size_t)j * m + i) * (m + 1);
        double* gj = g.data() + (size_t)j * (m + 1);
        double* csj = cs.data() + (size_t)j * m;
        double* snj = sn.data() + (size_t)j * m;
        double hn2 = 0.0;
        for (int q = 0; q <= i; ++q) {
          Hi[q] = hh[(size_t)q * k + j] + hh[(size_t)(m + 1) * k + (size_t)q * k + j];
          hn2 += Hi[q] * Hi[q];
        }
        Hi[i + 1] = std::sqrt(hh[(size_t)2 * (m + 1) * k + j]);
        hnorm[(size_t)j * m + i] = std::sqrt(hn2 + Hi[i + 1] * Hi[i + 1]);
        for (int q = 0; q < i; ++q) {  // earlier Givens rotations on column i
          const double t = csj[q] * Hi[q] + snj[q] * Hi[q + 1];
          Hi[q + 1] = -snj[q] * Hi[q] + csj[q] * Hi[q + 1];
          Hi[q] = t;
        }
        const double den = std::hypot(Hi[i], Hi[i + 1]);
        csj[i] = den > 0.0 ? Hi[i] / den : 1.0;
        snj[i] = den > 0.0 ? Hi[i + 1] / den : 0.0;
        Hi[i] = den;
        Hi[i + 1] = 0.0;
        gj[i + 1] = -snj[i] * gj[i];
        gj[i] = csj[i] * gj[i];
        nsteps[j] = i + 1;
        if (std::fabs(gj[i + 1]) / nb[j] <= 0.5 * tol) done[j] = 1;
        all &= done[j] != 0;
      }
      if (all) break;
    }
    // y = H(0:n, 0:n)^{-1} g(0:n) per column; x += Z y, r -= (A Z) y
    std::fill(coef.begin(), coef.end(), 0.0);
    for (int j = 0; j < k; ++j) {
      const int ns = nsteps[j];
      const double* Hj = H.data() + (size_t)j * m * (m + 1);
      const double* gj = g.data() + (size_t)j * (m + 1);
      for (int q = ns - 1; q >= 0; --q) {
        double acc = gj[q];
        for (int p = q + 1; p < ns; ++p) acc -= Hj[(size_t)p * (m + 1) + q] * y[p];
        const double hq = Hj[(size_t)q * (m + 1) + q];
        y[q] = hq != 0.0 ? acc / hq : 0.0;
      }
      double dr = 0.0;
      for (int q = 0; q < ns; ++q) {
        coef[(size_t)q * k + j] = y[q];
        dr += std::fabs(y[q]) * hnorm[(size_t)j * m + q];
      }
      drift[j] += 4.0 * 1.1102230246251565e-16 * dr / nb[j];
    }
    HODLR_CUDA(cudaMemcpyAsync(dev_coef, coef.data(), (size_t)nq * k * sizeof(double), cudaMemcpyHostToDevice, s));
    HODLR_CUDA(launch_bgemv(N, k, nq, Zb, dev_coef, 1.0, X, ldx, s));
    HODLR_CUDA(launch_bgemv(N, k, nq, Wb, dev_coef, -1.0, R, N, s));
  }
  if (iters_out) *iters_out = total_it;
  if (relres_out) *relres_out = worst;
  return worst <= tol ? HODLR_OK : HODLR_ERR_NOT_CONVERGED;
}

hodlr_status device_status(const Factor& F) {
  DevStatus ds{};
  if (cudaMemcpy(&ds, F.status, sizeof(ds), cudaMemcpyDeviceToHost) != cudaSuccess) return HODLR_ERR_CUDA;
  return static_cast<hodlr_status>(ds.code);
}

}  // namespace

hodlr_status hodlr_refine_workspace_size(hodlr_factor_t f, int32_t k, int32_t restart, size_t* bytes) {
  if (!valid_factor(f) || k < 1 || restart < 0 || restart > 200 || !bytes) return HODLR_ERR_ARG;
  *bytes = refine_layout(*f, k, restart).total;
  return HODLR_OK;
}

hodlr_status hodlr_solve_refined(hodlr_factor_t f, const double* D, const double* U, const double* V,
                                 const double* B, int64_t ldb, double* X, int64_t ldx, int32_t k, double tol,
                                 int32_t max_iter, int32_t restart, int32_t gmres_max_iter, void* workspace,
                                 size_t workspace_bytes, hodlr_stream_t stream, int32_t* iters, double* relres) {
  if (!valid_factor(f) || !D || !U || !V || !B || !X || k < 1 || ldb < f->d.N || ldx < f->d.N || max_iter < 0 ||
      restart < 0 || restart > 200 || gmres_max_iter < 0 || !(tol > 0.0))
    return HODLR_ERR_ARG;
  const RefineLayout lay = refine_layout(*f, k, restart);
  if (!workspace || !aligned(workspace, kAlign) || workspace_bytes < lay.total) return HODLR_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(workspace);
  double* R = reinterpret_cast<double*>(w + lay.R);
  void* sw = w + lay.solve;
  void* mw = w + lay.mv;
  double* scratch = reinterpret_cast<double*>(w + lay.dots);
  double* dev_n = reinterpret_cast<double*>(w + lay.scal);
  const hodlr_desc& d = f->d;
  const int64_t N = d.N;
  std::vector<double> nb(k), nr(k);
  hodlr_status st;
  HODLR_CUDA(launch_copy_cols<double, double>(N, k, B, ldb, X, ldx, s));
  if ((st = solve_any(*f, X, ldx, k, sw, 0, s)) != HODLR_OK) return st;
  if ((st = col_norms2(N, k, B, ldb, dev_n, scratch, nb.data(), s)) != HODLR_OK) return st;
  double prev = INFINITY, best = INFINITY;
  int grew = 0, it = 0;
  double worst = INFINITY;
  const bool keep_best = restart > 0 && gmres_max_iter > 0;
  double* Xb = keep_best ? reinterpret_cast<double*>(w + lay.Xb) : nullptr;
  for (;;) {
    if ((st = matvec_core(d, D, U, V, X, ldx, R, N, k, mw, s, matvec_ws_bytes(d, k))) != HODLR_OK) return st;
    HODLR_CUDA(launch_axpby_cols(N, k, 1.0, B, ldb, -1.0, R, N, s));  // R = B - A X
    if ((st = col_norms2(N, k, R, N, dev_n, scratch, nr.data(), s)) != HODLR_OK) return st;
    worst = 0.0;
    for (int j = 0; j < k; ++j) {
      const double rr = nb[j] > 0.0 ? std::sqrt(nr[j] / nb[j]) : std::sqrt(nr[j]);
      worst = std::isnan(rr) ? INFINITY : (rr > worst ? rr : worst);
    }
    if (keep_best && worst < best) {  // the iterate FGMRES continues from if refinement stalls
      best = worst;
      HODLR_CUDA(launch_copy_cols<double, double>(N, k, X, ldx, Xb, N, s));
    }
    if (worst <= tol || it >= max_iter) break;
    grew = worst > prev ? grew + 1 : 0;
    if (grew >= 2) break;
    prev = worst;
    if ((st = solve_any(*f, R, N, k, sw, 0, s)) != HODLR_OK) return st;
    HODLR_CUDA(launch_axpby_cols(N, k, 1.0, R, N, 1.0, X, ldx, s));  // X += correction
    ++it;
  }
  int git = 0;
  if (!(worst <= tol) && keep_best) {
    // refinement stalled (or ran out of corrections): FGMRES from its best iterate
    HODLR_CUDA(launch_copy_cols<double, double>(N, k, Xb, N, X, ldx, s));
    st = gmres_core(*f, D, U, V, B, ldb, X, ldx, k, tol, restart, gmres_max_iter, true, w, lay, s, &git, &worst);
    if (st != HODLR_OK && st != HODLR_ERR_NOT_CONVERGED) return st;
  }
  if (iters) *iters = it + git;
  if (relres) *relres = worst;
  if ((st = device_status(*f)) != HODLR_OK) return st;
  return worst <= tol ? HODLR_OK : HODLR_ERR_NOT_CONVERGED;
}

hodlr_status hodlr_gmres(hodlr_factor_t f, const double* D, const double* U, const double* V, const double* B,
                         int64_t ldb, double* X, int64_t ldx, int32_t k, double tol, int32_t restart,
                         int32_t max_iter, void* workspace, size_t workspace_bytes, hodlr_stream_t stream,
                         int32_t* iters, double* relres) {
  if (!valid_factor(f) || !D || !U || !V || !B || !X || k < 1 || ldb < f->d.N || ldx < f->d.N || restart < 1 ||
      restart > 200 || max_iter < 0 || !(tol > 0.0))
    return HODLR_ERR_ARG;
  const RefineLayout lay = refine_layout(*f, k, restart);
  if (!workspace || !aligned(workspace, kAlign) || workspace_bytes < lay.total) return HODLR_ERR_WORKSPACE;
  double worst = INFINITY;
  int it = 0;
  hodlr_status st = gmres_core(*f, D, U, V, B, ldb, X, ldx, k, tol, restart, max_iter, false,
                               static_cast<char*>(workspace), lay, reinterpret_cast<cudaStream_t>(stream), &it,
                               &worst);
  if (st != HODLR_OK && st != HODLR_ERR_NOT_CONVERGED) return st;
  if (iters) *iters = it;
  if (relres) *relres = worst;
  hodlr_status ds = device_status(*f);
  if (ds != HODLR_OK) return ds;
  return worst <= tol ? HODLR_OK : HODLR_ERR_NOT_CONVERGED;
}

// ------------------------------------------------------------------ gradient
}  // extern "C"

namespace {

struct GradLayout {
  size_t X, Lam, Z, Pb, E, H, HT, Ps, solve, dots, total;
};

GradLayout grad_layout(const Factor& F, int k) {
  const hodlr_desc& d = F.d;
  GradLayout l{};
  const size_t N = (size_t)d.N, rL = (size_t)d.r * d.L;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += align_up(bytes); return o; };
  l.X = take(N * k * 8);
  l.Lam = take(N * k * 8);
  l.Z = take(N * rL * 8);
  l.Pb = take(N * rL * 8);
  l.E = take(N * (size_t)d.m * 8);
  l.H = take(((size_t)1 << d.L) * d.r * d.r * 8);
  l.HT = take(((size_t)1 << d.L) * d.r * d.r * 8);
  size_t ps = 0;
  for (int c = 1; c <= d.L; ++c) {
    const size_t w = (size_t)num_chunks(d.N, c) *
                     std::max<size_t>((size_t)k * d.r, std::max<size_t>((size_t)d.r * d.r, (size_t)d.r * d.r * (c - 1)));
    ps = std::max(ps, w);
  }
  l.Ps = take(ps * 8);
  l.solve = take(solve_ws_bytes(F, k));
  l.dots = take((dot_scratch_elems(d.N, k) + (size_t)k) * 8);
  l.total = off;
  return l;
}

// TP: the factor's panel type (FP64 factor: double; FP32 factor: float, whose
// Y, leaf inverses / LUs and solves then carry FP32 rounding into the
// gradient; the coupling inverses and every accumulation stay FP64).
template <typename TP>
hodlr_status grad_core(const Factor& F, const double* U, const double* V, const double* B, int64_t ldb, int k,
                       double* dD, double* dU, double* dV, double* dB, int64_t lddb, char* w, const GradLayout& lay,
                       cudaStream_t s, double* loss) {
  const hodlr_desc& d = F.d;
  const int64_t N = d.N;
  const int r = d.r, L = d.L, m = d.m, rL = r * L;
  double* X = reinterpret_cast<double*>(w + lay.X);
  double* Lam = reinterpret_cast<double*>(w + lay.Lam);
  double* Z = reinterpret_cast<double*>(w + lay.Z);
  double* Pb = reinterpret_cast<double*>(w + lay.Pb);
  double* E = reinterpret_cast<double*>(w + lay.E);
  double* H = reinterpret_cast<double*>(w + lay.H);
  double* HT = reinterpret_cast<double*>(w + lay.HT);
  double* Ps = reinterpret_cast<double*>(w + lay.Ps);
  void* sw = w + lay.solve;
  double* dots = reinterpret_cast<double*>(w + lay.dots);
  const TP* Y = static_cast<const TP*>(F.Y);
  const int64_t ldu = d.ldu, ldv = d.ldv;
  hodlr_status st;
  // X = A^{-1} B, Lam = A^{-T} B, dB = X + Lam
  HODLR_CUDA(launch_copy_cols<double, double>(N, k, B, ldb, X, N, s));
  if ((st = solve_any(F, X, N, k, sw, 0, s)) != HODLR_OK) return st;
  HODLR_CUDA(launch_copy_cols<double, double>(N, k, B, ldb, Lam, N, s));
  if ((st = solve_any(F, Lam, N, k, sw, 1, s)) != HODLR_OK) return st;
  HODLR_CUDA(launch_copy_cols<double, double>(N, k, X, N, dB, lddb, s));
  HODLR_CUDA(launch_axpby_cols(N, k, 1.0, Lam, N, 1.0, dB, lddb, s));
  // quadratic term: dD_b = -Lam_b X_b^T; dU_a = -Lam_a (X_b^T V_b); dV_b = -X_b (Lam_a^T U_a)
  HODLR_CUDA(launch_leaf_outer(N, m, k, Lam, N, X, N, -1.0, 0.0, nullptr, dD, s));
  HODLR_CUDA(cudaMemsetAsync(dU, 0, (size_t)N * rL * 8, s));
  HODLR_CUDA(cudaMemsetAsync(dV, 0, (size_t)N * rL * 8, s));
  HODLR_CUDA(cudaMemsetAsync(Pb, 0, (size_t)N * rL * 8, s));
  for (int c = 1; c <= L; ++c) {
    const int64_t ws = chunks_per_node(N, c) * (int64_t)k * r;
    HODLR_CUDA((launch_project<double, double>(N, k, c, X, N, 0, V + (int64_t)(c - 1) * r * ldv, ldv, r, Ps, 1, s)));
    HODLR_CUDA(launch_reduce_chunks(N, k, c, Ps, r, s));
    HODLR_CUDA((launch_update<double, double>(N, k, c, Lam, N, 0, dU + (int64_t)(c - 1) * r * N, N, r, Ps, ws, 1,
                                              -1.0, 1, s)));
    HODLR_CUDA((launch_project<double, double>(N, k, c, Lam, N, 0, U + (int64_t)(c - 1) * r * ldu, ldu, r, Ps, 1, s)));
    HODLR_CUDA(launch_reduce_chunks(N, k, c, Ps, r, s));
    HODLR_CUDA((launch_update<double, double>(N, k, c, X, N, 0, dV + (int64_t)(c - 1) * r * N, N, r, Ps, ws, 1,
                                              -1.0, 1, s)));
  }
  // Z_alpha = A_alpha^{-T} V_alpha for every node: adjoint levels top-down on V_big's
  // ancestor columns, then D_b^{-T}
  HODLR_CUDA(launch_copy_cols<double, double>(N, rL, V, ldv, Z, N, s));
  for (int c = 2; c <= L; ++c) {
    const int anc = r * (c - 1);
    HODLR_CUDA((launch_project<TP, double>(N, r, c, Y, N, c - 1, Z, N, anc, Ps, 1, s)));
    HODLR_CUDA(launch_coupling_apply_any(F, c, Ps, anc, anc, 0, 1, s));
    const int64_t ws = chunks_per_node(N, c) * (int64_t)r * anc;
    HODLR_CUDA((launch_update<double, double>(N, r, c, V, ldv, c - 1, Z, N, anc, Ps, ws, 1, -1.0, 1, s)));
  }
  HODLR_CUDA((launch_leaf_solve<double, double>(F, Z, N, Z, N, rL, 1, s)));
  // log-det term at each coupling: dV_a += Y_a H_a^T, dU_a += Z_a H_a, Pb_a = -Z_a H_a
  for (int c = 1; c <= L; ++c) {
    HODLR_CUDA(launch_coupling_h(F, c, H, HT, s));
    const int64_t ws = (int64_t)r * r;
    HODLR_CUDA((launch_update<TP, double>(N, r, c, Y, N, c - 1, dV + (int64_t)(c - 1) * r * N, N, r, HT, ws, 0,
                                              1.0, 1, s)));
    HODLR_CUDA((launch_update<double, double>(N, r, c, Z, N, c - 1, dU + (int64_t)(c - 1) * r * N, N, r, H, ws, 0,
                                              1.0, 1, s)));
    HODLR_CUDA((launch_update<double, double>(N, r, c, Z, N, c - 1, Pb + (int64_t)(c - 1) * r * N, N, r, H, ws, 0,
                                              -1.0, 1, s)));
  }
  // push the rank-r terms Pb_a Y_a^T down to every pair (mu, nu) below a
  for (int c = 2; c <= L; ++c) {
    const int64_t ws = chunks_per_node(N, c) * (int64_t)r * r;
    for (int j = 0; j <= c - 2; ++j) {
      HODLR_CUDA((launch_project<TP, double>(N, r, c, Y, N, j, V + (int64_t)(c - 1) * r * ldv, ldv, r, Ps, 1, s)));
      HODLR_CUDA(launch_reduce_chunks(N, r, c, Ps, r, s));
      HODLR_CUDA((launch_update<double, double>(N, r, c, Pb, N, j, dU + (int64_t)(c - 1) * r * N, N, r, Ps, ws, 1,
                                                1.0, 1, s)));
      HODLR_CUDA((launch_project<double, double>(N, r, c, Pb, N, j, U + (int64_t)(c - 1) * r * ldu, ldu, r, Ps, 1, s)));
      HODLR_CUDA(launch_reduce_chunks(N, r, c, Ps, r, s));
      HODLR_CUDA((launch_update<TP, double>(N, r, c, Y, N, j, dV + (int64_t)(c - 1) * r * N, N, r, Ps, ws, 1, 1.0,
                                                1, s)));
    }
  }
  // leaves: dD_b += D_b^{-T} + Pb(I_b, :) Y(I_b, :)^T
  HODLR_CUDA(launch_leaf_identity(N, m, E, s));
  HODLR_CUDA((launch_leaf_solve<double, double>(F, E, N, E, N, m, 0, s)));
  HODLR_CUDA(launch_leaf_outer<TP>(N, m, rL, Pb, N, Y, N, 1.0, 1.0, E, dD, s));
  if (loss) {
    HODLR_CUDA(launch_dots(N, k, B, ldb, X, N, dots + dot_scratch_elems(N, k), dots, s));
    std::vector<double> q(k);
    HODLR_CUDA(cudaMemcpyAsync(q.data(), dots + dot_scratch_elems(N, k), (size_t)k * 8, cudaMemcpyDeviceToHost, s));
    HODLR_CUDA(launch_logdet_reduce(F, s));
    double ld[2];
    HODLR_CUDA(cudaMemcpyAsync(ld, F.ld_out, sizeof(ld), cudaMemcpyDeviceToHost, s));
    HODLR_CUDA(cudaStreamSynchronize(s));
    double acc = ld[1];
    for (int j = 0; j < k; ++j) acc += q[j];
    *loss = acc;
  }
  return HODLR_OK;
}

}  // namespace

extern "C" {

hodlr_status hodlr_grad_workspace_size(hodlr_factor_t f, int32_t k, size_t* bytes) {
  if (!valid_factor(f) || f->prec == HODLR_PREC_BF16 || k < 1 || k > 64 || !bytes)
    return HODLR_ERR_ARG;
  *bytes = grad_layout(*f, k).total;
  return HODLR_OK;
}

hodlr_status hodlr_grad(hodlr_factor_t f, const double* U, const double* V, const double* B, int64_t ldb, int32_t k,
                        double* dD, double* dU, double* dV, double* dB, int64_t lddb, void* workspace,
                        size_t workspace_bytes, hodlr_stream_t stream, double* loss) {
  if (!valid_factor(f) || f->prec == HODLR_PREC_BF16 || !U || !V || !B || !dD ||
      !dU || !dV || !dB || k < 1 || k > 64 || ldb < f->d.N || lddb < f->d.N)
    return HODLR_ERR_ARG;
  const GradLayout lay = grad_layout(*f, k);
  if (!workspace || !aligned(workspace, kAlign) || workspace_bytes < lay.total) return HODLR_ERR_WORKSPACE;
  char* w = static_cast<char*>(workspace);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  hodlr_status st = f->prec == HODLR_PREC_FP64
                        ? grad_core<double>(*f, U, V, B, ldb, k, dD, dU, dV, dB, lddb, w, lay, s, loss)
                        : grad_core<float>(*f, U, V, B, ldb, k, dD, dU, dV, dB, lddb, w, lay, s, loss);
  if (st != HODLR_OK) return st;
  if (loss) {
    DevStatus ds{};
    HODLR_CUDA(cudaMemcpy(&ds, f->status, sizeof(ds), cudaMemcpyDeviceToHost));
    if (ds.code != 0) return static_cast<hodlr_status>(ds.code);
  }
  return HODLR_OK;
}

int64_t hodlr_launch_count(void) { return g_launches.load(); }

void hodlr_tc_enable(int32_t on) { g_use_tc = on != 0; }

void hodlr_coupling_fp64_enable(int32_t on) { g_coupling_fp64 = on != 0; }

void hodlr_profile_enable(int32_t on) { g_prof.store(on != 0); }

void hodlr_profile_reset(void) {
  std::lock_guard<std::mutex> g(g_mu);
  for (int i = 0; i < KC_COUNT; ++i) {
    g_ms[i] = 0.0;
    g_n[i] = 0;
    g_bytes[i] = 0.0;
    g_flops[i] = 0.0;
  }
}

int32_t hodlr_profile_work(double* bytes, double* flops, int32_t n) {
  hodlr_profile_read(nullptr, nullptr, 0);
  std::lock_guard<std::mutex> g(g_mu);
  for (int i = 0; i < n && i < KC_COUNT; ++i) {
    if (bytes) bytes[i] = g_bytes[i];
    if (flops) flops[i] = g_flops[i];
  }
  return KC_COUNT;
}

int32_t hodlr_profile_read(double* ms, int64_t* launches, int32_t n) {
  cudaDeviceSynchronize();
  std::lock_guard<std::mutex> g(g_mu);
  for (const PendingBracket& p : g_pending) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
      g_ms[p.cls] += t;
      g_n[p.cls] += p.n;
      g_bytes[p.cls] += p.bytes;
      g_flops[p.cls] += p.flops;
    }
    g_pool.push_back(p.a);
    g_pool.push_back(p.b);
  }
  g_pending.clear();
  for (int i = 0; i < n && i < KC_COUNT; ++i) {
    if (ms) ms[i] = g_ms[i];
    if (launches) launches[i] = g_n[i];
  }
  return KC_COUNT;
}

const char* hodlr_profile_name(int32_t cls) {
  return (cls >= 0 && cls < KC_COUNT) ? kClassName[cls] : "";
}

}  // extern "C"
