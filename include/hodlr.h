/*
 * hodlr.h - C ABI of libhodlr, a GPU direct solver for HODLR matrices
 * (hierarchically off-diagonal low-rank; Chen & Martinsson, arXiv 2208.06290).
 *
 * The operator (Sec. 2, Def. 1-2, Eq. e:rank, Sec. 3.2 Eq. e:u)
 * ----------------------------------------------------------------
 * A is N x N with N = m * 2^L. The cluster tree is uniform: level c has 2^c
 * nodes, node i of level c owns rows [i*N/2^c, (i+1)*N/2^c). Leaves (level L)
 * own m rows. A is given by three device arrays, all FP64, all column-major:
 *   D  2^L consecutive m x m blocks, block b (rows b*m..b*m+m-1) at D + b*m*m,
 *      element (i, j) of a block at offset j*m + i      (the leaf blocks D_b);
 *   U  N x (r*L), leading dimension ldu >= N             (U_big of Eq. e:u);
 *   V  N x (r*L), leading dimension ldv >= N             (V_big).
 * Column block j (columns j*r .. j*r+r-1) of U and V holds the bases of the
 * level-(j+1) nodes on their own rows. For siblings alpha (left) and beta
 * (right) at level c: A(I_alpha, I_beta) = U_alpha V_beta^T and
 * A(I_beta, I_alpha) = U_beta V_alpha^T (Eq. e:rank). Only real FP64 input
 * is accepted; every rank is the same r (1 <= r <= 64, r <= m), m <= 256.
 *
 * Conventions for every entry point
 * ---------------------------------
 * - All matrix pointers are DEVICE pointers. Right-hand sides B / X / Y are
 *   N x k column-major with a leading dimension >= N.
 * - The library allocates no device memory. Calls that need scratch take a
 *   caller-owned device workspace; its size comes from the matching
 *   *_workspace_size query and it must be 256-byte aligned. A workspace may be
 *   reused once the stream work that used it has finished.
 * - Work is enqueued on the given stream (NULL = legacy default stream) and
 *   returns without waiting, except where a function says it synchronizes.
 * - Errors found on the host (bad sizes, null or misaligned pointers, a small
 *   workspace) are returned before anything is enqueued. Errors found on the
 *   device (a zero pivot, a non-finite input) are recorded in the factor and
 *   returned by hodlr_factor_status / hodlr_logdet / the refined solvers; the
 *   computation still runs to completion (LAPACK getrf "info" convention), and
 *   no kernel traps.
 */
#ifndef HODLR_H
#define HODLR_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define HODLR_API __attribute__((visibility("default")))
#else
#define HODLR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* hodlr_stream_t;

typedef enum {
  HODLR_OK = 0,
  HODLR_ERR_ARG = 1,               /* bad size, pointer, alignment or precision */
  HODLR_ERR_WORKSPACE = 2,         /* workspace too small or not 256-byte aligned */
  HODLR_ERR_CUDA = 3,              /* a CUDA runtime call failed */
  HODLR_ERR_SINGULAR_LEAF = 4,     /* exact zero pivot in a leaf LU (where = leaf, detail = column) */
  HODLR_ERR_SINGULAR_COUPLING = 5, /* exact zero pivot in a 2r x 2r coupling LU (where = heap node, detail = column) */
  HODLR_ERR_NONFINITE = 6,         /* NaN or Inf in D (where = leaf) */
  HODLR_ERR_NOT_CONVERGED = 7,     /* refinement / GMRES hit its iteration limit */
  HODLR_ERR_TIMEOUT = 8,           /* a device-side wait gave up after its spin limit (where = child level) */
  HODLR_ERR_SCRATCH_LIMIT = 9      /* problem too large for hodlr_matvec_noalloc's fixed scratch */
} hodlr_status;

/* Arithmetic of the factorization (not of the input, which is always FP64).
 *   FP64: everything in FP64.
 *   FP32: leaf LU, leaf solves and panel products in FP32 (FP32 accumulate).
 *   TF32: as FP32 (Y_big and V_big stored in FP32), but the per-level
 *         projections V^T Y run on the tensor cores with TF32 operands (the
 *         FP32 values' top 10 significand bits) and FP32 accumulation.
 *   BF16: as FP32, but Y_big and V_big are stored in bfloat16 and the panel
 *         products read them as such (FP32 accumulate); with r = 32 or 64 and
 *         node sizes that are multiples of 128 an ancestor update is added to
 *         the stored Y_big in bfloat16 (the update rounded, then the sum).
 * In every precision the 2r x 2r coupling matrices are formed, factored and
 * solved in FP64, and log-determinants are accumulated in FP64. A low-precision
 * factor is meant as the preconditioner of hodlr_solve_refined / hodlr_gmres. */
typedef enum {
  HODLR_PREC_FP64 = 0,
  HODLR_PREC_FP32 = 1,
  HODLR_PREC_TF32 = 2,
  HODLR_PREC_BF16 = 3
} hodlr_prec;

typedef struct {
  int64_t N;    /* matrix order, N = m << L */
  int32_t L;    /* number of levels below the root, 1 <= L <= 24 */
  int32_t m;    /* leaf size, 1 <= m <= 256 */
  int32_t r;    /* off-diagonal rank, 1 <= r <= min(m, 64) */
  int32_t reserved;  /* must be 0 */
  int64_t ldu;  /* leading dimension of U, >= N */
  int64_t ldv;  /* leading dimension of V, >= N */
} hodlr_desc;

typedef struct hodlr_factor_s* hodlr_factor_t;

/* Human-readable name of a status code (static string). */
HODLR_API const char* hodlr_strerror(hodlr_status s);

/* ---------------------------------------------------------------- factor --
 * Factorization stage of the level-by-level algorithm (Alg. 1; GPU form
 * Alg. 3): LU with partial pivoting of every leaf block; Y_big = D^{-1} U_big
 * leaf by leaf; then for child levels c = L..1: projections V^T Y of every
 * child on its own and ancestor columns, the 2r x 2r coupling matrix
 * K~ = [[I, V_beta^T Y_beta], [V_alpha^T Y_alpha, I]] of every parent (the
 * identity-diagonal variant given after Alg. 4) factored by LU with partial
 * pivoting, its solve with the ancestor projections as right-hand side
 * (Eq. e:node1), and the ancestor update Y(:, 1:r(c-1)) -= Y_own W (Eq. e:node2).
 *
 * hodlr_factor_workspace_size: bytes of device workspace hodlr_factor needs.
 * hodlr_factor: enqueues the factorization. D, U, V are read only and are not
 *   referenced after the call returns, except that in FP64 the factor keeps
 *   using V: the caller must keep V unchanged while the factor is in use. The
 *   workspace holds the factor and must stay allocated until hodlr_free.
 *   *out receives a host handle (owned by the caller, release with hodlr_free).
 */
HODLR_API hodlr_status hodlr_factor_workspace_size(const hodlr_desc* desc, hodlr_prec prec, size_t* bytes);
HODLR_API hodlr_status hodlr_factor(const hodlr_desc* desc, const double* D, const double* U, const double* V,
                          hodlr_prec prec, void* workspace, size_t workspace_bytes,
                          hodlr_stream_t stream, hodlr_factor_t* out);

/* In-place FP64 factorization (Sec. 3.2: the leaf LUs and Y_big take the
 * place of D and U_big): as hodlr_factor with HODLR_PREC_FP64, but the leaf
 * LU factors overwrite D (same block layout) and Y_big (D^{-1} U_big after
 * the level updates of Eq. e:node2) overwrites U, which must have ldu == N;
 * the workspace holds neither. The factor keeps using D, U and V: the caller must keep them
 * allocated and unchanged while the factor is in use, and keep its own copy of
 * the operator for residuals (hodlr_matvec, the refined solvers). V must not
 * alias U. */
HODLR_API hodlr_status hodlr_factor_inplace_workspace_size(const hodlr_desc* desc, size_t* bytes);
HODLR_API hodlr_status hodlr_factor_inplace(const hodlr_desc* desc, double* D, double* U, const double* V,
                                            void* workspace, size_t workspace_bytes, hodlr_stream_t stream,
                                            hodlr_factor_t* out);

/* Synchronizes the factor's stream and returns the first device-side error
 * (HODLR_OK if none). where / detail (may be NULL) locate it: leaf index and
 * column for a leaf, heap node number (root = 1) and column for a coupling. */
HODLR_API hodlr_status hodlr_factor_status(hodlr_factor_t f, int64_t* where, int64_t* detail);

/* Releases the host handle (not the caller's workspace). */
HODLR_API void hodlr_free(hodlr_factor_t f);

/* ----------------------------------------------------------------- solve --
 * hodlr_solve: B <- A^{-1} B in place for k columns (Alg. 2; GPU form Alg. 4):
 *   leaf solves with the stored LUs, then for child levels c = L..1 the
 *   projections V^T x, the stored coupling LU solve (Eq. e:node3) and the
 *   update x -= Y w (Eq. e:node4). In a low-precision factor the right-hand
 *   side is rounded to FP32 on entry and the result widened to FP64 on exit.
 * hodlr_solve_adjoint: B <- A^{-T} B in place. Uses the same factor read as
 *   A = F_0 F_L ... F_1 (Sec. 3.5, F_0 = blockdiag(D_b), F_c the 2x2-block
 *   factors of level c), so A^{-T} = F_0^{-T} F_L^{-T} ... F_1^{-T}: for
 *   c = 1..L (top-down) s = [Y_alpha^T x_alpha; Y_beta^T x_beta],
 *   K~^T t = s, x_alpha -= V_alpha t_2, x_beta -= V_beta t_1; then the leaf
 *   solves with D_b^T.
 * Workspace: hodlr_solve_workspace_size(f, k) bytes (same for both).
 */
HODLR_API hodlr_status hodlr_solve_workspace_size(hodlr_factor_t f, int32_t k, size_t* bytes);
HODLR_API hodlr_status hodlr_solve(hodlr_factor_t f, double* B, int64_t ldb, int32_t k,
                         void* workspace, size_t workspace_bytes, hodlr_stream_t stream);
HODLR_API hodlr_status hodlr_solve_adjoint(hodlr_factor_t f, double* B, int64_t ldb, int32_t k,
                                 void* workspace, size_t workspace_bytes, hodlr_stream_t stream);

/* ---------------------------------------------------------------- logdet --
 * (sign, log|det A|) from the factorization (Sec. 3.5): sum over leaves of
 * log|u_ii| of the leaf LUs plus, by Sylvester's determinant theorem, the
 * log|det K~| of every coupling matrix; sign = product of the signs with the
 * pivot-swap parities. Accumulated in FP64 in a fixed order (deterministic).
 * Synchronizes the stream. Returns the factor's device status (a singular
 * factor gives log|det| = -inf). */
HODLR_API hodlr_status hodlr_logdet(hodlr_factor_t f, hodlr_stream_t stream, double* sign, double* logabsdet);

/* ---------------------------------------------------------------- matvec --
 * Y = A X in FP64 from the unfactored (D, U, V), straight from the block
 * definition (Eq. e:rank): leaf products D_b X_b, then for every pair of
 * siblings U_alpha (V_beta^T X_beta) and U_beta (V_alpha^T X_alpha). X and Y
 * must not overlap. This is the residual operator of relres = |b - Ax| / |b|
 * (Sec. 4, Table t:notation2). */
HODLR_API hodlr_status hodlr_matvec_workspace_size(const hodlr_desc* desc, int32_t k, size_t* bytes);
HODLR_API hodlr_status hodlr_matvec(const hodlr_desc* desc, const double* D, const double* U, const double* V,
                          const double* X, int64_t ldx, double* Y, int64_t ldy, int32_t k,
                          void* workspace, size_t workspace_bytes, hodlr_stream_t stream);

/* Allocation-free variant of hodlr_matvec (no counterpart in the paper; a
 * service for callers that cannot allocate device memory where they need
 * A X: code inside a CUDA-graph capture that must not add allocation nodes,
 * plug-ins whose host application owns all device memory, real-time loops
 * where allocation latency or failure is not acceptable). It computes the
 * same FP64 Y = A X with the same kernels, but takes its scratch from one
 * fixed 32 MiB array of device memory defined by the library itself (every
 * GPU that loads the library holds it until the process exits) instead of a
 * caller workspace; it calls no allocator. The limit it enforces is on the
 * per-level projection partials: max over child levels c of
 * chunks(c) * r * k doubles must fit in 32 MiB, where chunks(c) = N / ch(c)
 * and ch(c) is the node size N / 2^c halved until it is at most 1024 rows;
 * larger problems are rejected with HODLR_ERR_SCRATCH_LIMIT before anything
 * is enqueued. That bound is the minimum of hodlr_matvec_workspace_size; with
 * k = 1 the four-launch one-column path runs only when its larger scratch
 * (the size hodlr_matvec_workspace_size(desc, 1) reports) also fits, else the
 * general per-level path runs (same result). The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture. All
 * calls share the array: calls that overlap on the GPU race and must be
 * serialized by the caller. Nothing in the scratch needs to start at zero. */
HODLR_API hodlr_status hodlr_matvec_noalloc(const hodlr_desc* desc, const double* D, const double* U, const double* V,
                                            const double* X, int64_t ldx, double* Y, int64_t ldy, int32_t k,
                                            hodlr_stream_t stream);

/* ------------------------------------------------------- refined solvers --
 * Mixed-precision solves recovered to FP64 accuracy. The factor f (any
 * precision) of the HODLR matrix (desc, D, U, V) is the preconditioner; the
 * residual uses the FP64 hodlr_matvec on the unfactored D, U, V. The k
 * right-hand sides advance together: every correction or inner iteration
 * applies the factor to all k columns in one k-column solve and the FP64
 * operator in one k-column matvec.
 *
 * hodlr_solve_refined: iterative refinement, X <- X + f^{-1}(B - A X),
 *   starting from X = f^{-1} B, until max_j |b_j - A x_j| / |b_j| <= tol or
 *   max_iter corrections; it stops early when the residual grows twice in a
 *   row. If tol is not reached then and restart > 0, flexible GMRES(restart)
 *   continues from the best refined iterate for at most gmres_max_iter inner
 *   iterations (restart = 0: no continuation; the workspace then holds no
 *   Krylov basis).
 * hodlr_gmres: flexible GMRES (restart length `restart`, at most max_iter
 *   inner iterations in total) right-preconditioned by f, started from
 *   X = f^{-1} B, stopping on the FP64 residual <= tol. Per cycle the residual
 *   is b - A x of the first iterate (one FP64 matvec) and then r - (A Z) y
 *   from the stored FP64 products A z_i; when that recursive residual meets
 *   tol while its accumulated rounding bound (about eps sum |y_i| |A z_i|, the
 *   drift between it and b - A x on ill-conditioned operators) could exceed
 *   tol / 100, b - A x is recomputed and iteration continues from it.
 *   Classical Gram-Schmidt twice, per
 *   column; a column whose residual estimate has converged stops extending
 *   its basis while the others continue.
 * Both write the solution to X (N x k, ldx), leave B unchanged, return
 * HODLR_ERR_NOT_CONVERGED if tol was not reached, report the iteration count
 * (refinement corrections plus FGMRES inner iterations) in *iters and the
 * final max relative residual in *relres. They synchronize the stream once per
 * iteration to read residual norms.
 * Workspace: hodlr_refine_workspace_size(f, k, restart) (restart 0 for
 * refinement without FGMRES continuation; 1 <= restart <= 200 otherwise);
 * FGMRES holds 3 * restart + 2 vectors of N x k doubles.
 */
HODLR_API hodlr_status hodlr_refine_workspace_size(hodlr_factor_t f, int32_t k, int32_t restart, size_t* bytes);
HODLR_API hodlr_status hodlr_solve_refined(hodlr_factor_t f, const double* D, const double* U, const double* V,
                                 const double* B, int64_t ldb, double* X, int64_t ldx, int32_t k,
                                 double tol, int32_t max_iter, int32_t restart, int32_t gmres_max_iter,
                                 void* workspace, size_t workspace_bytes,
                                 hodlr_stream_t stream, int32_t* iters, double* relres);
HODLR_API hodlr_status hodlr_gmres(hodlr_factor_t f, const double* D, const double* U, const double* V,
                         const double* B, int64_t ldb, double* X, int64_t ldx, int32_t k,
                         double tol, int32_t restart, int32_t max_iter,
                         void* workspace, size_t workspace_bytes, hodlr_stream_t stream,
                         int32_t* iters, double* relres);

/* -------------------------------------------------------------- gradient --
 * Gradient of  loss = sum_j b_j^T A^{-1} b_j + log|det A|  (k columns b_j of
 * B) with respect to B, the leaf blocks D_b and the bases U_big, V_big, for an
 * FP64 factor f of (D, U, V). With X = A^{-1} B, Lam = A^{-T} B and
 * G = dloss/dA = -Lam X^T + A^{-T}:
 *   dB = X + Lam;  dD_b = G(I_b, I_b);  for siblings (alpha, beta):
 *   dU_alpha = G(I_alpha, I_beta) V_beta,  dV_beta = G(I_alpha, I_beta)^T U_alpha.
 * The -Lam X^T part is rank k and is applied block by block. The A^{-T} part
 * is taken through the factorization A = F_0 F_L ... F_1 (Sec. 3.5):
 * log|det A| = sum log|det D_b| + sum log|det K~_gamma|; with
 * Z_alpha = A_alpha^{-T} V_alpha (a top-down sweep of the adjoint levels over
 * V_big) and H_alpha the off-diagonal block of K~_gamma^{-T} facing alpha,
 * dV_alpha += Y_alpha H_alpha^T, dU_alpha += Z_alpha H_alpha, and the rank-r
 * term -Z_alpha H_alpha Y_alpha^T of dloss/dA_alpha is pushed to every pair
 * and leaf below alpha; dD_b also gets D_b^{-T}.
 * dD has D's layout, dU and dV are N x rL with leading dimension N, dB is
 * N x k (lddb). Results overwrite the outputs. If loss is not NULL the call
 * synchronizes and stores the loss value. FP64, FP32 and TF32 factors
 * (HODLR_ERR_ARG for BF16). With an FP32 factor the solves, Y_big and the
 * leaf inverses / LUs carry FP32 rounding (coupling inverses, log-dets and
 * accumulations stay FP64): its gradient approximates the FP64 one to about
 * the FP32 factor's solve accuracy. */
HODLR_API hodlr_status hodlr_grad_workspace_size(hodlr_factor_t f, int32_t k, size_t* bytes);
HODLR_API hodlr_status hodlr_grad(hodlr_factor_t f, const double* U, const double* V, const double* B, int64_t ldb,
                                  int32_t k, double* dD, double* dU, double* dV, double* dB, int64_t lddb,
                                  void* workspace, size_t workspace_bytes, hodlr_stream_t stream, double* loss);

/* ----------------------------------------------------------- construction --
 * GPU construction of the HODLR approximation (Sec. 2.2) of a built-in
 * kernel or boundary-integral matrix, in the layout every other entry point
 * takes. Leaf blocks D_b are evaluated exactly in FP64. Every off-diagonal
 * sibling block A(I_alpha, I_beta) is compressed to the fixed rank r of desc
 * by a partial-pivoted cross approximation (the approximate partial-pivoted
 * LU the paper's kernel experiments used for this step): with i_0 the
 * block's first row, for k = 0 .. r-1 the residual row at i_k, its largest
 * entry (column j_k, first maximum among unused columns), v_k = row / that
 * entry, the residual column u_k at j_k and i_{k+1} = its largest entry among
 * the unused rows; A(I_alpha, I_beta) ~= sum u_k v_k^T = U_alpha V_beta^T.
 * A block whose residual vanishes keeps zero bases from then on; with
 * tol > 0 a block also stops at the first step whose pivot is at most
 * tol times its first pivot (tolerance-driven, per-block ranks <= r; the
 * bases beyond a block's rank are zero, so the output is the zero-padded
 * uniform layout of a variable-rank HODLR matrix). Entries are evaluated
 * from FP64 geometry and rounded to FP32; the residual updates are FP32; the
 * bases are stored in FP64. For the symmetric
 * kernel matrices one cross per sibling pair gives both blocks, so U = V.
 *
 * Kernels (hodlr_kernel_desc.kind):
 *   HODLR_KERNEL_BIE_STAR: 2D Laplace double-layer second-kind BIE on the
 *     star curve rho(t) = 1 + 0.3 cos 5t, N trapezoid nodes t_i = 2 pi i / N
 *     in curve order: A = -1/2 I + D, D(i, j) = n_j.(x_i - x_j) /
 *     (2 pi |x_i - x_j|^2) w_j (n the outward normal, w_j = |gamma'(t_j)|
 *     2 pi / N), diagonal -1/2 - w_i kappa_i / (4 pi) (kappa the curvature);
 *     points, dim, scale and nugget are ignored.
 *   HODLR_KERNEL_GAUSSIAN: exp(-|x_i - x_j|^2 / (2 scale^2)) + nugget delta_ij;
 *   HODLR_KERNEL_MATERN32: (1 + sqrt(3) d / scale) exp(-sqrt(3) d / scale)
 *     + nugget delta_ij, d = |x_i - x_j|;
 *   for these two, points is a DEVICE array of N points of dim (1..3) FP64
 *   coordinates, point i at points + i * dim, already in the cluster tree's
 *   order (node i of level c owns points i N / 2^c ..).
 * D, U, V are outputs in the layout of hodlr_factor (ldu, ldv of desc).
 * pivots (optional, device, 2 r (2^(L+1) - 2) int32): per level c = 1..L at
 * offset 2 r (2^c - 2), the pivot rows [block][k] then the pivot columns
 * [block][k] (indices local to the block; -1 after a vanished residual); the
 * blocks of level c are its 2^c nodes (row node = block; for a symmetric
 * kernel only the even ones are used). ranks (optional, device,
 * 2^(L+1) - 2 int32): the rank of every block, level c at offset 2^c - 2.
 * Workspace: hodlr_compress_workspace_size. Enqueued on the stream; no
 * allocation. */
typedef enum {
  HODLR_KERNEL_BIE_STAR = 0,
  HODLR_KERNEL_GAUSSIAN = 1,
  HODLR_KERNEL_MATERN32 = 2
} hodlr_kernel;

typedef struct {
  int32_t kind;          /* hodlr_kernel */
  int32_t dim;           /* point dimension, 1..3 (kernel matrices) */
  const double* points;  /* device, N x dim (kernel matrices), NULL for the BIE */
  double scale;          /* Gaussian sigma / Matern lengthscale */
  double nugget;         /* added to the diagonal (kernel matrices) */
  double tol;            /* relative pivot tolerance of the cross approximation, 0 <= tol < 1 (0: rank r) */
} hodlr_kernel_desc;

HODLR_API hodlr_status hodlr_compress_workspace_size(const hodlr_desc* desc, size_t* bytes);
HODLR_API hodlr_status hodlr_compress(const hodlr_desc* desc, const hodlr_kernel_desc* kern, double* D, double* U,
                                      double* V, int32_t* pivots, int32_t* ranks, void* workspace,
                                      size_t workspace_bytes, hodlr_stream_t stream);

/* Variable ranks per level (Eq. e:u, Sec. 3.2 with per-level widths): the
 * ragged Ur / Vr (N x sum r_c, leading dimensions ldur, ldvr >= N) hold level
 * c's bases in columns off_c .. off_c + r_c - 1 (off_c = r_1 + ... + r_{c-1}),
 * each node's basis left-aligned (zeros right of a lower-rank node's basis).
 * hodlr_pack_level_ranks writes the same matrix in the uniform layout of
 * desc (r >= every r_c; level blocks zero-padded on the right), which every
 * other entry point takes; the padding changes no product (U_alpha V_beta^T
 * is unchanged) and costs r / r_c of a level's panel work. level_ranks is a
 * HOST array of L entries; workspace >= 2 L ints (device). Synchronizes the
 * stream. */
HODLR_API hodlr_status hodlr_pack_level_ranks(const hodlr_desc* desc, const int32_t* level_ranks, const double* Ur,
                                              int64_t ldur, const double* Vr, int64_t ldvr, double* U, double* V,
                                              void* workspace, size_t workspace_bytes, hodlr_stream_t stream);

/* ------------------------------------------------------------ diagnostics --
 * Accounting of the library's own kernel launches, for benchmarks; not part
 * of the method. hodlr_launch_count: kernels enqueued by this library since
 * it was loaded (all threads). hodlr_profile_enable(1): from then on every
 * launch is bracketed by CUDA events recorded on the launching stream, and
 * hodlr_profile_read synchronizes the device, folds the elapsed times into
 * per-kernel-class totals, copies up to n of them (milliseconds and launch
 * counts, in class order) and returns the number of classes;
 * hodlr_profile_name gives a class's name, hodlr_profile_reset clears the
 * totals. hodlr_profile_work gives, per class, the algorithmic bytes and
 * flops of the profiled launches (the operation's definition: every operand
 * read once and every result written once, not the traffic the kernels
 * actually cause). Profiling is process-wide and not thread-safe; it is off
 * by default. */
HODLR_API int64_t hodlr_launch_count(void);
/* Tensor-core kernels (tcgen05/TMA) for the BF16 factor's panel products:
 * on by default; off selects the CUDA-core kernels (same results up to FP32
 * summation order). Process-wide; for tests and benchmarks. */
HODLR_API void hodlr_tc_enable(int32_t on);
/* BF16 factor, r <= 32: on forms S = I - T_alpha T_beta and the products of
 * the explicit coupling inverse in FP64 (as the FP64 and FP32 factors do);
 * off (default) forms them with FP32 products, the elimination of S staying
 * FP64. Process-wide; for the precision experiment of benchmarks and tests. */
HODLR_API void hodlr_coupling_fp64_enable(int32_t on);
HODLR_API void hodlr_profile_enable(int32_t on);
HODLR_API void hodlr_profile_reset(void);
HODLR_API int32_t hodlr_profile_read(double* ms, int64_t* launches, int32_t n);
HODLR_API int32_t hodlr_profile_work(double* bytes, double* flops, int32_t n);
HODLR_API const char* hodlr_profile_name(int32_t cls);

/* FP64 pipe probe (a diagnostic, not part of the method): enqueues one kernel
 * of blocks_per_sm (1..64) blocks of 256 threads per SM of the current
 * device, each thread running 8 independent chains of `iters` dependent FP64
 * FMAs on registers only; *fmas receives the total FMA count. `out` is a
 * device pointer to one double that the kernel never writes in practice (it
 * only keeps the chains from being optimized away). Timing the launch with
 * events on `stream` gives the FP64 FMA rate that bounds FP64-pipe-bound
 * kernels on this GPU at its current clock. */
HODLR_API hodlr_status hodlr_probe_fp64_fma(int64_t iters, int32_t blocks_per_sm, double* out,
                                            hodlr_stream_t stream, int64_t* fmas);

#ifdef __cplusplus
}
#endif
#endif /* HODLR_H */
