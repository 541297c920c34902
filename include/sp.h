/*
 * sp.h -- C ABI of the GB300 (sm_103a) spectral-projector library.
 *
 * Computes Pi_{<mu}(A) = (I - sign(A - mu I)) / 2 for a symmetric banded A
 * with the hQDWH algorithm of Kressner & Susnjara, "Fast computation of
 * spectral projectors of banded matrices" (arXiv 1608.01164): the QDWH
 * iteration for the matrix sign function (Sec. 2, Eqs. (reccur),
 * (qdwh_qr_reccur), (qdwh_chol_reccur)) carried out in HODLR format
 * (Sec. 3.1.1), with one QR-based first step built from Givens rotations
 * (Sec. 4, Algorithms 1 and 2) and Cholesky-based steps afterwards
 * (Algorithm 3).
 *
 * Conventions (all entry points):
 *  - Every call returns an int status: SP_OK = 0 or one of the SP_E* codes
 *    below.  No C++ exception crosses this boundary.  The message of the last
 *    failure on a context is available from sp_last_error().
 *  - Dense matrices are column-major with an explicit leading dimension (ld).
 *    Band input uses LAPACK lower band storage: ab[(i-j) + j*ldab] = A(i,j)
 *    for 0 <= i-j <= b, ldab >= b+1; entries with i >= n are ignored.
 *  - Pointers are device or host pointers as stated per argument; where a
 *    call accepts either, it detects the kind with cudaPointerGetAttributes.
 *    The caller keeps ownership of every buffer it passes.  sp_ctx_t and
 *    sp_hodlr_t handles are owned by the library until their *_destroy call.
 *  - All device work is ordered on the context's CUDA stream.  Calls return
 *    after enqueueing unless stated otherwise ("synchronising").
 *  - Arithmetic is IEEE binary64 unless the options select a mixed-precision
 *    mode.
 */
#ifndef SP_H
#define SP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define SP_OK 0
#define SP_EINVAL 1      /* invalid argument (size, leaf, tolerance, pointer) */
#define SP_ENOMEM 2      /* device allocation failed */
#define SP_ECUDA 3       /* a CUDA runtime call or kernel launch failed */
#define SP_EBREAKDOWN 4  /* H-Cholesky met a non-positive pivot */
#define SP_ENONFINITE 5  /* NaN/Inf detected in an iterate */
#define SP_ERANK 6       /* a truncated rank exceeded the rank capacity */
#define SP_ETIMEOUT 7    /* a bounded device wait gave up */
#define SP_EINTERNAL 8   /* internal consistency check failed */

/* Precision modes for sp_qdwh_sign. */
#define SP_FP64 0        /* every step in binary64 */
#define SP_MIXED_FP32 1  /* Cholesky steps with 1 - l_k^2 <= 1e-2 in residual form
                            X + (a-1) X Z^{-1} (I - X^2) with binary32 GEMM
                            arithmetic (binary64 storage, residual, sum and
                            recompression), then binary64 Newton-Schulz polish */
#define SP_MIXED_NS 2    /* once 1 - l_k^2 <= 1e-2 the remaining QDWH steps are
                            replaced by Newton-Schulz steps in residual form
                            X + X (I - X^2)/2: I - X^2 in binary64, the product
                            X (I - X^2) with binary32 GEMM arithmetic, as many
                            steps as the scalar map l <- l(3 - l^2)/2 needs to
                            reach 1 - l <= 1e-12; then the binary64 polish.
                            No H-Cholesky in the late steps (not the paper's
                            iteration; a growth direction). */

typedef struct sp_ctx* sp_ctx_t;
typedef struct sp_hodlr* sp_hodlr_t;

/* Options of the QDWH iteration (Sec. 2.1, Algorithm 3). */
typedef struct {
  int max_iter;      /* hard cap on QDWH iterations (default 10) */
  double delta;      /* stopping tolerance: stop when |1 - l_k| <= delta (default 1e-15) */
  int precision;     /* SP_FP64 (default), SP_MIXED_FP32 or SP_MIXED_NS */
  int polish_steps;  /* binary64 Newton-Schulz steps X <- X (3I - X^2)/2 after a mixed run (default 1) */
  double alpha;      /* > 0: use as the bound alpha >= ||A - mu I||_2; 0: estimate it */
  double l0;         /* > 0: use as the bound l0 <= sigma_min(X_0); 0: estimate it */
  int qr_steps;      /* number of QR-based steps; the paper uses exactly one (default 1) */
} sp_qdwh_opts;

/* Diagnostics filled by sp_qdwh_sign (synchronising when non-NULL). */
typedef struct {
  int iters;               /* QDWH iterations performed */
  double alpha, l0;        /* the parameters used */
  double l[16], a[16], b[16], c[16]; /* l_k, a_k, b_k, c_k per iteration */
  int kind[16];            /* 1 = QR-based, 2 = Cholesky-based, 3 = mixed residual, 4 = mixed Newton-Schulz step */
  int max_rank;            /* largest off-diagonal rank of the result */
  size_t bytes;            /* device bytes held by the result (allocated at the rank capacity) */
  double ms_param, ms_qr, ms_chol, ms_total; /* phase times (CUDA events) */
  double flops;            /* nominal binary64 flops counted by the kernels' task lists */
  /* inside the Cholesky-based steps: formatted products, H-Cholesky (with the
   * inverse factor), the two products with the inverse factor, and the final
   * combination + symmetrisation (CUDA events, summed over iterations) */
  double ms_mult, ms_factor, ms_solve, ms_combine;
  double ms_polish;        /* binary64 Newton-Schulz polish (mixed precision) */
  /* Structure of the result (Sec. 3.1.1; the memory estimate of Sec. 3.2):
   * per tree level l = 1..levels, the largest and the mean off-diagonal rank
   * of its 2^l blocks (index l-1; levels beyond 32 are not reported), and the
   * nominal storage 8 * (sum of leaf sizes^2 + sum over blocks of
   * (rows + cols) * rank) bytes of the same matrix at its actual ranks. */
  int levels;
  int max_rank_level[32];
  double mean_rank_level[32];
  double nominal_bytes;
} sp_info;

/* Returns opts filled with the defaults listed above. */
void sp_qdwh_opts_default(sp_qdwh_opts* opts);

/* Stream-ordered device allocator supplied by the caller (for example a host
 * program's own caching pool).  alloc returns `bytes` bytes of device memory
 * usable by work enqueued on `stream` after the call (NULL on failure, which
 * the library reports as SP_ENOMEM); free releases a buffer that work already
 * enqueued on `stream` may still be using, so the allocator must not hand it
 * out again before that work completes (stream-ordered reuse, as
 * cudaFreeAsync or a caching allocator that records stream events does).
 * `stream` is the cudaStream_t the buffer is used on; `user` is passed
 * through.  The paper has no counterpart (memory management of this library). */
typedef void* (*sp_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*sp_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

/* Creates a context bound to the current CUDA device and the given stream
 * (a cudaStream_t; NULL selects the legacy default stream).  Every device
 * buffer the context's calls make (temporaries and result handles) comes from
 * alloc/free when both are given, else from the device's default memory pool
 * (cudaMallocAsync; freed memory is kept in the pool across synchronisations).
 * Giving only one of the two is SP_EINVAL.  The paper has no counterpart. */
int sp_ctx_create(void* cuda_stream, sp_alloc_fn alloc, sp_free_fn free_fn, void* user, sp_ctx_t* out);
void sp_ctx_destroy(sp_ctx_t ctx);
const char* sp_last_error(sp_ctx_t ctx);
/* Blocks until all work enqueued on the context's stream has finished and
 * reports any sticky device error flag (rank overflow, breakdown, timeout). */
int sp_ctx_sync(sp_ctx_t ctx);

/* ---- measurement (not part of the method) ---- */

/* Profiling switch: when on, every launch of a kernel family is bracketed by
 * CUDA events on the context stream and the binary64 kernels count the
 * floating-point operations they perform (from the actual, device-resident
 * sizes) into device counters.  Turning it on or off resets the counters.
 * Synchronising. */
int sp_ctx_set_profiling(sp_ctx_t ctx, int on);
/* Accumulated launches, elapsed milliseconds (sum of event pairs) and counted
 * flops of kernel family `kernel` (0 <= kernel < sp_kernel_count()) since the
 * last reset.  Synchronising. */
int sp_ctx_profile(sp_ctx_t ctx, int kernel, int64_t* launches, double* ms, double* flops);

/* Per-tree-level self time (ms) of the H-Cholesky recursion while profiling
 * is on: for each node, the time of its own work on the context's stream
 * (Schur complement and inverse blocks for inner nodes, factor and inverse for
 * leaves), excluding its children, summed over the nodes of each level
 * 0..nlevels-1 and over every factorisation since profiling was enabled.
 * Synchronises the context's stream.  Measurement hook; the paper has no
 * counterpart.  Returns SP_EINVAL for nlevels < 0 or a NULL array. */
int sp_ctx_profile_levels(sp_ctx_t ctx, int nlevels, double* ms_self);
/* Name of a kernel family ("k_gemm", "k_qr", ...), "" if out of range. */
const char* sp_kernel_name(int kernel);
int sp_kernel_count(void);
/* Number of kernels this library has launched in the process so far. */
int64_t sp_launch_count(void);

/* HODLR representation of X_0 = A - mu I (Sec. 3.1.1): the index set is split
 * by balanced bisection into 2^L leaves of at most `leaf` indices (L the
 * smallest depth with ceil(n / 2^L) <= leaf); leaves are dense and every
 * off-diagonal block of the band is stored exactly as a rank-b corner
 * (Lemma 2: a band of width b has off-diagonal rank <= b).
 *   n >= 1; 1 <= b; leaf >= max(2, 2b) (so band corners stay inside sibling
 *   blocks), or leaf = 0 for the tuned / rule-based choice (sp_ctx_load_tuning); tol > 0 is the truncation tolerance epsilon of Sec. 3.1.1 and
 *   Sec. 5, an absolute threshold on the singular values of every recompressed
 *   block, kept with the matrix and used by every later formatted operation; rank_cap >= 2b is the per-block
 *   rank capacity (0 selects max(160, 20b)).
 *   ab: host or device pointer.  On success *out is a new handle. */
int sp_hodlr_from_band(sp_ctx_t ctx, int64_t n, int32_t b, const double* ab, int64_t ldab, double mu,
                       int32_t leaf, double tol, int32_t rank_cap, sp_hodlr_t* out);

/* sign(A - mu I) by hQDWH (Algorithm 3).  A is the handle produced by
 * sp_hodlr_from_band (it keeps the band, which the QR-based first step
 * needs).  opts may be NULL (defaults).  On success *sign_out is a new
 * handle; info (may be NULL) receives diagnostics. */
int sp_qdwh_sign(sp_ctx_t ctx, sp_hodlr_t A, const sp_qdwh_opts* opts, sp_hodlr_t* sign_out, sp_info* info);

/* Projectors of many independent banded instances (uneven n, b and mu):
 * instance i is A_i = ab[i] (lower band storage, ldab[i] >= b[i]+1, host or
 * device pointer) shifted by mu[i]; P_out[i] receives Pi_{<mu_i}(A_i) in HODLR
 * format (Algorithm 3 per instance).  Instances are spread over `nstreams`
 * CUDA streams (0 selects 16), each driven by its own host worker thread, so
 * the small kernels of many instances run concurrently; larger instances are
 * started first.  leaf = 0 picks the leaf size per instance from n and b
 * (64 for n <= 2048, 128 for n <= 8192, else 256, at least 2b).  infos (may be
 * NULL) receives per-instance diagnostics.  On return all work has finished
 * and the handles belong to the context's stream.  On failure no handle is
 * returned and the status of the first failing instance is reported. */
int sp_batched_projector(sp_ctx_t ctx, int32_t nbatch, const int64_t* n, const int32_t* b, const double* const* ab,
                         const int64_t* ldab, const double* mu, int32_t leaf, double tol, int32_t rank_cap,
                         const sp_qdwh_opts* opts, int32_t nstreams, sp_hodlr_t* P_out, sp_info* infos);

/* P = (I - S) / 2 (Algorithm 3, last line); new handle in *P_out. */
int sp_projector(sp_ctx_t ctx, sp_hodlr_t S, sp_hodlr_t* P_out);

/* Y = M X for a HODLR M and a dense n x nrhs block X (HODLR matrix-vector
 * product, Table "complexity_HODLR": O(k n log n) per column).
 * X, Y: column-major, ldx, ldy >= n; Y must not alias X.  Device pointers:
 * the product is enqueued on the context's stream (asynchronous).  Host
 * pointers (either one): the operand is staged through device memory and the
 * call returns once Y holds the result. */
int sp_apply(sp_ctx_t ctx, sp_hodlr_t M, int64_t nrhs, const double* X, int64_t ldx, double* Y, int64_t ldy);

/* Rows row0 .. row0+nrows-1 of M as a dense nrows x n panel (column-major,
 * ld >= nrows); out: host or device pointer.  Expands the HODLR format of
 * Sec. 3.1.1 (Eq. (HODLR): dense diagonal leaves, off-diagonal blocks U V^T);
 * the paper uses the dense matrix only to measure errors (Eq.
 * (error_measures)).  Host out: synchronising. */
int sp_to_dense(sp_ctx_t ctx, sp_hodlr_t M, int64_t row0, int64_t nrows, double* out, int64_t ld);

/* tr(M) (sum of the leaves' diagonals), summed in a fixed order (bitwise
 * reproducible).  For the projector, trace(P) is the number of eigenvalues
 * below mu (Sec. 1) and enters e_trace of Eq. (error_measures).
 * Synchronising. */
int sp_trace(sp_ctx_t ctx, sp_hodlr_t M, double* tr);

/* trace(M A) for a symmetric band A of M's order (lower band storage, ldab >=
 * b+1; ab host or device): sum_i M(i,i) a_ii + sum_{d=1..b} (M(i+d,i) +
 * M(i,i+d)) a_{i+d,i}, summed in a fixed order.  With M the projector
 * Pi_{<mu}(A) of the same A this is the sum of the eigenvalues below mu, the
 * band energy of the density-matrix application that motivates the paper
 * (Sec. 1).  Synchronising. */
int sp_trace_product_band(sp_ctx_t ctx, sp_hodlr_t M, int32_t b, const double* ab, int64_t ldab, double* out);

/* Sizes of a handle: order, tree depth L of the HODLR partition (Sec. 3.1.1,
 * Eq. (HODLR); n not a power of two is split by balanced bisection), largest
 * off-diagonal rank (the k of Table "complexity_HODLR") and device bytes held
 * (the memory of Sec. 3.2, at the rank capacity).  Synchronising. */
int sp_hodlr_info(sp_ctx_t ctx, sp_hodlr_t M, int64_t* n, int32_t* levels, int32_t* max_rank, size_t* bytes);
/* Releases a handle's device memory stream-ordered on the stream of the
 * context that created it (work already enqueued there completes first); call
 * it before that stream is destroyed. */
void sp_hodlr_destroy(sp_hodlr_t M);
/* Per-level ranks of a handle (the off-diagonal ranks whose growth with the
 * gap Sec. 3.2 bounds): for tree level l = 1..min(L, nlevels), max_rank[l-1]
 * and mean_rank[l-1] over the 2^l blocks of that level, and *nominal_bytes =
 * 8 * (sum of leaf sizes^2 + sum over blocks of (rows + cols) * rank), the
 * storage at the actual ranks.  Any output may be NULL.  Synchronising. */
int sp_hodlr_level_ranks(sp_ctx_t ctx, sp_hodlr_t M, int32_t nlevels, int32_t* max_rank, double* mean_rank,
                         double* nominal_bytes);

/* ---- formatted HODLR arithmetic (Table "complexity_HODLR") ---- */

/* C = alpha A + beta B + gamma I, recompressed at C's tolerance (A's). */
int sp_hodlr_add(sp_ctx_t ctx, double alpha, sp_hodlr_t A, double beta, sp_hodlr_t B, double gamma, sp_hodlr_t* C);
/* T = M^T (exact: leaves transposed, the U and V factors of sibling blocks
 * exchanged; Sec. 3.1.1).  Used for Q2^T in the QR-based step (Eq.
 * (qdwh_qr)). */
int sp_hodlr_transpose(sp_ctx_t ctx, sp_hodlr_t M, sp_hodlr_t* T);
/* C = A * B (formatted product, O(k^2 n log^2 n)). */
int sp_hodlr_mult(sp_ctx_t ctx, sp_hodlr_t A, sp_hodlr_t B, sp_hodlr_t* C);
/* Lower-triangular HODLR L with L L^T = Z (H-Cholesky of a symmetric
 * positive definite Z); SP_EBREAKDOWN on a non-positive leaf pivot. */
int sp_hodlr_cholesky(sp_ctx_t ctx, sp_hodlr_t Z, sp_hodlr_t* L);
/* X = op(L)^{-1} B for the lower-triangular HODLR L and a HODLR B (formatted
 * triangular solve); trans = 0: op(L) = L, trans = 1: op(L) = L^T. */
int sp_hodlr_trsm(sp_ctx_t ctx, sp_hodlr_t L, int trans, sp_hodlr_t B, sp_hodlr_t* X);

/* ---- parameter estimation (Sec. 5, Eq. (param_estimation)) ---- */

/* counts[i] = #{eigenvalues of A < shifts[i]} (inertia by LDL^T, Sylvester's
 * law; tridiagonal: Sturm recurrence).  ab, shifts: host or device;
 * counts: host.  Synchronising. */
int sp_inertia(sp_ctx_t ctx, int64_t n, int32_t b, const double* ab, int64_t ldab, int32_t nshift,
               const double* shifts, int64_t* counts);
/* Locates a shift mu with exactly nu eigenvalues below it, mu the midpoint of
 * the inertia brackets of lambda_nu and lambda_{nu+1}; also returns bounds
 * lam_nu_hi > lambda_nu and lam_nu1_lo <= lambda_{nu+1}.  Synchronising. */
int sp_locate_shift(sp_ctx_t ctx, int64_t n, int32_t b, const double* ab, int64_t ldab, int64_t nu, double* mu,
                    double* lam_nu_hi, double* lam_nu1_lo);
/* Inertia counts without any device allocation, for callers that cannot call
 * cudaMalloc: for example a host program that hands the whole GPU to its own
 * memory pool up front, or code that must not touch the CUDA allocator while
 * it runs.  The paper has no counterpart; it computes the same counts as
 * sp_inertia.
 *   ab (band, ldab >= b+1), shifts (nshift doubles) and counts (nshift
 *   int64) are DEVICE pointers owned by the caller.
 *   Scratch: a library-owned device array of SP_NOALLOC_SCRATCH_DOUBLES
 *   doubles (8 MiB), held by every GPU that loads the library until the
 *   process exits.  A call needs 520 + nshift * (b*b + b) doubles of it (b > 1;
 *   520 for b <= 1); larger requests return SP_EINVAL with a message.
 *   The first call on a device looks the array's device address up (with that
 *   device current) and caches it; make that first call before any CUDA stream
 *   capture.  Every call reuses the same array: calls whose work overlaps on the
 *   GPU (other streams, other threads) race on it and must be serialised by the
 *   caller.  Enqueues on the context stream; does not synchronise. */
#define SP_NOALLOC_SCRATCH_DOUBLES (1 << 20)
int sp_inertia_noalloc(sp_ctx_t ctx, int64_t n, int32_t b, const double* ab, int64_t ldab, int32_t nshift,
                       const double* shifts, int64_t* counts);

/* QDWH start: alpha >= ||A - mu I||_2 and l0 <= sigma_min((A - mu I)/alpha)
 * from inertia brackets of the extreme eigenvalues and of the eigenvalues
 * next to mu.  Synchronising. */
int sp_qdwh_start(sp_ctx_t ctx, int64_t n, int32_t b, const double* ab, int64_t ldab, double mu, double* alpha,
                  double* l0);

/* The paper's own start parameters (Sec. 5, Eq. (param_estimation)):
 * alpha = normest(A - mu I), the power method on (A - mu I)^T (A - mu I) from
 * the vector of absolute column sums, stopped at relative change <= 1e-6;
 * l0 = ||X0||_1 / (sqrt(n) condest(X0)) with X0 = (A - mu I)/alpha and
 * condest(X0) = ||X0||_1 est(||X0^{-1}||_1), est the 1-norm estimator of
 * Hager with Higham's refinements (at most 5 sign-vector iterations plus the
 * alternating-sign safeguard; the one-column case of Higham-Tisseur) using a
 * banded LU with partial pivoting.  Estimates, not bounds: alpha may fall
 * short of ||A - mu I||_2 and l0 may exceed sigma_min(X0).  To run QDWH with
 * them, pass them in sp_qdwh_opts.alpha / .l0.  iters (may be NULL) receives
 * {power iterations, LU solves}.  ab: host or device.  Synchronising;
 * SP_EBREAKDOWN if the LU meets an exactly zero pivot (A - mu I singular). */
int sp_qdwh_params_paper(sp_ctx_t ctx, int64_t n, int32_t b, const double* ab, int64_t ldab, double mu,
                         double* alpha, double* l0, int32_t* iters);

/* ---- autotuning (not in the paper; Sec. 6 fixes n_min by hand) ---- */

typedef struct {
  int32_t leaf;        /* chosen leaf size (the paper's n_min) */
  int32_t tsqr_chunk;  /* rows per TSQR chunk of the recompression QR */
  int32_t small_tiles; /* 1: small GEMMs laid out in 16 x 16 tiles */
  double ms;           /* time of one projector of the tuning problem with this choice */
  int32_t trials;      /* projectors timed (0: the answer came from the cache) */
  int64_t n_tuned;     /* order of the tuning problem (0 when cached) */
} sp_tune_result;

/* Chooses leaf size, TSQR chunk and GEMM tiling by timing whole projectors
 * (HODLR ingest, sign by hQDWH in the given precision mode, projector, trace)
 * of the leading min(n, 16384) block of the band at shift mu: every leaf in
 * {64, 128, 256, 512} with 2b <= leaf <= half the tuning order, then chunks of
 * 256 / 512 rows and small tiles on / off at the best leaf.  The result is
 * appended to cache_path (JSON lines keyed by floor(log2 n), b, precision; may
 * be NULL) and added to the context's table; a cache hit returns at once with
 * trials = 0.  ab: host or device.  Synchronising. */
int sp_autotune(sp_ctx_t ctx, int64_t n, int32_t b, const double* ab, int64_t ldab, double mu, double tol,
                int32_t precision, const char* cache_path, sp_tune_result* out);
/* Loads a tuning cache into the context's table (replacing it).  Afterwards
 * a leaf argument of 0 (sp_hodlr_from_band, sp_batched_projector) takes the
 * tuned leaf of the nearest size class with the same b, else the rule 64 /
 * 128 / 256 by n (at least 2b). */
int sp_ctx_load_tuning(sp_ctx_t ctx, const char* cache_path);
/* Sets the recompression's TSQR chunk rows (32..8192; default 512) and the
 * small-problem 16 x 16 GEMM tiling (default on) for the context's calls. */
int sp_ctx_set_tuning(sp_ctx_t ctx, int32_t tsqr_chunk, int32_t small_tiles);

/* ---- QR-based first iteration (Sec. 4, Algorithms 1/2, Remark "construct_off") ---- */

/* Givens rotations of the fast QR of [scale * A; I] for the banded A
 * (Algorithm 1 for b = 1, Algorithm 2 for b > 1), in the algorithm's order:
 * rotation t acts on the ordered row pair (p_t, q_t) (0-based rows of the
 * 2n x n stacked matrix) as [[c, s], [-s, c]] and annihilates the entry of
 * row q_t.  cs: device pointer to 2 * count doubles (c_0, s_0, c_1, s_1, ...),
 * count = (2b+1) n - b^2 - b.  ab: device pointer. */
int sp_givens_generate(sp_ctx_t ctx, int64_t n, int32_t b, const double* ab, int64_t ldab, double scale, double* cs);
/* Q1 and Q2 of [scale * A; I] = [Q1; Q2] R in HODLR format on A's tree
 * (Remark "construct_off", Theorems 4 and 6: off-diagonal ranks <= 2b).
 * Q2's blocks are returned recompressed (orthonormal V, U = Q Sigma, at A's
 * tolerance): the nested-basis factors can differ in scale by many orders of
 * magnitude for localised eigenvectors, which costs products accuracy. */
int sp_fastqr_factors(sp_ctx_t ctx, sp_hodlr_t A, double scale, sp_hodlr_t* Q1, sp_hodlr_t* Q2);

#ifdef __cplusplus
}
#endif
#endif /* SP_H */
