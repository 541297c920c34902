// sp_internal.h -- data structures shared by the library's translation units.
//
// HODLR layout in HBM (Sec. 3.1.1 of the paper, "HODLR matrices"):
//  * The index set [0, n) is split by balanced bisection (left child gets
//    ceil(m/2)) into a complete binary tree of depth L; heap numbering, root 1,
//    children 2c and 2c+1, level l holds nodes 2^l .. 2^(l+1)-1.  Leaves sit at
//    level L and hold at most leaf_max indices.
//  * Every non-root node c owns the off-diagonal block B_c = M(I_c, I_sib(c))
//    = U_c V_c^T of rank rank[c] <= cap.  For level l the U factors of all
//    level-l nodes live in one n x cap column-major array (ld = n): rows I_c
//    hold U_c.  The V factor of B_c lives in the level's V array at rows
//    I_sib(c).  So a block's factors are two row-slices of level arrays, and a
//    row range of a level array is "the factor of the block whose rows (or
//    columns) are that range".
//  * Leaves are dense leaf_max x leaf_max column-major slots (ld = leaf_max).
//  * Columns of U_c/V_c beyond rank[c] are kept zero, so a kernel that reads a
//    capacity-wide slice still computes the right product.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "sp.h"

namespace sp {

// Device memory source of a context: the caller's stream-ordered callbacks
// (sp_ctx_create) or, when both are null, the device's default memory pool
// (cudaMallocAsync / cudaFreeAsync).
struct Allocator {
  sp_alloc_fn alloc = nullptr;
  sp_free_fn free = nullptr;
  void* user = nullptr;
  bool custom() const { return alloc != nullptr; }
};

struct Tree {
  cudaStream_t stream = nullptr;  // stream its device arrays were allocated on
  int64_t n = 0;
  int L = 0;         // depth; leaves at level L
  int leaf_max = 0;  // largest leaf size
  std::vector<int64_t> lo, sz;  // per heap node (index 0 unused)
  int64_t* d_lo = nullptr;      // device copies
  int64_t* d_sz = nullptr;
  ~Tree();
  int nodes() const { return 1 << (L + 1); }
  int nleaves() const { return 1 << L; }
  static int level_of(int c) { return 31 - __builtin_clz((unsigned)c); }
};

std::shared_ptr<Tree> make_tree(int64_t n, int leaf, cudaStream_t stream);
// Two HODLR matrices can be combined when their partitions coincide.
inline bool same_tree(const Tree& a, const Tree& b) { return a.n == b.n && a.L == b.L && a.lo == b.lo; }

}  // namespace sp

struct sp_hodlr {
  std::shared_ptr<sp::Tree> tree;
  cudaStream_t stream = nullptr;  // allocation stream: buffers are freed stream-ordered on it
  int cap = 0;
  double tol = 0.0;
  int leaf_ld = 0;
  double* leaves = nullptr;  // nleaves * leaf_ld^2
  double* U = nullptr;       // L * n * cap
  double* V = nullptr;       // L * n * cap
  int* rank = nullptr;       // device, tree->nodes() ints
  // band of the source matrix (kept by sp_hodlr_from_band for the QR step)
  double* band = nullptr;
  int b = 0;
  double mu = 0.0;
  size_t bytes = 0;
  int64_t n() const { return tree->n; }
  int L() const { return tree->L; }
  double* Ul(int l) const { return U + (size_t)(l - 1) * (size_t)tree->n * (size_t)cap; }
  double* Vl(int l) const { return V + (size_t)(l - 1) * (size_t)tree->n * (size_t)cap; }
  double* leaf(int j) const { return leaves + (size_t)j * (size_t)leaf_ld * (size_t)leaf_ld; }
  // block B_c factors
  double* Uc(int c) const { return Ul(sp::Tree::level_of(c)) + tree->lo[c]; }
  double* Vc(int c) const { return Vl(sp::Tree::level_of(c)) + tree->lo[c ^ 1]; }
};

namespace sp {
// Kernel families timed and flop-counted by the profiler.
enum KernelId {
  KID_GEMM = 0, KID_QR, KID_APPLYQ, KID_CORE_SVD, KID_GATHER, KID_POTRF, KID_LEAF_INV, KID_GIVENS, KID_REPLAY_LEAF,
  KID_REPLAY_TRACK, KID_INERTIA, KID_MISC, KID_GEMM_APPLY, KID_GEMM_CHOL, KID_GEMM_MULT, KID_GEMM_F32, KID_LEAF_CLUSTER, KID_HOST_WAIT,
  KID_COUNT
};
}  // namespace sp

struct sp_ctx {
  cudaStream_t stream = nullptr;
  int device = 0;
  sp::Allocator alloc;     // where every device buffer of this context comes from
  int num_sms = 152;
  std::string err;
  int* d_flags = nullptr;  // [0] rank overflow, [1] breakdown, [2] non-finite, [3] timeout
  double flops = 0.0;      // nominal flops of enqueued task lists
  // profiler: CUDA events around every launch of a kernel family, and the
  // algorithmic flops the kernels count themselves (d_fc[kid])
  bool profiling = false;
  int gemm_kid = sp::KID_GEMM;  // profiler bucket of k_gemm launches (call site)
  bool gemm_fp32 = false;       // mixed-precision scope: GEMMs on the tensor cores
  // tunables (sp_ctx_set_tuning / sp_autotune): rows per TSQR chunk of the
  // recompression (at least twice the stacked width), small-problem 16 x 16
  // GEMM tiles on/off, and the tuned leaf sizes by (log2 n, b, precision)
  int tsqr_chunk = 512;
  bool small_tiles = true;
  struct TunedLeaf {
    int nbucket, b, precision, leaf, tsqr_chunk, small_tiles;
  };
  std::vector<TunedLeaf> tuned;
  double* d_fc = nullptr;
  double fc_host[sp::KID_COUNT] = {};  // flops folded in from batched workers' contexts
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[sp::KID_COUNT];
  int64_t launches[sp::KID_COUNT] = {};
  double ms[sp::KID_COUNT] = {};
  // H-Cholesky nodes: events bracketing each node's own work (not its
  // children's), folded into per-tree-level self times when read
  struct NodeEvents {
    int level;
    int nev;
    cudaEvent_t e[5];
  };
  std::vector<NodeEvents> chol_ev;
  double chol_level_ms[64] = {};
};

namespace sp {

enum Flag { FLAG_RANK = 0, FLAG_BREAKDOWN = 1, FLAG_NONFINITE = 2, FLAG_TIMEOUT = 3, NFLAGS = 8 };

// ------------------------------------------------------------------ errors --
struct Error {
  int code;
  std::string msg;
};
[[noreturn]] void fail(int code, const std::string& msg);
void check_cuda(cudaError_t e, const char* what);
void check_launch(const char* what);

// Process-wide count of kernel launches made by the library.
int64_t launch_count();

// Brackets one launch of a kernel family with CUDA events when profiling.
struct ProfScope {
  sp_ctx* ctx;
  int kid;
  cudaEvent_t a = nullptr;
  ProfScope(sp_ctx* c, int k);
  ~ProfScope();
};
// Routes the k_gemm launches of a scope to a call-site bucket of the profiler.
struct GemmSite {
  sp_ctx* ctx;
  int prev;
  GemmSite(sp_ctx* c, int kid) : ctx(c), prev(c->gemm_kid) { ctx->gemm_kid = kid; }
  ~GemmSite() { ctx->gemm_kid = prev; }
};
// Binary32 GEMM arithmetic inside a scope (mixed-precision steps).
struct Fp32Gemms {
  sp_ctx* ctx;
  bool prev;
  explicit Fp32Gemms(sp_ctx* c) : ctx(c), prev(c->gemm_fp32) { ctx->gemm_fp32 = true; }
  ~Fp32Gemms() { ctx->gemm_fp32 = prev; }
};
// Device flop counter of a family (null unless profiling).
inline double* fc_ptr(sp_ctx* ctx, int kid) { return ctx->profiling ? ctx->d_fc + kid : nullptr; }

// ------------------------------------------------------------------ memory --
// Stream-ordered device buffer (freed on the context stream when destroyed).
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t st = nullptr;
  DBuf() = default;
  DBuf(size_t b, cudaStream_t s);
  ~DBuf();
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), bytes(o.bytes), st(o.st) { o.p = nullptr; }
  DBuf& operator=(DBuf&& o) noexcept;
  template <class T> T* as() const { return static_cast<T*>(p); }
};
// Allocations go through the allocator of the context whose entry point is
// running on this thread (AllocScope, set by every entry point); frees find
// the allocator that made the buffer.
void* dmalloc(size_t bytes, cudaStream_t st);
struct AllocScope {
  const Allocator* prev;
  explicit AllocScope(const Allocator* a);
  ~AllocScope();
};
// Dynamic shared memory above the 48 KB default.  Each kernel that may need
// it gets its limit raised once per device, to the opt-in maximum, when the
// first context on that device is created (configure_*_kernels), before any
// worker thread launches anything: changing a kernel's attribute while another
// host thread launches the same kernel made those launches fail.  Launch sites
// only check their need against the limit (ensure_dynamic_smem, SP_EINVAL).
void configure_dynamic_smem(const void* func);
void ensure_dynamic_smem(const void* func, size_t bytes);
void configure_blas_kernels();
void configure_lowrank_kernels();
void configure_param_kernels();
void dfree(void* p, cudaStream_t st);
// Copies a host array into a fresh device buffer on the stream.
template <class T>
DBuf upload(const std::vector<T>& v, cudaStream_t st) {
  DBuf b(v.size() * sizeof(T) + 16, st);
  if (!v.empty()) check_cuda(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st), "upload");
  return b;
}

// ------------------------------------------------------------- batched GEMM --
// C = alpha * op(A) op(B) + beta * C for a list of problems.  Sizes are static
// upper bounds; a non-null pm/pn/pk points to a device int whose value (capped
// by the static bound) is the actual size.  op = transpose when the launch's
// ta/tb flag is set.  With atomic = true the tile result alpha*AB is added to C
// with atomics (C must already hold beta*C); used for split-k and for
// accumulating several products into one output.
struct GemmTask {
  const double* A;
  const double* B;
  double* C;
  int64_t lda, ldb, ldc;
  int m, n, k;
  const int* pm;
  const int* pn;
  const int* pk;
  double alpha, beta;
  double* W;  // split-k partial tiles (set by gemm_batched)
  int nsplit = 0;  // reduction: number of W slots of this task (0: from k and the launch's k chunk)
};
void gemm_batched(sp_ctx* ctx, bool ta, bool tb, const std::vector<GemmTask>& tasks, int ksplit = 0);
// Split-BF16 tensor-core GEMM of the mixed-precision scope (sp_tc.cu): tiles of
// gemm_tc_tile_rows() x gemm_tc_tile_cols(), gemm_tc_smem() bytes of dynamic
// shared memory per CTA; split = 1 writes k-chunk partials to the tasks' W.
size_t gemm_tc_smem();
int gemm_tc_tile_rows();
int gemm_tc_tile_cols();
void launch_gemm_tc(sp_ctx* ctx, bool ta, bool tb, dim3 grid, const GemmTask* tasks, int kchunk, int split,
                    double* fc);
void configure_tc_kernels();
inline GemmTask gt(const double* A, int64_t lda, const double* B, int64_t ldb, double* C, int64_t ldc, int m, int n,
                   int k, double alpha, double beta, const int* pm = nullptr, const int* pn = nullptr,
                   const int* pk = nullptr) {
  return GemmTask{A, B, C, lda, ldb, ldc, m, n, k, pm, pn, pk, alpha, beta, nullptr};
}

// ------------------------------------------------------------ small kernels --
// Y = a X + b Y over m x n strided blocks (optionally + g on the diagonal, and
// sizes capped by device ints); with b == 0, Y is not read.
struct AxpbyTask {
  const double* X;
  double* Y;
  int64_t ldx, ldy;
  int m, n;
  const int* pm;
  const int* pn;
  double a, b, g;
};
void axpby_batched(sp_ctx* ctx, const std::vector<AxpbyTask>& tasks);
// Zero columns [rank, cap) of m-row slices (keeps factor arrays clean).
struct ZeroTailTask {
  double* P;
  int64_t ld;
  int m;
  const int* prank;
  int cap;
};
void zero_tail_batched(sp_ctx* ctx, const std::vector<ZeroTailTask>& tasks);

// Dense leaf kernels (one CTA per task).
struct LeafTask {
  double* A;  // leaf (n x n), ld
  int64_t lda;
  int n;
  double* X;  // right-hand side (n x w) for trsm
  int64_t ldx;
  int w;
  const int* pw;
};
// In-place lower Cholesky of each leaf (upper triangle zeroed); sets the
// breakdown flag on a non-positive pivot.
void leaf_potrf(sp_ctx* ctx, const std::vector<LeafTask>& tasks);
// Cholesky factor (in place, upper triangle zeroed) and its inverse (into X)
// of each leaf in one cluster kernel; returns false, doing nothing, when a
// leaf is too large for it (n > 256) or X is missing.
bool leaf_chol_inv(sp_ctx* ctx, const std::vector<LeafTask>& tasks);
// X <- L^{-1} (the whole n x n inverse) for lower-triangular leaves, n <= 1024.
void leaf_inverse_batched(sp_ctx* ctx, const std::vector<LeafTask>& tasks);
// Sets the context's non-finite flag if any of the `count` doubles at p is
// NaN or infinite (enqueued, no synchronisation).
void check_finite(sp_ctx* ctx, const double* p, size_t count);

// --------------------------------------------------------- recompression ----
// A block given as a sum of products sum_s scale_s U_s V_s^T (U_s: m x w_s,
// V_s: q x w_s) is recompressed to U V^T with the singular values > tol of
// the sum kept: an absolute threshold on the singular values, applied after
// every formatted operation (Sec. 3.1.1; Sec. 5).  Stacked factors are
// orthogonalised by Householder QR (tall blocks by a binary TSQR tree), the
// r_U x r_V core R_U R_V^T is diagonalised by a one-sided Jacobi SVD.
struct Seg {
  const double* U;
  const double* V;
  int64_t ldu, ldv;
  int w;           // static width bound
  const int* pw;   // device width (capped by w) or null
  double scale;    // multiplies V_s
};
struct LrBlock {
  int m, q;              // rows of U side, rows of V side
  std::vector<Seg> segs;
  double* Uout;          // m x cap (ld ldu_out)
  double* Vout;          // q x cap
  int64_t ldu_out, ldv_out;
  int* rank_out;         // device int
  int cap;
};
void recompress(sp_ctx* ctx, const std::vector<LrBlock>& blocks, double tol);

// ------------------------------------------------------------- HODLR ops ----
sp_hodlr* hodlr_alloc(sp_ctx* ctx, std::shared_ptr<Tree> tree, int cap, double tol);
void hodlr_free(sp_hodlr* M);
void hodlr_copy(sp_ctx* ctx, const sp_hodlr* S, sp_hodlr* D);
void hodlr_set_zero(sp_ctx* ctx, sp_hodlr* M);
std::vector<int> host_ranks(sp_ctx* ctx, const sp_hodlr* M);

// Y(I_c) (+)= op(M_sub(c)) X(I_c) for every node c of level `lev` (lev = 0:
// the whole matrix).  X, Y: n x w column-major (ld n); the width of rows I_c
// is *pw[c] if pw is given (device int array indexed by heap node) else w.
// trans: use M^T.  accumulate: add to Y instead of overwriting it.
void hodlr_apply_level(sp_ctx* ctx, const sp_hodlr* M, int lev, const double* X, int64_t ldx, double* Y,
                       int64_t ldy, int w, const int* pw_node, bool trans, bool accumulate);

// Same restricted to the subtree of node c (X, Y point at row lo[c]).
void hodlr_apply_sub(sp_ctx* ctx, const sp_hodlr* M, int c, const double* X, int64_t ldx, double* Y, int64_t ldy,
                     int w, const int* pw, bool trans, bool accumulate);

sp_hodlr* hodlr_from_band(sp_ctx* ctx, int64_t n, int b, const double* ab_dev, int64_t ldab, double mu, int leaf,
                          double tol, int cap);
void hodlr_to_dense(sp_ctx* ctx, const sp_hodlr* M, int64_t row0, int64_t nrows, double* out, int64_t ld);
double hodlr_trace(sp_ctx* ctx, const sp_hodlr* M);
// symmetric = true: the caller knows the result is symmetric (up to rounding
// and truncation); only the left child of every sibling pair is recompressed,
// the right one is its transpose (half the recompression work), and the
// leaves are symmetrised.
sp_hodlr* hodlr_add(sp_ctx* ctx, double alpha, const sp_hodlr* A, double beta, const sp_hodlr* B, double gamma,
                    bool symmetric = false);
sp_hodlr* hodlr_mult(sp_ctx* ctx, const sp_hodlr* A, const sp_hodlr* B, bool symmetric = false);
sp_hodlr* hodlr_cholesky(sp_ctx* ctx, const sp_hodlr* Z);
// H-Cholesky returning both the factor L and its HODLR inverse L^{-1}.
void hodlr_cholesky_inv(sp_ctx* ctx, const sp_hodlr* Z, sp_hodlr** L, sp_hodlr** Li);
sp_hodlr* hodlr_tri_inverse(sp_ctx* ctx, const sp_hodlr* L);
sp_hodlr* hodlr_trsm(sp_ctx* ctx, const sp_hodlr* L, bool trans, const sp_hodlr* B);
sp_hodlr* hodlr_transpose(sp_ctx* ctx, const sp_hodlr* M);

// Inertia counts and the QR-based first step.
void inertia_counts(sp_ctx* ctx, int64_t n, int b, const double* ab_dev, int64_t ldab, int nshift,
                    const double* shifts_dev, int64_t* counts_dev);
void givens_generate(sp_ctx* ctx, int64_t n, int b, const double* ab_dev, int64_t ldab, double mu, double scale,
                     double* cs_dev);
void fastqr_factors(sp_ctx* ctx, const sp_hodlr* A, double scale, sp_hodlr** Q1, sp_hodlr** Q2);

int64_t givens_count(int64_t n, int b);

}  // namespace sp
