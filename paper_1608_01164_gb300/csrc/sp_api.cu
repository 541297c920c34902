// sp_api.cu -- the C ABI (include/sp.h) and the hQDWH driver (Algorithm 3).
//
// hQDWH for sign(A - mu I) (Sec. 5, Algorithm 3):
//   alpha, l0 from inertia brackets (reading of Eq. (param_estimation));
//   X_0 = (A - mu I)/alpha in HODLR (exact: off-diagonal rank b);
//   k = 0: QR-based step from the Givens rotations of Algorithm 1/2:
//          X_1 = (b/c) X_0 + (1/sqrt c)(a - b/c) Q1 Q2^T        (Eq. (qdwh_qr))
//   k >= 1: Cholesky-based steps:
//          Z = I + c X^2,  L L^T = Z (H-Cholesky),
//          X <- (b/c) X + (a - b/c) L^{-T} L^{-1} X              (Eq. (qdwh_chol2))
//          (the paper's (X W^{-1}) W^{-*} with W = L^T, evaluated as two
//          formatted left solves since X and Z commute and are symmetric)
//   stop when |1 - l_k| <= delta; P = (I - X)/2.
// Mixed precision (not in the paper): late Cholesky steps in residual form
// with binary32 GEMMs (SP_MIXED_FP32), or late steps replaced by residual
// Newton-Schulz steps (SP_MIXED_NS); binary64 polish at the end.
// The iteration count depends only on the scalars, so the host runs the
// scalar recurrence and every matrix operation stays on the device.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <atomic>
#include <mutex>
#include <new>
#include <numeric>
#include <thread>

#include "sp_internal.h"

namespace sp {
void gershgorin(sp_ctx* ctx, int64_t n, int b, const double* ab_dev, int64_t ldab, double* lo, double* hi);
void locate_shift(sp_ctx* ctx, int64_t n, int b, const double* ab_dev, int64_t ldab, int64_t nu, double* mu,
                  double* lam_nu_hi, double* lam_nu1_lo);
void qdwh_start(sp_ctx* ctx, int64_t n, int b, const double* ab_dev, int64_t ldab, double mu, double* alpha,
                double* l0);
void qdwh_params_paper(sp_ctx* ctx, int64_t n, int b, const double* ab_dev, int64_t ldab, double mu, double* alpha,
                       double* l0, int* iters);
void hodlr_scale_shift(sp_ctx* ctx, sp_hodlr* M, double alpha, double gamma);
void inertia_counts_noalloc(sp_ctx* ctx, int64_t n, int b, const double* ab_dev, int64_t ldab, int nshift,
                            const double* shifts_dev, int64_t* counts_dev);
int hodlr_max_rank(sp_ctx* ctx, const sp_hodlr* M);
int tuned_leaf(sp_ctx* ctx, int64_t n, int b);
void hodlr_level_stats(sp_ctx* ctx, const sp_hodlr* M, int nlevels, int* max_rank, double* mean_rank,
                       double* nominal_bytes);
void hodlr_check_finite(sp_ctx* ctx, const sp_hodlr* M);
double hodlr_trace_band(sp_ctx* ctx, const sp_hodlr* M, int b, const double* ab_dev, int64_t ldab);

namespace {

// iterations with 1 - l_k^2 <= this take the mixed-precision residual step
constexpr double kMixedThreshold = 1e-2;

template <class F>
int guarded(sp_ctx* ctx, F&& f) {
  // device buffers made while the call runs come from the context's allocator
  AllocScope scope(ctx ? &ctx->alloc : nullptr);
  try {
    f();
    return SP_OK;
  } catch (const Error& e) {
    if (ctx) ctx->err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    if (ctx) ctx->err = "host allocation failed";
    return SP_ENOMEM;
  } catch (const std::exception& e) {
    if (ctx) ctx->err = e.what();
    return SP_EINTERNAL;
  }
}

bool is_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device copy of a band given as host or device pointer, repacked with
// ldab = b+1.
DBuf band_on_device(sp_ctx* ctx, int64_t n, int b, const double* ab, int64_t ldab) {
  DBuf d((size_t)(b + 1) * n * sizeof(double), ctx->stream);
  const cudaMemcpyKind kind = is_device(ab) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  check_cuda(cudaMemcpy2DAsync(d.p, sizeof(double) * (b + 1), ab, sizeof(double) * ldab, sizeof(double) * (b + 1), n,
                               kind, ctx->stream),
             "band upload");
  return d;
}

int read_flags(sp_ctx* ctx) {
  int h[NFLAGS];
  check_cuda(cudaMemcpyAsync(h, ctx->d_flags, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream), "flags");
  const auto t0 = std::chrono::steady_clock::now();
  check_cuda(cudaStreamSynchronize(ctx->stream), "sync");
  if (ctx->profiling) {
    // host time blocked here: the device was still busy with enqueued work
    ctx->ms[KID_HOST_WAIT] += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    ctx->launches[KID_HOST_WAIT] += 1;
  }
  if (h[FLAG_RANK]) return SP_ERANK;
  if (h[FLAG_BREAKDOWN]) return SP_EBREAKDOWN;
  if (h[FLAG_NONFINITE]) return SP_ENONFINITE;
  if (h[FLAG_TIMEOUT]) return SP_ETIMEOUT;
  return SP_OK;
}

void check_flags(sp_ctx* ctx, const char* where) {
  const int f = read_flags(ctx);
  if (f != SP_OK) {
    check_cuda(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int) * NFLAGS, ctx->stream), "flags reset");
    const char* what = f == SP_ERANK ? "rank capacity exceeded" : f == SP_EBREAKDOWN ? "H-Cholesky breakdown"
                                                              : f == SP_ENONFINITE ? "non-finite value"
                                                                                   : "device wait timed out";
    fail(f, std::string(what) + " in " + where);
  }
}

struct Owned {
  sp_hodlr* p = nullptr;
  explicit Owned(sp_hodlr* q = nullptr) : p(q) {}
  ~Owned() { hodlr_free(p); }
  Owned(const Owned&) = delete;
  Owned& operator=(const Owned&) = delete;
  void reset(sp_hodlr* q) {
    hodlr_free(p);
    p = q;
  }
  sp_hodlr* release() {
    sp_hodlr* q = p;
    p = nullptr;
    return q;
  }
};

struct Timer {
  cudaEvent_t a, b;
  cudaStream_t st;
  explicit Timer(cudaStream_t s) : st(s) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
  }
  double stop() {
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

// one Cholesky-based QDWH step: X <- (b/c) X + (a - b/c) Z^{-1} X, Z = I + c X^2,
// with Z = L L^T and Z^{-1} X = L^{-T} (L^{-1} X) as two formatted products with
// the HODLR inverse factor built during the factorisation.
sp_hodlr* chol_step(sp_ctx* ctx, const sp_hodlr* X, double a, double b, double c, sp_info* inf) {
  Timer t1(ctx->stream);
  Owned Z(hodlr_mult(ctx, X, X, true));
  hodlr_scale_shift(ctx, Z.p, c, 1.0);
  inf->ms_mult += t1.stop();
  Timer t2(ctx->stream);
  sp_hodlr *lf = nullptr, *li = nullptr;
  hodlr_cholesky_inv(ctx, Z.p, &lf, &li);
  Owned Lf(lf), Li(li);
  Z.reset(nullptr);
  Lf.reset(nullptr);
  inf->ms_factor += t2.stop();
  Timer t3(ctx->stream);
  Owned Y(hodlr_mult(ctx, Li.p, X));
  Owned LiT(hodlr_transpose(ctx, Li.p));
  Li.reset(nullptr);
  Owned V(hodlr_mult(ctx, LiT.p, Y.p, true));
  Y.reset(nullptr);
  LiT.reset(nullptr);
  inf->ms_solve += t3.stop();
  Timer t4(ctx->stream);
  Owned Xn(hodlr_add(ctx, b / c, X, a - b / c, V.p, 0.0, true));
  V.reset(nullptr);
  inf->ms_combine += t4.stop();
  return Xn.release();
}

// Mixed-precision Cholesky-based step in residual form (for iterations whose
// lower bound l_k has 1 - l_k^2 small):  f(x) - x = (a-1) x (1-x^2)/(1+c x^2)
// (b - c = 1 - a), so
//   X+ = X + (a - 1) X Z^{-1} R,   R = I - X^2,  Z = I + c X^2,
// with R and the final sum in binary64 and the factorisation, the two
// products with the inverse factor and X * (Z^{-1} R) using binary32 GEMM
// arithmetic (recompression stays binary64).  The binary32 error multiplies
// ||R|| ~ 1 - l_k^2 instead of ||X|| ~ 1.
sp_hodlr* mixed_step(sp_ctx* ctx, const sp_hodlr* X, double a, double c, sp_info* inf) {
  Timer t1(ctx->stream);
  Owned Z(hodlr_mult(ctx, X, X, true));
  Owned R(hodlr_add(ctx, -1.0, Z.p, 0.0, nullptr, 1.0, true));
  hodlr_scale_shift(ctx, Z.p, c, 1.0);
  inf->ms_mult += t1.stop();
  Owned D(nullptr);
  {
    Fp32Gemms fp32(ctx);
    Timer t2(ctx->stream);
    sp_hodlr *lf = nullptr, *li = nullptr;
    hodlr_cholesky_inv(ctx, Z.p, &lf, &li);
    Owned Lf(lf), Li(li);
    Z.reset(nullptr);
    Lf.reset(nullptr);
    inf->ms_factor += t2.stop();
    Timer t3(ctx->stream);
    Owned Y(hodlr_mult(ctx, Li.p, R.p));
    Owned LiT(hodlr_transpose(ctx, Li.p));
    Li.reset(nullptr);
    Owned W(hodlr_mult(ctx, LiT.p, Y.p, true));
    Y.reset(nullptr);
    D.reset(hodlr_mult(ctx, X, W.p, true));
    inf->ms_solve += t3.stop();
  }
  Timer t4(ctx->stream);
  Owned Xn(hodlr_add(ctx, 1.0, X, a - 1.0, D.p, 0.0, true));
  D.reset(nullptr);
  inf->ms_combine += t4.stop();
  return Xn.release();
}

// Binary64 Newton-Schulz step for the sign function in residual form:
// X <- X + X (I - X^2) / 2  (= X (3I - X^2)/2).
sp_hodlr* newton_schulz_step(sp_ctx* ctx, const sp_hodlr* X) {
  Owned XX(hodlr_mult(ctx, X, X, true));
  Owned R(hodlr_add(ctx, -1.0, XX.p, 0.0, nullptr, 1.0, true));
  XX.reset(nullptr);
  Owned D(hodlr_mult(ctx, X, R.p, true));
  R.reset(nullptr);
  Owned Xn(hodlr_add(ctx, 1.0, X, 0.5, D.p, 0.0, true));
  return Xn.release();
}

// Newton-Schulz step in residual form with the correction product in binary32
// GEMM arithmetic: R = I - X^2 (binary64), D = X R (binary32 GEMMs, binary64
// storage and recompression), X <- X + D/2 (binary64).  The binary32 rounding
// error scales with ||R||, which the iteration drives to zero.
sp_hodlr* newton_schulz_step_mixed(sp_ctx* ctx, const sp_hodlr* X, sp_info* inf) {
  Timer t1(ctx->stream);
  Owned XX(hodlr_mult(ctx, X, X, true));
  Owned R(hodlr_add(ctx, -1.0, XX.p, 0.0, nullptr, 1.0, true));
  XX.reset(nullptr);
  inf->ms_mult += t1.stop();
  Owned D(nullptr);
  {
    Fp32Gemms fp32(ctx);
    Timer t2(ctx->stream);
    D.reset(hodlr_mult(ctx, X, R.p, true));
    inf->ms_solve += t2.stop();
  }
  R.reset(nullptr);
  Timer t3(ctx->stream);
  Owned Xn(hodlr_add(ctx, 1.0, X, 0.5, D.p, 0.0, true));
  D.reset(nullptr);
  inf->ms_combine += t3.stop();
  return Xn.release();
}

// QR-based first step on the band kept by A (A = A - mu I in HODLR)
sp_hodlr* qr_step(sp_ctx* ctx, const sp_hodlr* A, double alpha, double a, double b, double c) {
  const double sc = std::sqrt(c);
  sp_hodlr *q1 = nullptr, *q2 = nullptr;
  fastqr_factors(ctx, A, sc / alpha, &q1, &q2);
  Owned Q1(q1), Q2(q2);
  Owned Q2t(hodlr_transpose(ctx, Q2.p));
  Q2.reset(nullptr);
  Owned P(hodlr_mult(ctx, Q1.p, Q2t.p, true));
  Q1.reset(nullptr);
  Q2t.reset(nullptr);
  Owned X1(hodlr_add(ctx, (b / c) / alpha, A, (a - b / c) / sc, P.p, 0.0, true));
  return X1.release();
}

}  // namespace
}  // namespace sp

using namespace sp;

extern "C" {

void sp_qdwh_opts_default(sp_qdwh_opts* o) {
  if (!o) return;
  o->max_iter = 10;
  o->delta = 1e-15;
  o->precision = SP_FP64;
  o->polish_steps = 1;
  o->alpha = 0.0;
  o->l0 = 0.0;
  o->qr_steps = 1;
}

int sp_ctx_create(void* cuda_stream, sp_alloc_fn alloc, sp_free_fn free_fn, void* user, sp_ctx_t* out) {
  if (!out || (alloc == nullptr) != (free_fn == nullptr)) return SP_EINVAL;
  auto* ctx = new (std::nothrow) sp_ctx;
  if (!ctx) return SP_ENOMEM;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  ctx->alloc.alloc = alloc;
  ctx->alloc.free = free_fn;
  ctx->alloc.user = user;
  const int rc = guarded(ctx, [&] {
    check_cuda(cudaGetDevice(&ctx->device), "cudaGetDevice");
    check_cuda(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device), "attr");
    ctx->d_flags = static_cast<int*>(dmalloc(sizeof(int) * NFLAGS, ctx->stream));
    check_cuda(cudaMemsetAsync(ctx->d_flags, 0, sizeof(int) * NFLAGS, ctx->stream), "flags");
    check_cuda(cudaStreamSynchronize(ctx->stream), "sync");
    {
      static std::mutex mu;
      static bool configured[64] = {};
      std::lock_guard<std::mutex> lock(mu);
      if (ctx->device >= 0 && ctx->device < 64 && !configured[ctx->device]) {
        configure_blas_kernels();
        configure_lowrank_kernels();
        configure_param_kernels();
        configure_tc_kernels();
        configured[ctx->device] = true;
      }
    }
    // Every formatted operation allocates and frees its temporaries in stream
    // order from the device's default pool.  Keep freed memory in the pool
    // across synchronisations (the default threshold 0 hands it back to the
    // driver at every sync, and the next step maps it again).  Per process.
    if (!ctx->alloc.custom()) {
      cudaMemPool_t pool;
      check_cuda(cudaDeviceGetDefaultMemPool(&pool, ctx->device), "default mem pool");
      uint64_t keep = UINT64_MAX;
      check_cuda(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep), "mem pool threshold");
    }
  });
  if (rc != SP_OK) {
    if (ctx->d_flags) dfree(ctx->d_flags, ctx->stream);
    delete ctx;
    return rc;
  }
  *out = ctx;
  return SP_OK;
}

void sp_ctx_destroy(sp_ctx_t ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  dfree(ctx->d_flags, ctx->stream);
  dfree(ctx->d_fc, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  for (int k = 0; k < KID_COUNT; ++k)
    for (auto& e : ctx->ev[k]) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
  for (auto& ne : ctx->chol_ev)
    for (int k = 0; k < ne.nev; ++k) cudaEventDestroy(ne.e[k]);
  delete ctx;
}

const char* sp_last_error(sp_ctx_t ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int sp_ctx_sync(sp_ctx_t ctx) {
  if (!ctx) return SP_EINVAL;
  return guarded(ctx, [&] { check_flags(ctx, "enqueued work"); });
}

int sp_ctx_set_profiling(sp_ctx_t ctx, int on) {
  if (!ctx) return SP_EINVAL;
  return guarded(ctx, [&] {
    check_cuda(cudaStreamSynchronize(ctx->stream), "sync");
    if (!ctx->d_fc) ctx->d_fc = static_cast<double*>(dmalloc(sizeof(double) * KID_COUNT, ctx->stream));
    check_cuda(cudaMemsetAsync(ctx->d_fc, 0, sizeof(double) * KID_COUNT, ctx->stream), "profiler counters");
    check_cuda(cudaStreamSynchronize(ctx->stream), "sync");
    for (int k = 0; k < KID_COUNT; ++k) {
      for (auto& e : ctx->ev[k]) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
      }
      ctx->ev[k].clear();
      ctx->launches[k] = 0;
      ctx->ms[k] = 0.0;
      ctx->fc_host[k] = 0.0;
    }
    for (auto& ne : ctx->chol_ev)
      for (int k = 0; k < ne.nev; ++k) cudaEventDestroy(ne.e[k]);
    ctx->chol_ev.clear();
    for (double& v : ctx->chol_level_ms) v = 0.0;
    ctx->profiling = on != 0;
  });
}

int sp_ctx_profile(sp_ctx_t ctx, int kernel, int64_t* launches, double* ms, double* flops) {
  if (!ctx || kernel < 0 || kernel >= KID_COUNT) return SP_EINVAL;
  return guarded(ctx, [&] {
    check_cuda(cudaStreamSynchronize(ctx->stream), "sync");
    for (int k = 0; k < KID_COUNT; ++k) {
      for (auto& e : ctx->ev[k]) {
        float t = 0.f;
        check_cuda(cudaEventElapsedTime(&t, e.first, e.second), "event time");
        ctx->ms[k] += t;
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
      }
      ctx->ev[k].clear();
    }
    double h[KID_COUNT] = {};
    if (ctx->d_fc) {
      check_cuda(cudaMemcpyAsync(h, ctx->d_fc, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream), "profiler counters");
      check_cuda(cudaStreamSynchronize(ctx->stream), "sync");
    }
    if (launches) *launches = ctx->launches[kernel];
    if (ms) *ms = ctx->ms[kernel];
    if (flops) *flops = h[kernel] + ctx->fc_host[kernel];
  });
}

int sp_ctx_profile_levels(sp_ctx_t ctx, int nlevels, double* ms_self) {
  if (!ctx || nlevels < 0 || (nlevels > 0 && !ms_self)) return SP_EINVAL;
  return guarded(ctx, [&] {
    check_cuda(cudaStreamSynchronize(ctx->stream), "sync");
    for (auto& ne : ctx->chol_ev) {
      float a = 0.f, b = 0.f;
      if (ne.nev == 2) {
        check_cuda(cudaEventElapsedTime(&a, ne.e[0], ne.e[1]), "event time");
      } else if (ne.nev == 5) {
        check_cuda(cudaEventElapsedTime(&a, ne.e[1], ne.e[2]), "event time");
        check_cuda(cudaEventElapsedTime(&b, ne.e[3], ne.e[4]), "event time");
      }
      if (ne.level >= 0 && ne.level < 64) ctx->chol_level_ms[ne.level] += (double)a + (double)b;
      for (int k = 0; k < ne.nev; ++k) cudaEventDestroy(ne.e[k]);
    }
    ctx->chol_ev.clear();
    for (int l = 0; l < nlevels; ++l) ms_self[l] = l < 64 ? ctx->chol_level_ms[l] : 0.0;
  });
}

const char* sp_kernel_name(int kernel) {
  static const char* names[KID_COUNT] = {"k_gemm", "k_qr", "k_apply_q", "k_core_svd", "k_gather",
                                         "k_leaf_potrf", "k_leaf_inv", "k_givens", "k_replay_leaf",
                                         "k_replay_track", "k_inertia", "misc", "k_gemm[apply]",
                                         "k_gemm[chol]", "k_gemm[mult]", "k_gemm_tc",
                                         "k_leaf_chol_inv_cluster", "host_wait"};
  return (kernel >= 0 && kernel < KID_COUNT) ? names[kernel] : "";
}

int sp_kernel_count(void) { return KID_COUNT; }

int64_t sp_launch_count(void) { return launch_count(); }

int sp_hodlr_from_band(sp_ctx_t ctx, int64_t n, int32_t b, const double* ab, int64_t ldab, double mu, int32_t leaf,
                       double tol, int32_t rank_cap, sp_hodlr_t* out) {
  if (!ctx || !out || !ab) return SP_EINVAL;
  if (rank_cap == 0) rank_cap = std::max(160, 20 * b);
  if (leaf == 0 && n >= 1 && b >= 1) leaf = tuned_leaf(ctx, n, b);
  if (n < 1 || b < 1 || ldab < b + 1 || leaf < 2 || leaf < 2 * b || !(tol > 0.0) || rank_cap < 2 * b) {
    ctx->err = "sp_hodlr_from_band: need n >= 1, b >= 1, ldab >= b+1, leaf >= max(2, 2b), tol > 0, rank_cap >= 2b";
    return SP_EINVAL;
  }
  return guarded(ctx, [&] {
    DBuf d = band_on_device(ctx, n, b, ab, ldab);
    *out = hodlr_from_band(ctx, n, b, d.as<double>(), b + 1, mu, leaf, tol, rank_cap);
  });
}

int sp_qdwh_sign(sp_ctx_t ctx, sp_hodlr_t A, const sp_qdwh_opts* opts_in, sp_hodlr_t* sign_out, sp_info* info) {
  if (!ctx || !A || !sign_out) return SP_EINVAL;
  sp_qdwh_opts o;
  sp_qdwh_opts_default(&o);
  if (opts_in) o = *opts_in;
  if (o.max_iter < 1 || o.max_iter > 16 || !(o.delta > 0.0) || o.qr_steps < 0 || o.qr_steps > 1 ||
      (o.precision != SP_FP64 && o.precision != SP_MIXED_FP32 && o.precision != SP_MIXED_NS) ||
      o.polish_steps < 0 || o.polish_steps > 4) {
    ctx->err = "sp_qdwh_sign: invalid options (max_iter in 1..16, delta > 0, qr_steps in {0, 1}, precision, "
               "polish_steps in 0..4)";
    return SP_EINVAL;
  }
  if (o.qr_steps == 1 && !A->band) {
    ctx->err = "sp_qdwh_sign: the QR-based step needs a handle made by sp_hodlr_from_band";
    return SP_EINVAL;
  }
  return guarded(ctx, [&] {
    sp_info inf;
    std::memset(&inf, 0, sizeof(inf));
    ctx->flops = 0.0;
    Timer total(ctx->stream);
    // a NaN or infinity in the band (flagged at ingest) stops here
    check_flags(ctx, "input band");
    double alpha = o.alpha, l0 = o.l0;
    {
      Timer t(ctx->stream);
      if (!(alpha > 0.0) || !(l0 > 0.0)) {
        if (!A->band) fail(SP_EINVAL, "parameter estimation needs the band (or give alpha and l0)");
        double ea = 0.0, el = 0.0;
        qdwh_start(ctx, A->n(), A->b, A->band, A->b + 1, A->mu, &ea, &el);
        if (!(alpha > 0.0)) alpha = ea;
        if (!(l0 > 0.0)) l0 = el;
      }
      inf.ms_param = t.stop();
    }
    inf.alpha = alpha;
    inf.l0 = l0;
    // scalar schedule (Eq. (qdwh_parameters_abc)); stop when |1 - l_k| <= delta
    std::vector<double> as, bs, cs, ls;
    double l = l0;
    while (std::fabs(1.0 - l) > o.delta) {
      if ((int)as.size() >= o.max_iter) fail(SP_EINVAL, "QDWH schedule exceeds max_iter");
      const double l2 = l * l;
      const double g = std::cbrt(4.0 * (1.0 - l2) / (l2 * l2));
      const double sg = std::sqrt(1.0 + g);
      const double a = sg + 0.5 * std::sqrt(8.0 - 4.0 * g + 8.0 * (2.0 - l2) / (l2 * sg));
      const double bb = 0.25 * (a - 1.0) * (a - 1.0);
      const double c = a + bb - 1.0;
      ls.push_back(l);
      as.push_back(a);
      bs.push_back(bb);
      cs.push_back(c);
      l = l * (a + bb * l2) / (1.0 + c * l2);
    }
    Owned X(nullptr);
    int K = (int)as.size();
    for (int k = 0; k < K; ++k) {
      if (o.precision == SP_MIXED_NS && k > 0 && (1.0 - ls[k] * ls[k]) <= kMixedThreshold) {
        // the remaining QDWH steps are replaced by Newton-Schulz steps,
        // counted by the scalar map on l until 1 - l <= 1e-12
        if (!X.p) X.reset(hodlr_add(ctx, 1.0 / alpha, A, 0.0, nullptr, 0.0));
        double lns = ls[k];
        int s = k;
        while (1.0 - lns > 1e-12 && s < 16) {
          Timer t(ctx->stream);
          inf.l[s] = lns;
          inf.a[s] = 1.5;
          inf.b[s] = -0.5;
          inf.c[s] = 0.0;
          X.reset(newton_schulz_step_mixed(ctx, X.p, &inf));
          inf.kind[s] = 4;
          hodlr_check_finite(ctx, X.p);
          check_flags(ctx, "Newton-Schulz step");
          inf.ms_chol += t.stop();
          lns = 0.5 * lns * (3.0 - lns * lns);
          ++s;
        }
        K = s;
        break;
      }
      inf.l[k] = ls[k];
      inf.a[k] = as[k];
      inf.b[k] = bs[k];
      inf.c[k] = cs[k];
      Timer t(ctx->stream);
      if (k == 0 && o.qr_steps == 1) {
        X.reset(qr_step(ctx, A, alpha, as[k], bs[k], cs[k]));
        inf.kind[k] = 1;
        hodlr_check_finite(ctx, X.p);
        check_flags(ctx, "QR-based step");
        inf.ms_qr += t.stop();
      } else {
        if (!X.p) {
          X.reset(hodlr_add(ctx, 1.0 / alpha, A, 0.0, nullptr, 0.0));
        }
        const bool mixed = o.precision == SP_MIXED_FP32 && (1.0 - ls[k] * ls[k]) <= kMixedThreshold;
        if (mixed) {
          X.reset(mixed_step(ctx, X.p, as[k], cs[k], &inf));
          inf.kind[k] = 3;
        } else {
          X.reset(chol_step(ctx, X.p, as[k], bs[k], cs[k], &inf));
          inf.kind[k] = 2;
        }
        hodlr_check_finite(ctx, X.p);
        check_flags(ctx, "Cholesky-based step");
        inf.ms_chol += t.stop();
      }
    }
    if (o.precision != SP_FP64 && X.p) {
      Timer t(ctx->stream);
      for (int p = 0; p < o.polish_steps; ++p) X.reset(newton_schulz_step(ctx, X.p));
      hodlr_check_finite(ctx, X.p);
      check_flags(ctx, "Newton-Schulz polish");
      inf.ms_polish = t.stop();
    }
    if (!X.p) X.reset(hodlr_add(ctx, 1.0 / alpha, A, 0.0, nullptr, 0.0));
    inf.iters = K;
    inf.ms_total = total.stop();
    inf.flops = ctx->flops;
    if (info) {
      inf.max_rank = hodlr_max_rank(ctx, X.p);
      inf.bytes = X.p->bytes;
      inf.levels = X.p->L();
      hodlr_level_stats(ctx, X.p, 32, inf.max_rank_level, inf.mean_rank_level, &inf.nominal_bytes);
      *info = inf;
    }
    *sign_out = X.release();
  });
}

int sp_batched_projector(sp_ctx_t ctx, int32_t nbatch, const int64_t* n, const int32_t* b, const double* const* ab,
                         const int64_t* ldab, const double* mu, int32_t leaf, double tol, int32_t rank_cap,
                         const sp_qdwh_opts* opts, int32_t nstreams, sp_hodlr_t* P_out, sp_info* infos) {
  if (!ctx || nbatch < 0 || (nbatch > 0 && (!n || !b || !ab || !ldab || !mu || !P_out))) return SP_EINVAL;
  for (int i = 0; i < nbatch; ++i)
    if (n[i] < 1 || b[i] < 1 || !ab[i] || ldab[i] < b[i] + 1 || (leaf > 0 && leaf < 2 * b[i])) {
      ctx->err = "sp_batched_projector: invalid instance " + std::to_string(i);
      return SP_EINVAL;
    }
  if (nbatch == 0) return SP_OK;
  const int T = std::max(1, std::min(nstreams > 0 ? nstreams : 16, std::min(nbatch, 64)));
  std::vector<int> order(nbatch);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int x, int y) { return n[x] * (int64_t)b[x] > n[y] * (int64_t)b[y]; });
  std::vector<sp_hodlr_t> outs(nbatch, nullptr);
  std::atomic<int> next{0};
  std::atomic<int> first_err{SP_OK};
  std::mutex mu_err;
  std::string err_msg;
  auto worker = [&]() {
    sp_ctx sub;
    sub.device = ctx->device;
    sub.num_sms = ctx->num_sms;
    sub.alloc = ctx->alloc;
    sub.tsqr_chunk = ctx->tsqr_chunk;
    sub.small_tiles = ctx->small_tiles;
    sub.tuned = ctx->tuned;
    sub.profiling = ctx->profiling;
    cudaSetDevice(ctx->device);
    cudaStream_t s = nullptr;
    const int src = guarded(&sub, [&] {
      check_cuda(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "worker stream");
      sub.stream = s;
      sub.d_flags = static_cast<int*>(dmalloc(sizeof(int) * NFLAGS, s));
      check_cuda(cudaMemsetAsync(sub.d_flags, 0, sizeof(int) * NFLAGS, s), "worker flags");
      if (sub.profiling) {
        sub.d_fc = static_cast<double*>(dmalloc(sizeof(double) * KID_COUNT, s));
        check_cuda(cudaMemsetAsync(sub.d_fc, 0, sizeof(double) * KID_COUNT, s), "worker profiler counters");
      }
    });
    if (src != SP_OK) {
      int expect = SP_OK;
      first_err.compare_exchange_strong(expect, src);
      if (s) cudaStreamDestroy(s);
      return;
    }
    std::vector<int> mine;
    for (;;) {
      if (first_err.load() != SP_OK) break;
      const int k = next.fetch_add(1);
      if (k >= nbatch) break;
      const int i = order[k];
      sp_hodlr_t A = nullptr, S = nullptr, P = nullptr;
      sp_info inf;
      int rc = sp_hodlr_from_band(&sub, n[i], b[i], ab[i], ldab[i], mu[i], leaf > 0 ? leaf : tuned_leaf(ctx, n[i], b[i]),
                                  tol, rank_cap, &A);
      if (rc == SP_OK) rc = sp_qdwh_sign(&sub, A, opts, &S, infos ? &inf : nullptr);
      if (rc == SP_OK) rc = sp_projector(&sub, S, &P);
      hodlr_free(A);
      hodlr_free(S);
      if (rc != SP_OK) {
        int expect = SP_OK;
        if (first_err.compare_exchange_strong(expect, rc)) {
          std::lock_guard<std::mutex> lk(mu_err);
          err_msg = "instance " + std::to_string(i) + ": " + sub.err;
        }
        hodlr_free(P);
        break;
      }
      outs[i] = P;
      if (infos) infos[i] = inf;
      mine.push_back(i);
    }
    cudaStreamSynchronize(s);
    // the results now belong to the caller's stream
    for (int i : mine) {
      outs[i]->stream = ctx->stream;
      outs[i]->tree->stream = ctx->stream;
    }
    if (sub.profiling) {
      // fold the worker's launch times, launch counts and flop counters into
      // the caller's context (its kernels ran concurrently with the other
      // workers', so the times add up to more than the wall time)
      double hfc[KID_COUNT] = {};
      if (sub.d_fc) cudaMemcpy(hfc, sub.d_fc, sizeof(hfc), cudaMemcpyDeviceToHost);
      for (int k = 0; k < KID_COUNT; ++k) {
        for (auto& e : sub.ev[k]) {
          float t = 0.f;
          if (cudaEventElapsedTime(&t, e.first, e.second) == cudaSuccess) sub.ms[k] += t;
          cudaEventDestroy(e.first);
          cudaEventDestroy(e.second);
        }
        sub.ev[k].clear();
      }
      for (auto& ne : sub.chol_ev)
        for (int k = 0; k < ne.nev; ++k) cudaEventDestroy(ne.e[k]);
      sub.chol_ev.clear();
      std::lock_guard<std::mutex> lk(mu_err);
      for (int k = 0; k < KID_COUNT; ++k) {
        ctx->ms[k] += sub.ms[k];
        ctx->launches[k] += sub.launches[k];
        ctx->fc_host[k] += hfc[k];
      }
    }
    {
      AllocScope scope(&sub.alloc);
      dfree(sub.d_flags, s);
      dfree(sub.d_fc, s);
    }
    sub.d_flags = nullptr;
    sub.d_fc = nullptr;
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  };
  std::vector<std::thread> th;
  for (int t = 0; t < T; ++t) th.emplace_back(worker);
  for (auto& x : th) x.join();
  const int rc = first_err.load();
  if (rc != SP_OK) {
    for (auto* P : outs) hodlr_free(P);
    ctx->err = err_msg;
    return rc;
  }
  for (int i = 0; i < nbatch; ++i) P_out[i] = outs[i];
  return SP_OK;
}

int sp_projector(sp_ctx_t ctx, sp_hodlr_t S, sp_hodlr_t* P_out) {
  if (!ctx || !S || !P_out) return SP_EINVAL;
  return guarded(ctx, [&] { *P_out = hodlr_add(ctx, -0.5, S, 0.0, nullptr, 0.5); });
}

int sp_apply(sp_ctx_t ctx, sp_hodlr_t M, int64_t nrhs, const double* X, int64_t ldx, double* Y, int64_t ldy) {
  if (!ctx || !M || !X || !Y || nrhs < 0 || ldx < M->n() || ldy < M->n()) return SP_EINVAL;
  if (nrhs == 0) return SP_OK;
  return guarded(ctx, [&] {
    const int64_t n = M->n();
    const bool hx = !is_device(X), hy = !is_device(Y);
    // host operands are staged through device buffers and the call returns
    // once Y holds the result; device operands stay asynchronous
    DBuf dx(hx ? (size_t)n * nrhs * sizeof(double) : 0, ctx->stream);
    DBuf dy(hy ? (size_t)n * nrhs * sizeof(double) : 0, ctx->stream);
    const double* Xd = X;
    int64_t ldxd = ldx;
    double* Yd = Y;
    int64_t ldyd = ldy;
    if (hx) {
      check_cuda(cudaMemcpy2DAsync(dx.p, n * sizeof(double), X, ldx * sizeof(double), n * sizeof(double), nrhs,
                                   cudaMemcpyHostToDevice, ctx->stream),
                 "apply X upload");
      Xd = dx.as<double>();
      ldxd = n;
    }
    if (hy) {
      Yd = dy.as<double>();
      ldyd = n;
    }
    for (int64_t c0 = 0; c0 < nrhs; c0 += 256) {
      const int w = (int)std::min<int64_t>(256, nrhs - c0);
      hodlr_apply_level(ctx, M, 0, Xd + c0 * ldxd, ldxd, Yd + c0 * ldyd, ldyd, w, nullptr, false, false);
    }
    if (hy) {
      check_cuda(cudaMemcpy2DAsync(Y, ldy * sizeof(double), Yd, n * sizeof(double), n * sizeof(double), nrhs,
                                   cudaMemcpyDeviceToHost, ctx->stream),
                 "apply Y download");
      check_cuda(cudaStreamSynchronize(ctx->stream), "sync");
    }
  });
}

int sp_to_dense(sp_ctx_t ctx, sp_hodlr_t M, int64_t row0, int64_t nrows, double* out, int64_t ld) {
  if (!ctx || !M || !out || row0 < 0 || nrows < 0 || row0 + nrows > M->n() || ld < nrows) return SP_EINVAL;
  if (nrows == 0) return SP_OK;
  return guarded(ctx, [&] {
    if (is_device(out)) {
      hodlr_to_dense(ctx, M, row0, nrows, out, ld);
    } else {
      DBuf d((size_t)nrows * M->n() * sizeof(double), ctx->stream);
      hodlr_to_dense(ctx, M, row0, nrows, d.as<double>(), nrows);
      check_cuda(cudaMemcpy2DAsync(out, ld * sizeof(double), d.p, nrows * sizeof(double), nrows * sizeof(double),
                                   M->n(), cudaMemcpyDeviceToHost, ctx->stream),
                 "to_dense copy");
      check_cuda(cudaStreamSynchronize(ctx->stream), "sync");
    }
  });
}

int sp_trace(sp_ctx_t ctx, sp_hodlr_t M, double* tr) {
  if (!ctx || !M || !tr) return SP_EINVAL;
  return guarded(ctx, [&] { *tr = hodlr_trace(ctx, M); });
}

int sp_trace_product_band(sp_ctx_t ctx, sp_hodlr_t M, int32_t b, const double* ab, int64_t ldab, double* out) {
  if (!ctx || !M || !ab || !out || b < 0 || ldab < b + 1) return SP_EINVAL;
  return guarded(ctx, [&] {
    DBuf d = band_on_device(ctx, M->n(), b, ab, ldab);
    *out = hodlr_trace_band(ctx, M, b, d.as<double>(), b + 1);
  });
}

int sp_hodlr_info(sp_ctx_t ctx, sp_hodlr_t M, int64_t* n, int32_t* levels, int32_t* max_rank, size_t* bytes) {
  if (!ctx || !M) return SP_EINVAL;
  return guarded(ctx, [&] {
    if (n) *n = M->n();
    if (levels) *levels = M->L();
    if (max_rank) *max_rank = hodlr_max_rank(ctx, M);
    if (bytes) *bytes = M->bytes;
  });
}

void sp_hodlr_destroy(sp_hodlr_t M) { hodlr_free(M); }

int sp_hodlr_level_ranks(sp_ctx_t ctx, sp_hodlr_t M, int32_t nlevels, int32_t* max_rank, double* mean_rank,
                         double* nominal_bytes) {
  if (!ctx || !M || nlevels < 0) return SP_EINVAL;
  return guarded(ctx, [&] {
    std::vector<int> mx(std::max(nlevels, 1));
    std::vector<double> mean(std::max(nlevels, 1));
    hodlr_level_stats(ctx, M, nlevels, mx.data(), mean.data(), nominal_bytes);
    for (int l = 0; l < nlevels; ++l) {
      if (max_rank) max_rank[l] = mx[l];
      if (mean_rank) mean_rank[l] = mean[l];
    }
  });
}

int sp_hodlr_add(sp_ctx_t ctx, double alpha, sp_hodlr_t A, double beta, sp_hodlr_t B, double gamma, sp_hodlr_t* C) {
  if (!ctx || !A || !C) return SP_EINVAL;
  if (B && !same_tree(*B->tree, *A->tree)) return SP_EINVAL;
  return guarded(ctx, [&] {
    *C = hodlr_add(ctx, alpha, A, beta, B, gamma);
    check_flags(ctx, "sp_hodlr_add");
  });
}

int sp_hodlr_mult(sp_ctx_t ctx, sp_hodlr_t A, sp_hodlr_t B, sp_hodlr_t* C) {
  if (!ctx || !A || !B || !C || !same_tree(*A->tree, *B->tree)) return SP_EINVAL;
  return guarded(ctx, [&] {
    *C = hodlr_mult(ctx, A, B);
    check_flags(ctx, "sp_hodlr_mult");
  });
}

int sp_hodlr_transpose(sp_ctx_t ctx, sp_hodlr_t M, sp_hodlr_t* T) {
  if (!ctx || !M || !T) return SP_EINVAL;
  return guarded(ctx, [&] { *T = hodlr_transpose(ctx, M); });
}

int sp_hodlr_cholesky(sp_ctx_t ctx, sp_hodlr_t Z, sp_hodlr_t* L) {
  if (!ctx || !Z || !L) return SP_EINVAL;
  return guarded(ctx, [&] {
    sp_hodlr* r = hodlr_cholesky(ctx, Z);
    try {
      check_flags(ctx, "sp_hodlr_cholesky");
    } catch (...) {
      hodlr_free(r);
      throw;
    }
    *L = r;
  });
}

int sp_hodlr_trsm(sp_ctx_t ctx, sp_hodlr_t L, int trans, sp_hodlr_t B, sp_hodlr_t* X) {
  if (!ctx || !L || !B || !X || !same_tree(*L->tree, *B->tree)) return SP_EINVAL;
  return guarded(ctx, [&] {
    *X = hodlr_trsm(ctx, L, trans != 0, B);
    check_flags(ctx, "sp_hodlr_trsm");
  });
}

int sp_inertia(sp_ctx_t ctx, int64_t n, int32_t b, const double* ab, int64_t ldab, int32_t nshift,
               const double* shifts, int64_t* counts) {
  if (!ctx || !ab || !shifts || !counts || n < 1 || b < 0 || ldab < b + 1 || nshift < 0) return SP_EINVAL;
  return guarded(ctx, [&] {
    DBuf d = band_on_device(ctx, n, b, ab, ldab);
    DBuf s((size_t)nshift * sizeof(double) + 8, ctx->stream);
    check_cuda(cudaMemcpyAsync(s.p, shifts, nshift * sizeof(double),
                               is_device(shifts) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream),
               "shifts");
    DBuf c((size_t)nshift * sizeof(int64_t) + 8, ctx->stream);
    inertia_counts(ctx, n, b, d.as<double>(), b + 1, nshift, s.as<double>(), c.as<int64_t>());
    check_cuda(cudaMemcpyAsync(counts, c.p, nshift * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream), "counts");
    check_cuda(cudaStreamSynchronize(ctx->stream), "sync");
  });
}

// Inertia counts for callers that cannot allocate device memory: scratch in
// a file-scope device array (see include/sp.h); no cudaMalloc/cudaFree.
int sp_inertia_noalloc(sp_ctx_t ctx, int64_t n, int32_t b, const double* ab, int64_t ldab, int32_t nshift,
                       const double* shifts, int64_t* counts) {
  if (!ctx || !ab || !shifts || !counts || n < 1 || b < 0 || ldab < b + 1 || nshift < 0) return SP_EINVAL;
  return guarded(ctx, [&] {
    int dev = -1;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != ctx->device)
      fail(SP_EINVAL, "sp_inertia_noalloc: the current device (" + std::to_string(dev) +
                          ") is not the context's device (" + std::to_string(ctx->device) + ")");
    // a host pointer would reach the kernel: reject it here
    if (!is_device(ab) || !is_device(shifts) || !is_device(counts))
      fail(SP_EINVAL, "sp_inertia_noalloc: ab, shifts and counts must be device pointers");
    inertia_counts_noalloc(ctx, n, b, ab, ldab, nshift, shifts, counts);
  });
}

int sp_locate_shift(sp_ctx_t ctx, int64_t n, int32_t b, const double* ab, int64_t ldab, int64_t nu, double* mu,
                    double* lam_nu_hi, double* lam_nu1_lo) {
  if (!ctx || !ab || !mu || n < 1 || b < 0 || ldab < b + 1 || nu < 0 || nu > n) return SP_EINVAL;
  return guarded(ctx, [&] {
    DBuf d = band_on_device(ctx, n, b, ab, ldab);
    double h1 = 0, h2 = 0;
    locate_shift(ctx, n, b, d.as<double>(), b + 1, nu, mu, &h1, &h2);
    if (lam_nu_hi) *lam_nu_hi = h1;
    if (lam_nu1_lo) *lam_nu1_lo = h2;
  });
}

int sp_qdwh_start(sp_ctx_t ctx, int64_t n, int32_t b, const double* ab, int64_t ldab, double mu, double* alpha,
                  double* l0) {
  if (!ctx || !ab || !alpha || !l0 || n < 1 || b < 0 || ldab < b + 1) return SP_EINVAL;
  return guarded(ctx, [&] {
    DBuf d = band_on_device(ctx, n, b, ab, ldab);
    // the counts are of A - mu I's eigenvalues relative to mu: count A at
    // shifts mu +- d directly
    qdwh_start(ctx, n, b, d.as<double>(), b + 1, mu, alpha, l0);
  });
}

int sp_qdwh_params_paper(sp_ctx_t ctx, int64_t n, int32_t b, const double* ab, int64_t ldab, double mu,
                         double* alpha, double* l0, int32_t* iters) {
  if (!ctx || !ab || !alpha || !l0 || n < 1 || b < 0 || ldab < b + 1) return SP_EINVAL;
  return guarded(ctx, [&] {
    DBuf d = band_on_device(ctx, n, b, ab, ldab);
    int it[2] = {0, 0};
    qdwh_params_paper(ctx, n, b, d.as<double>(), b + 1, mu, alpha, l0, it);
    check_flags(ctx, "banded LU of the 1-norm estimator");
    if (iters) {
      iters[0] = it[0];
      iters[1] = it[1];
    }
  });
}

int sp_givens_generate(sp_ctx_t ctx, int64_t n, int32_t b, const double* ab, int64_t ldab, double scale, double* cs) {
  if (!ctx || !ab || !cs || n < 1 || b < 1 || ldab < b + 1) return SP_EINVAL;
  return guarded(ctx, [&] { givens_generate(ctx, n, b, ab, ldab, 0.0, scale, cs); });
}

int sp_fastqr_factors(sp_ctx_t ctx, sp_hodlr_t A, double scale, sp_hodlr_t* Q1, sp_hodlr_t* Q2) {
  if (!ctx || !A || !Q1 || !Q2) return SP_EINVAL;
  return guarded(ctx, [&] { fastqr_factors(ctx, A, scale, Q1, Q2); });
}

}  // extern "C"
