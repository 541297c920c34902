// sp_blas.cu -- dense building blocks of the HODLR arithmetic: batched
// binary64 (and binary32) GEMM with device-side sizes, leaf Cholesky, leaf
// inverses, and small strided element-wise kernels.  Every kernel takes a task list so
// that one launch covers all blocks of one kind across the HODLR tree.
//
// Roofline note: on GB300 binary64 runs at ~1.2 TFLOP/s (8 GFLOP/s per SM)
// while HBM delivers ~6.8 TB/s, so every binary64 kernel here is bound by the
// FP64 pipe (ridge ~0.18 flop/byte); the tiling aims at keeping each SM's
// DFMA pipe busy, not at saving bytes.
#include <cooperative_groups.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <atomic>
#include <cstdio>
#include <stdexcept>
#include <unordered_map>

#include <vector>
#include "sp_internal.h"

namespace sp {

// ------------------------------------------------------------------ errors --
[[noreturn]] void fail(int code, const std::string& msg) { throw Error{code, msg}; }

void check_cuda(cudaError_t e, const char* what) {
  if (e != cudaSuccess) fail(SP_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

namespace {
std::atomic<int64_t> g_launches{0};
}

void check_launch(const char* what) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  check_cuda(cudaGetLastError(), what);
}

int64_t launch_count() { return g_launches.load(); }

ProfScope::ProfScope(sp_ctx* c, int k) : ctx(c), kid(k) {
  if (ctx->profiling) {
    cudaEventCreate(&a);
    cudaEventRecord(a, ctx->stream);
  }
}

ProfScope::~ProfScope() {
  if (ctx->profiling && a) {
    cudaEvent_t b = nullptr;
    cudaEventCreate(&b);
    cudaEventRecord(b, ctx->stream);
    ctx->ev[kid].emplace_back(a, b);
    ctx->launches[kid] += 1;
  }
}

// ------------------------------------------------------------------ memory --
namespace {
// Allocator of the entry point running on this thread (null: default pool).
thread_local const Allocator* t_alloc = nullptr;
// Buffers made by a caller's allocator, with the allocator and size to free
// them with (only consulted once a caller's allocator has been used).
std::mutex g_custom_mu;
std::unordered_map<void*, std::pair<Allocator, size_t>> g_custom;
std::atomic<bool> g_any_custom{false};
}  // namespace

AllocScope::AllocScope(const Allocator* a) : prev(t_alloc) { t_alloc = a; }
AllocScope::~AllocScope() { t_alloc = prev; }

void* dmalloc(size_t bytes, cudaStream_t st) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  if (t_alloc && t_alloc->custom()) {
    p = t_alloc->alloc(bytes, (void*)st, t_alloc->user);
    if (!p) fail(SP_ENOMEM, "caller's allocator returned NULL for " + std::to_string(bytes) + " bytes");
    std::lock_guard<std::mutex> lk(g_custom_mu);
    g_custom[p] = {*t_alloc, bytes};
    g_any_custom.store(true);
    return p;
  }
  cudaError_t e = cudaMallocAsync(&p, bytes, st);
  if (e != cudaSuccess || !p) {
    (void)cudaGetLastError();
    fail(SP_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  }
  return p;
}

void dfree(void* p, cudaStream_t st) {
  if (!p) return;
  if (g_any_custom.load()) {
    std::unique_lock<std::mutex> lk(g_custom_mu);
    auto it = g_custom.find(p);
    if (it != g_custom.end()) {
      const Allocator a = it->second.first;
      const size_t bytes = it->second.second;
      g_custom.erase(it);
      lk.unlock();
      a.free(p, bytes, (void*)st, a.user);
      return;
    }
  }
  (void)cudaFreeAsync(p, st);
}

DBuf::DBuf(size_t b, cudaStream_t s) : p(dmalloc(b, s)), bytes(b), st(s) {}
DBuf::~DBuf() { dfree(p, st); }
DBuf& DBuf::operator=(DBuf&& o) noexcept {
  if (this != &o) {
    dfree(p, st);
    p = o.p;
    bytes = o.bytes;
    st = o.st;
    o.p = nullptr;
  }
  return *this;
}

void configure_dynamic_smem(const void* func) {
  int dev = 0, optin = 0;
  check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  check_cuda(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "smem opt-in");
  cudaFuncAttributes fa;
  check_cuda(cudaFuncGetAttributes(&fa, func), "function attributes");
  const int dyn = optin - (int)fa.sharedSizeBytes;
  if (dyn > fa.maxDynamicSharedSizeBytes)
    check_cuda(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn), "smem attribute");
}

void ensure_dynamic_smem(const void* func, size_t bytes) {
  if (bytes <= 48 * 1024) return;
  cudaFuncAttributes fa;
  check_cuda(cudaFuncGetAttributes(&fa, func), "function attributes");
  if (bytes > (size_t)fa.maxDynamicSharedSizeBytes)
    fail(SP_EINVAL, "problem needs " + std::to_string(bytes) + " bytes of shared memory per CTA, above the limit " +
                        std::to_string(fa.maxDynamicSharedSizeBytes));
}

// ------------------------------------------------------------ batched GEMM --
namespace {
constexpr int kGT = 64;  // output tile edge
constexpr int kGK = 16;  // k step staged in shared memory

__device__ __forceinline__ int dsize(int s, const int* p) {
  if (p) {
    int v = *p;
    v = v < 0 ? 0 : v;
    return v < s ? v : s;
  }
  return s;
}

// MT is the arithmetic type of the tile (binary64 here; the mixed-precision
// scope runs on the tensor cores instead, sp_tc.cu).
//
// The grid is laid out in 64 x 64 output tiles; each CTA then computes only
// the part of its tile inside the actual (device-resident) m x n: a
// (16 MI) x (16 MJ) sub-tile with MI, MJ in {1, 2, 4}, each of the 256
// threads an MI x MJ micro-tile.  Rank-sized dimensions (~30 of a capacity of
// 160) thus cost no padded FMAs.
template <bool TA, bool TB, typename MT, int MI, int MJ>
__device__ __forceinline__ void gemm_tile(const GemmTask& t, int m, int n, int row0, int col0, int kbeg, int kend,
                                          int split, MT (*As)[kGT + 1], MT (*Bs)[kGT + 1]) {
  constexpr int TM = 16 * MI, TN = 16 * MJ;
  // independent partial sums per output (up to 16 accumulators a thread):
  // the k range is otherwise one dependent FMA chain per output, 64 cycles
  // a link on this part, which is what a small GEMM on few SMs waits for;
  // summed in a fixed order at the end
  constexpr int NP = (16 / (MI * MJ)) < 4 ? 16 / (MI * MJ) : 4;
  const int tid = threadIdx.x, r = tid & 15, c = tid >> 4;
  MT acc[NP][MI][MJ];
#pragma unroll
  for (int p = 0; p < NP; ++p)
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
      for (int j = 0; j < MJ; ++j) acc[p][i][j] = (MT)0;
  for (int kb = kbeg; kb < kend; kb += kGK) {
    for (int e = tid; e < TM * kGK; e += 256) {
      int row, kk;
      if (!TA) { row = e % TM; kk = e / TM; } else { kk = e % kGK; row = e / kGK; }
      const int gr = row0 + row, gk = kb + kk;
      double v = 0.0;
      if (gr < m && gk < kend) v = TA ? t.A[gk + (int64_t)gr * t.lda] : t.A[gr + (int64_t)gk * t.lda];
      As[kk][row] = (MT)v;
    }
    for (int e = tid; e < TN * kGK; e += 256) {
      int col, kk;
      if (!TB) { kk = e % kGK; col = e / kGK; } else { col = e % TN; kk = e / TN; }
      const int gc = col0 + col, gk = kb + kk;
      double v = 0.0;
      if (gc < n && gk < kend) v = TB ? t.B[gc + (int64_t)gk * t.ldb] : t.B[gk + (int64_t)gc * t.ldb];
      Bs[kk][col] = (MT)v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      MT a[MI], b[MJ];
#pragma unroll
      for (int i = 0; i < MI; ++i) a[i] = As[kk][r + 16 * i];
#pragma unroll
      for (int j = 0; j < MJ; ++j) b[j] = Bs[kk][c + 16 * j];
#pragma unroll
      for (int i = 0; i < MI; ++i)
#pragma unroll
        for (int j = 0; j < MJ; ++j) acc[kk % NP][i][j] = fma(a[i], b[j], acc[kk % NP][i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 1; p < NP; ++p)
#pragma unroll
    for (int i = 0; i < MI; ++i)
#pragma unroll
      for (int j = 0; j < MJ; ++j) acc[0][i][j] += acc[p][i][j];
#pragma unroll
  for (int i = 0; i < MI; ++i)
#pragma unroll
    for (int j = 0; j < MJ; ++j) {
      const int gr = row0 + r + 16 * i, gc = col0 + c + 16 * j;
      if (gr < m && gc < n) {
        const double v = t.alpha * (double)acc[0][i][j];
        if (split) {
          // partial tile of k chunk blockIdx.z (static m x n slot per chunk)
          t.W[(size_t)blockIdx.z * (size_t)t.m * (size_t)t.n + gr + (int64_t)gc * t.m] = v;
        } else {
          double* p = t.C + gr + (int64_t)gc * t.ldc;
          *p = (t.beta == 0.0) ? v : v + t.beta * (*p);
        }
      }
    }
}

// te: edge of the output tiles the grid is laid out in (64, or 16 for small
// problems, so that their few outputs still spread over many SMs).
template <bool TA, bool TB, typename MT>
__global__ void __launch_bounds__(256) k_gemm(const GemmTask* __restrict__ tasks, int kchunk, int split, int te,
                                              double* fc) {
  const GemmTask t = tasks[blockIdx.y];
  const int m = dsize(t.m, t.pm), n = dsize(t.n, t.pn), k = dsize(t.k, t.pk);
  const int tiles_m = (m + te - 1) / te;
  const int tile = blockIdx.x;
  if (tile >= tiles_m * ((n + te - 1) / te)) return;
  const int row0 = (tile % tiles_m) * te, col0 = (tile / tiles_m) * te;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(k, kbeg + kchunk);
  if (kbeg >= kend && blockIdx.z > 0) return;
  __shared__ MT As[kGK][kGT + 1];
  __shared__ MT Bs[kGK][kGT + 1];
  const int em = min(te, m - row0), en = min(te, n - col0);
  const int mi = em <= 16 ? 1 : (em <= 32 ? 2 : 4);
  const int mj = en <= 16 ? 1 : (en <= 32 ? 2 : 4);
  switch (mi * 8 + mj) {
    case 9: gemm_tile<TA, TB, MT, 1, 1>(t, m, n, row0, col0, kbeg, kend, split, As, Bs); break;
    case 10: gemm_tile<TA, TB, MT, 1, 2>(t, m, n, row0, col0, kbeg, kend, split, As, Bs); break;
    case 12: gemm_tile<TA, TB, MT, 1, 4>(t, m, n, row0, col0, kbeg, kend, split, As, Bs); break;
    case 17: gemm_tile<TA, TB, MT, 2, 1>(t, m, n, row0, col0, kbeg, kend, split, As, Bs); break;
    case 18: gemm_tile<TA, TB, MT, 2, 2>(t, m, n, row0, col0, kbeg, kend, split, As, Bs); break;
    case 20: gemm_tile<TA, TB, MT, 2, 4>(t, m, n, row0, col0, kbeg, kend, split, As, Bs); break;
    case 33: gemm_tile<TA, TB, MT, 4, 1>(t, m, n, row0, col0, kbeg, kend, split, As, Bs); break;
    case 34: gemm_tile<TA, TB, MT, 4, 2>(t, m, n, row0, col0, kbeg, kend, split, As, Bs); break;
    default: gemm_tile<TA, TB, MT, 4, 4>(t, m, n, row0, col0, kbeg, kend, split, As, Bs); break;
  }
  if (fc && threadIdx.x == 0) atomicAdd(fc, 2.0 * (double)em * (double)en * (double)max(kend - kbeg, 0));
}

// Flags NaN / infinity anywhere in p[0, count).
__global__ void k_nonfinite(const double* __restrict__ p, size_t count, int* flags) {
  bool bad = false;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    bad |= !isfinite(p[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&flags[FLAG_NONFINITE], 1);
}

// Sums the k chunks of a split GEMM in chunk order (reproducible, unlike
// atomics): C = sum_z W_z + beta C over the device-resident m x n.
__global__ void k_splitk_reduce(const GemmTask* __restrict__ tasks, int kchunk) {
  const GemmTask t = tasks[blockIdx.y];
  const int m = dsize(t.m, t.pm), n = dsize(t.n, t.pn), k = dsize(t.k, t.pk);
  const int nz = t.nsplit > 0 ? t.nsplit : (k > 0 ? (k + kchunk - 1) / kchunk : 1);
  const size_t slot = (size_t)t.m * (size_t)t.n;
  const int64_t total = (int64_t)m * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    const size_t w = i + (size_t)j * t.m;
    double v = 0.0;
    for (int z = 0; z < nz; ++z) v += t.W[z * slot + w];
    double* p = t.C + i + (int64_t)j * t.ldc;
    *p = (t.beta == 0.0) ? v : v + t.beta * (*p);
  }
}

__global__ void k_axpby(const AxpbyTask* __restrict__ tasks) {
  const AxpbyTask t = tasks[blockIdx.y];
  const int m = dsize(t.m, t.pm), n = dsize(t.n, t.pn);
  const int64_t total = (int64_t)m * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    double v = (t.X && t.a != 0.0) ? t.a * t.X[i + (int64_t)j * t.ldx] : 0.0;
    double* y = t.Y + i + (int64_t)j * t.ldy;
    if (t.b != 0.0) v += t.b * (*y);
    if (i == j) v += t.g;
    *y = v;
  }
}

__global__ void k_zero_tail(const ZeroTailTask* __restrict__ tasks) {
  const ZeroTailTask t = tasks[blockIdx.y];
  int r = t.prank ? *t.prank : 0;
  r = r < 0 ? 0 : (r > t.cap ? t.cap : r);
  const int64_t total = (int64_t)t.m * (t.cap - r);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % t.m), j = r + (int)(e / t.m);
    t.P[i + (int64_t)j * t.ld] = 0.0;
  }
}

// Blocked right-looking Cholesky of one leaf per CTA (1024 threads): each
// 32-column panel (rows jb..n-1) is factored in shared memory (two barriers
// per column, pivots by one thread), written back,
// and the trailing lower triangle gets A22 -= P P^T, every thread producing
// 2x2 outputs from the shared-memory panel.  The upper triangle is zeroed.
constexpr int kPW = 32;  // panel width

__global__ void __launch_bounds__(1024) k_leaf_potrf(const LeafTask* __restrict__ tasks, int* flags, double* fc) {
  const LeafTask t = tasks[blockIdx.x];
  double* A = t.A;
  const int64_t lda = t.lda;
  const int n = t.n;
  // algorithmic work of a Cholesky factorisation: n^3/3 + n^2/2 + n/6 flops
  if (fc && threadIdx.x == 0) atomicAdd(fc, (double)n * n * n / 3.0 + (double)n * n / 2.0 + n / 6.0);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* P = reinterpret_cast<double*>(smem_raw);  // panel, row-major (n rows x (kPW+1))
  constexpr int LDP = kPW + 1;
  __shared__ double dsq[kPW];
  __shared__ double s_inv;
  for (int jb = 0; jb < n; jb += kPW) {
    const int w = min(kPW, n - jb);
    const int pr = n - jb;  // panel rows
    for (int e = threadIdx.x; e < pr * w; e += blockDim.x) {
      const int r = e % pr, c = e / pr;
      P[r * LDP + c] = A[(jb + r) + (int64_t)(jb + c) * lda];
    }
    __syncthreads();
    // Square roots and reciprocals of the pivots are taken by thread 0 only:
    // binary64 divides and square roots are expensive on this part, and 1024
    // threads repeating them would cost more than the factorisation.  Thread
    // 0 also updates the next pivot (its first element of every update phase),
    // so the next reciprocal is ready at the barrier that ends the phase.
    auto pivot = [&](int j) {
      double d = P[j * LDP + j];
      if (!(d > 0.0)) {
        atomicOr(&flags[FLAG_BREAKDOWN], 1);
        d = 1.0;
      }
      d = sqrt(d);
      dsq[j] = d;
      s_inv = 1.0 / d;
    };
    if (threadIdx.x == 0) pivot(0);
    __syncthreads();
    for (int j = 0; j < w; ++j) {
      const double inv = s_inv;
      for (int r = j + 1 + threadIdx.x; r < pr; r += blockDim.x) P[r * LDP + j] *= inv;
      __syncthreads();
      // update panel columns j+1..w-1, rows >= column (element 0 is the next pivot)
      const int nc = w - j - 1;
      for (int e = threadIdx.x; e < (pr - j - 1) * nc; e += blockDim.x) {
        const int r = j + 1 + e / nc, c = j + 1 + e % nc;
        if (r >= c) P[r * LDP + c] -= P[r * LDP + j] * P[c * LDP + j];
      }
      if (threadIdx.x == 0 && j + 1 < w) pivot(j + 1);
      __syncthreads();
    }
    if (threadIdx.x < w) P[threadIdx.x * LDP + threadIdx.x] = dsq[threadIdx.x];
    __syncthreads();
    for (int e = threadIdx.x; e < pr * w; e += blockDim.x) {
      const int r = e % pr, c = e / pr;
      A[(jb + r) + (int64_t)(jb + c) * lda] = (r >= c) ? P[r * LDP + c] : 0.0;
    }
    // trailing update: rows/cols jb+w..n-1, lower triangle, 2x2 per thread
    const int m = n - jb - w;
    const int mb = (m + 1) / 2;
    for (int e = threadIdx.x; e < mb * mb; e += blockDim.x) {
      const int bi = e % mb, bc = e / mb;
      if (bi < bc) continue;
      const int r0 = w + 2 * bi, c0 = w + 2 * bc;  // panel-relative rows
      double a00 = 0.0, a01 = 0.0, a10 = 0.0, a11 = 0.0;
      const bool r1ok = r0 + 1 < pr, c1ok = c0 + 1 < pr;
#pragma unroll 8
      for (int k = 0; k < w; ++k) {
        const double x0 = P[r0 * LDP + k], y0 = P[c0 * LDP + k];
        const double x1 = r1ok ? P[(r0 + 1) * LDP + k] : 0.0, y1 = c1ok ? P[(c0 + 1) * LDP + k] : 0.0;
        a00 = fma(x0, y0, a00);
        a01 = fma(x0, y1, a01);
        a10 = fma(x1, y0, a10);
        a11 = fma(x1, y1, a11);
      }
      const int64_t R0 = jb + r0, C0 = jb + c0;
      A[R0 + C0 * lda] -= a00;
      if (c1ok && r0 >= c0 + 1) A[R0 + (C0 + 1) * lda] -= a01;
      if (r1ok) A[(R0 + 1) + C0 * lda] -= a10;
      if (r1ok && c1ok) A[(R0 + 1) + (C0 + 1) * lda] -= a11;
    }
    __syncthreads();
  }
  for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
    const int i = (int)(e % n), c = (int)(e / n);
    if (i < c) A[i + (int64_t)c * lda] = 0.0;
  }
}

// ----------------------------- leaf Cholesky and inverse on a cluster ----
// L = chol(A) and X = L^{-1} of one leaf (n <= 256) by a cluster of kCC CTAs
// on kCC SMs, blocked in 16 x 16 blocks.  Binary64 runs at about two FMAs per
// clock per SM on this part, so one SM needs ~0.3 ms for the factorisation of
// a 195-row leaf alone, and the leaf factorisations form the H-Cholesky's
// sequential critical path.
//
// The lower-triangular blocks of A (and of the inverse's work array B, which
// starts as I) are dealt over the cluster by their row-major index q: block q
// lives in CTA q % kCC, slot q / kCC of its shared memory, and its owner does
// every update of it.  Other CTAs read it through distributed shared memory.
// Right-looking block step p (two cluster barriers per step):
//  (B) L_ip = A_ip L_pp^{-T} for the blocks below the diagonal block, and the
//      inverse's row block X_pj = L_pp^{-1} B_pj (forward substitution of
//      L X = I, Sec. "H-Cholesky" inverse factor); barrier;
//  (C) each CTA copies the column panel L_.p and the row panel X_p. into its
//      own shared memory and applies its blocks' updates
//      A_ij -= L_ip L_jp^T (p < j <= i) and B_ij -= L_ip X_pj (i > p, j <= p);
//      the owner of block (p+1, p+1) updates it first and factors it at once
//      (one warp, row i of the block in lane i's registers, a reciprocal
//      square root per column), so the next diagonal factorisation overlaps
//      the other CTAs' updates; barrier.
// Rows beyond n are padded as identity.  A non-positive pivot sets the
// breakdown flag and continues with pivot 1.
constexpr int kCB = 16;                                                  // block edge
constexpr int kCC = 8;                                                   // CTAs per cluster (portable)
constexpr int kCMaxNB = 16;                                              // block rows: n <= 256
constexpr int kCMaxN = kCB * kCMaxNB;
constexpr int kCSlots = (kCMaxNB * (kCMaxNB + 1) / 2 + kCC - 1) / kCC;  // blocks per CTA
constexpr int kCP = kCB + 1;                                             // padded row

struct ClusterSmem {
  double A[kCSlots][kCB][kCP];    // owned blocks of A, then L
  double X[kCSlots][kCB][kCP];    // owned blocks of B, then X = L^{-1}
  double Lpan[kCMaxNB][kCB][kCP];  // column panel L_ip of the current step
  double Xpan[kCMaxNB][kCB][kCP];  // row panel X_pj of the current step
  double Linv[kCB][kCP];           // inverse of this CTA's latest diagonal block
  double Lcp[kCB][kCP];            // copy of the current step's L_pp^{-1}
  double yv[kCB];                  // reciprocals of the diagonal block's pivots
};

__device__ __forceinline__ int blk_q(int i, int j) { return i * (i + 1) / 2 + j; }
__device__ __forceinline__ int blk_owner(int i, int j) { return blk_q(i, j) % kCC; }
__device__ __forceinline__ int blk_slot(int i, int j) { return blk_q(i, j) / kCC; }

// Factor the 16 x 16 diagonal block D (row-major, ld kCP, lower triangle) in
// place and write its inverse to Linv (zero above the diagonal), with the
// CTA's first four warps: on this part a binary64 warp instruction occupies
// its sub-partition's FP64 pipe for many cycles, so one warp per
// sub-partition (not one warp in all) carries the column chain.  Thread t of
// 0..127 owns entries (r, c0) and (r, c0 + 8), r = t % 16, c0 = t / 16.
// Column step j: the pivot's reciprocal square root (computed by every
// thread from the shared pivot), the column scaled, then the trailing entries
// updated; two 128-thread barriers per column.  Then the inverse by rows of
// the forward substitution L X = I (X_kk = 1/L_kk), one barrier per row.
__device__ __forceinline__ void bar128() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

__device__ void cluster_diag_block(double (*D)[kCP], double (*Linv)[kCP], double* yv, int* flags) {
  const int t = threadIdx.x;
  const int r = t & 15, c0 = t >> 4, c1 = c0 + 8;
  bool bad = false;
  for (int j = 0; j < kCB; ++j) {
    double d = D[j][j];
    if (!(d > 0.0)) {
      bad = true;
      d = 1.0;
    }
    const double y = rsqrt(d);
    bar128();  // every thread has read the pivot before it is overwritten
    if (c0 == j || c1 == j) {
      if (r > j) D[r][j] *= y;
      else if (r == j) {
        D[j][j] = d * y;
        yv[j] = y;
      }
    }
    bar128();
    if (c0 > j && c0 <= r) D[r][c0] = fma(-D[r][j], D[c0][j], D[r][c0]);
    if (c1 > j && c1 <= r) D[r][c1] = fma(-D[r][j], D[c1][j], D[r][c1]);
    bar128();
  }
  if (bad && t == 0) atomicOr(&flags[FLAG_BREAKDOWN], 1);
  // inverse: s_r[c] = sum_{k<r} L_rk X_kc; row k final after k steps
  double s0 = 0.0, s1 = 0.0;
  Linv[r][c0] = 0.0;
  Linv[r][c1] = 0.0;
  for (int k = 0; k < kCB; ++k) {
    if (r == k) {
      const double yk = yv[k];
      Linv[k][c0] = (c0 < k) ? -yk * s0 : (c0 == k ? yk : 0.0);
      Linv[k][c1] = (c1 < k) ? -yk * s1 : (c1 == k ? yk : 0.0);
    }
    bar128();
    if (r > k) {
      const double l = D[r][k];
      if (c0 <= k) s0 = fma(l, Linv[k][c0], s0);
      if (c1 <= k) s1 = fma(l, Linv[k][c1], s1);
    }
  }
  // the strict upper triangle of D is not part of L
  if (c0 > r) D[r][c0] = 0.0;
  if (c1 > r) D[r][c1] = 0.0;
}

// The diagonal step of the block's owner: factor, then X_pp = L_pp^{-1}.
__device__ void cluster_diag_step(ClusterSmem& S, int p, int* flags) {
  const int sl = blk_slot(p, p);
  if (threadIdx.x < 128) cluster_diag_block(S.A[sl], S.Linv, S.yv, flags);
  __syncthreads();
  const int r = threadIdx.x & 15, c = threadIdx.x >> 4;
  S.X[sl][r][c] = S.Linv[r][c];
  __syncthreads();
}

__global__ void __cluster_dims__(kCC, 1, 1) __launch_bounds__(256)
    k_leaf_chol_inv_cluster(const LeafTask* __restrict__ tasks, int* flags, double* fc_potrf, double* fc_inv) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ClusterSmem& S = *reinterpret_cast<ClusterSmem*>(smem_raw);
  const int rank = (int)cl.block_rank();
  const LeafTask t = tasks[blockIdx.y];
  const int n = t.n;
  const int NB = (n + kCB - 1) / kCB;
  const int nq = NB * (NB + 1) / 2;
  const int tid = threadIdx.x;
  const int r = tid & 15, c = tid >> 4;  // 256 threads = one 16 x 16 block
  if (rank == 0 && tid == 0) {
    const double dn = (double)n;
    if (fc_potrf) atomicAdd(fc_potrf, dn * dn * dn / 3.0 + dn * dn / 2.0 + dn / 6.0);
    // triangular inverse: sum over columns of m^2, m = n - c  ->  n(n+1)(2n+1)/6
    if (fc_inv) atomicAdd(fc_inv, dn * (dn + 1.0) * (2.0 * dn + 1.0) / 6.0);
  }
  // owned blocks: A (lower triangle; rows beyond n padded as identity), B = I
  for (int q = rank; q < nq; q += kCC) {
    int i = 0;
    while ((i + 1) * (i + 2) / 2 <= q) ++i;
    const int j = q - i * (i + 1) / 2;
    const int gr = i * kCB + r, gc = j * kCB + c;
    double a;
    if (gr < n && gc < n) a = (i != j || r >= c) ? t.A[gr + (int64_t)gc * t.lda] : 0.0;
    else a = (gr == gc) ? 1.0 : 0.0;
    S.A[q / kCC][r][c] = a;
    S.X[q / kCC][r][c] = (i == j && r == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  if (rank == blk_owner(0, 0)) cluster_diag_step(S, 0, flags);
  cl.sync();
  for (int p = 0; p < NB; ++p) {
    // (B) L_ip = A_ip L_pp^{-T} (i > p); X_pj = L_pp^{-1} B_pj (j < p)
    const double* Lo = cl.map_shared_rank(&S.Linv[0][0], blk_owner(p, p));
    S.Lcp[r][c] = Lo[r * kCP + c];
    __syncthreads();
    for (int i = p + 1; i < NB; ++i) {
      if (blk_owner(i, p) != rank) continue;
      double(*Bk)[kCP] = S.A[blk_slot(i, p)];
      double a0 = 0.0, a1 = 0.0;
#pragma unroll
      for (int k = 0; k < kCB; k += 2) {
        a0 = fma(Bk[r][k], S.Lcp[c][k], a0);
        a1 = fma(Bk[r][k + 1], S.Lcp[c][k + 1], a1);
      }
      __syncthreads();
      Bk[r][c] = a0 + a1;
      __syncthreads();
    }
    for (int j = 0; j < p; ++j) {
      if (blk_owner(p, j) != rank) continue;
      double(*Bk)[kCP] = S.X[blk_slot(p, j)];
      double a0 = 0.0, a1 = 0.0;
#pragma unroll
      for (int k = 0; k < kCB; k += 2) {
        a0 = fma(S.Lcp[r][k], Bk[k][c], a0);
        a1 = fma(S.Lcp[r][k + 1], Bk[k + 1][c], a1);
      }
      __syncthreads();
      Bk[r][c] = a0 + a1;
      __syncthreads();
    }
    cl.sync();
    // (C) panels L_ip (i > p) and X_pj (j <= p) into local shared memory
    for (int i = p + 1; i < NB; ++i) {
      const double* src = cl.map_shared_rank(&S.A[blk_slot(i, p)][0][0], blk_owner(i, p));
      S.Lpan[i][r][c] = src[r * kCP + c];
    }
    for (int j = 0; j <= p; ++j) {
      const double* src = cl.map_shared_rank(&S.X[blk_slot(p, j)][0][0], blk_owner(p, j));
      S.Xpan[j][r][c] = src[r * kCP + c];
    }
    __syncthreads();
    const int nx = p + 1;
    if (nx < NB && blk_owner(nx, nx) == rank) {
      double(*Ak)[kCP] = S.A[blk_slot(nx, nx)];
      double a0 = 0.0, a1 = 0.0;
#pragma unroll
      for (int k = 0; k < kCB; k += 2) {
        a0 = fma(S.Lpan[nx][r][k], S.Lpan[nx][c][k], a0);
        a1 = fma(S.Lpan[nx][r][k + 1], S.Lpan[nx][c][k + 1], a1);
      }
      if (r >= c) Ak[r][c] -= a0 + a1;
      __syncthreads();
      cluster_diag_step(S, nx, flags);
    }
    for (int i = p + 1; i < NB; ++i)
      for (int j = p + 1; j <= i; ++j) {
        if (blk_owner(i, j) != rank || (i == nx && j == nx)) continue;
        double(*Ak)[kCP] = S.A[blk_slot(i, j)];
        double a0 = 0.0, a1 = 0.0;
#pragma unroll
        for (int k = 0; k < kCB; k += 2) {
          a0 = fma(S.Lpan[i][r][k], S.Lpan[j][c][k], a0);
          a1 = fma(S.Lpan[i][r][k + 1], S.Lpan[j][c][k + 1], a1);
        }
        if (i != j || r >= c) Ak[r][c] -= a0 + a1;
      }
    for (int i = p + 1; i < NB; ++i)
      for (int j = 0; j <= p; ++j) {
        if (blk_owner(i, j) != rank) continue;
        double(*Xk)[kCP] = S.X[blk_slot(i, j)];
        double a0 = 0.0, a1 = 0.0;
#pragma unroll
        for (int k = 0; k < kCB; k += 2) {
          a0 = fma(S.Lpan[i][r][k], S.Xpan[j][k][c], a0);
          a1 = fma(S.Lpan[i][r][k + 1], S.Xpan[j][k + 1][c], a1);
        }
        Xk[r][c] -= a0 + a1;
      }
    cl.sync();
  }
  // results: owned blocks of L and X (entries inside the leaf), then the
  // strict upper blocks are zeroed
  for (int q = rank; q < nq; q += kCC) {
    int i = 0;
    while ((i + 1) * (i + 2) / 2 <= q) ++i;
    const int j = q - i * (i + 1) / 2;
    const int gr = i * kCB + r, gc = j * kCB + c;
    if (gr < n && gc < n) {
      t.A[gr + (int64_t)gc * t.lda] = S.A[q / kCC][r][c];
      t.X[gr + (int64_t)gc * t.ldx] = (i != j || r >= c) ? S.X[q / kCC][r][c] : 0.0;
    }
  }
  for (int q = rank; q < NB * NB; q += kCC) {
    const int i = q % NB, j = q / NB;
    if (j <= i) continue;
    const int gr = i * kCB + r, gc = j * kCB + c;
    if (gr < n && gc < n) {
      t.A[gr + (int64_t)gc * t.lda] = 0.0;
      t.X[gr + (int64_t)gc * t.ldx] = 0.0;
    }
  }
}

// Li = L^{-1} for a lower-triangular leaf L (n <= kInvRows * 256).  CTA =
// (block of kInvCols identity columns, task); forward substitution L X = I
// restricted to those columns, which are zero above their first column c0,
// so the sweep starts at step c0.  Thread t owns rows t, t + 256, ...; its
// entries of the block stay in registers, and one pivot row per step goes
// through shared memory (double-buffered: one barrier per step).  Many
// small CTAs per leaf spread the n^3/3 flops over many SMs.
constexpr int kInvCols = 4;
constexpr int kInvRows = 4;

// Work of the forward substitution for identity column c of an n x n
// triangular inverse: one scaling and (n-c-1) multiply-adds per row below c.
__device__ __forceinline__ double inv_col_flops(int n, int c) {
  const double r = (double)(n - c);
  return r + r * (r - 1.0);
}

__device__ __forceinline__ void count_inv_flops(double* fc, int n, int c0) {
  if (fc && threadIdx.x == 0) {
    double f = 0.0;
    for (int c = c0; c < c0 + kInvCols && c < n; ++c) f += inv_col_flops(n, c);
    atomicAdd(fc, f);
  }
}

__global__ void __launch_bounds__(256) k_leaf_inv(const LeafTask* __restrict__ tasks, double* fc) {
  const LeafTask t = tasks[blockIdx.y];
  const int n = t.n;
  const int c0 = blockIdx.x * kInvCols;
  if (c0 >= n) return;
  count_inv_flops(fc, n, c0);
  const double* L = t.A;
  const int64_t lda = t.lda;
  __shared__ double dinv[kInvRows * 256];
  __shared__ double piv[2][kInvCols];
  for (int j = c0 + threadIdx.x; j < n; j += blockDim.x) dinv[j] = 1.0 / L[j + (int64_t)j * lda];
  double x[kInvRows][kInvCols];
#pragma unroll
  for (int r = 0; r < kInvRows; ++r)
#pragma unroll
    for (int c = 0; c < kInvCols; ++c) x[r][c] = (threadIdx.x + 256 * r == c0 + c) ? 1.0 : 0.0;
  double lcur[kInvRows];
#pragma unroll
  for (int r = 0; r < kInvRows; ++r) {
    const int i = threadIdx.x + 256 * r;
    lcur[r] = (i < n) ? L[i + (int64_t)c0 * lda] : 0.0;
  }
  __syncthreads();
  for (int j = c0; j < n; ++j) {
    const int owner = j & 255, slot = j >> 8;
    if (threadIdx.x == owner) {
      const double di = dinv[j];
#pragma unroll
      for (int r = 0; r < kInvRows; ++r)
        if (r == slot) {
#pragma unroll
          for (int c = 0; c < kInvCols; ++c) {
            x[r][c] *= di;
            piv[j & 1][c] = x[r][c];
          }
        }
    }
    __syncthreads();
    double lnext[kInvRows];
#pragma unroll
    for (int r = 0; r < kInvRows; ++r) {
      const int i = threadIdx.x + 256 * r;
      lnext[r] = (j + 1 < n && i < n) ? L[i + (int64_t)(j + 1) * lda] : 0.0;
    }
    double p[kInvCols];
#pragma unroll
    for (int c = 0; c < kInvCols; ++c) p[c] = piv[j & 1][c];
#pragma unroll
    for (int r = 0; r < kInvRows; ++r) {
      const int i = threadIdx.x + 256 * r;
      if (i > j && i < n) {
#pragma unroll
        for (int c = 0; c < kInvCols; ++c) x[r][c] = fma(-lcur[r], p[c], x[r][c]);
      }
      lcur[r] = lnext[r];
    }
  }
#pragma unroll
  for (int r = 0; r < kInvRows; ++r) {
    const int i = threadIdx.x + 256 * r;
    if (i < n)
#pragma unroll
      for (int c = 0; c < kInvCols; ++c)
        if (c0 + c < n) t.X[i + (int64_t)(c0 + c) * t.ldx] = x[r][c];
  }
}

// Same forward substitution as k_leaf_inv, with the part of L the block needs
// (columns c0..n-1, lower triangle) staged once in shared memory, packed by
// columns, so a step costs a shared-memory read and one barrier instead of a
// round trip to L2.  For leaves of at most kInvSmemRows rows.
constexpr int kInvSmemRows = 220;

__global__ void __launch_bounds__(256) k_leaf_inv_smem(const LeafTask* __restrict__ tasks, double* fc) {
  const LeafTask t = tasks[blockIdx.y];
  const int n = t.n;
  const int c0 = blockIdx.x * kInvCols;
  if (c0 >= n) return;
  count_inv_flops(fc, n, c0);
  const double* L = t.A;
  const int64_t lda = t.lda;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* Ls = reinterpret_cast<double*>(smem_raw);  // packed columns c0..n-1
  __shared__ double dinv[kInvSmemRows];
  __shared__ double piv[2][kInvCols];
  const int m = n - c0;
  // column j (j >= c0) holds rows j..n-1 at offset off(j) = sum_{t<j-c0} (m - t)
  for (int jj = threadIdx.x >> 5; jj < m; jj += blockDim.x >> 5) {
    const int64_t off = (int64_t)jj * m - (int64_t)jj * (jj - 1) / 2;
    const int j = c0 + jj;
    for (int i = j + (threadIdx.x & 31); i < n; i += 32) Ls[off + (i - j)] = L[i + (int64_t)j * lda];
  }
  __syncthreads();
  for (int jj = threadIdx.x; jj < m; jj += blockDim.x) {
    const int64_t off = (int64_t)jj * m - (int64_t)jj * (jj - 1) / 2;
    dinv[jj] = 1.0 / Ls[off];
  }
  const int i = threadIdx.x;  // one row per thread (n <= 220 < 256)
  double x[kInvCols];
#pragma unroll
  for (int c = 0; c < kInvCols; ++c) x[c] = (i == c0 + c) ? 1.0 : 0.0;
  __syncthreads();
  for (int j = c0; j < n; ++j) {
    const int jj = j - c0;
    if (i == j) {
      const double di = dinv[jj];
#pragma unroll
      for (int c = 0; c < kInvCols; ++c) {
        x[c] *= di;
        piv[j & 1][c] = x[c];
      }
    }
    __syncthreads();
    if (i > j && i < n) {
      const int64_t off = (int64_t)jj * m - (int64_t)jj * (jj - 1) / 2;
      const double l = Ls[off + (i - j)];
#pragma unroll
      for (int c = 0; c < kInvCols; ++c) x[c] = fma(-l, piv[j & 1][c], x[c]);
    }
  }
  if (i < n)
#pragma unroll
    for (int c = 0; c < kInvCols; ++c)
      if (c0 + c < n) t.X[i + (int64_t)(c0 + c) * t.ldx] = x[c];
}
}  // namespace

namespace {
// One GEMM launch (and its split-k reduction) over `tasks`, grid
// (tiles, tasks, nz), in parts of at most 65535 tasks.
void gemm_launch(sp_ctx* ctx, bool ta, bool tb, const std::vector<GemmTask>& tasks, int maxtiles, int te, int nz,
                 int kchunk, bool split, bool tc) {
  int64_t maxe = 1;
  for (const auto& t : tasks) maxe = std::max<int64_t>(maxe, (int64_t)t.m * t.n);
  for (size_t off = 0; off < tasks.size(); off += 65535) {
    const size_t cnt = std::min<size_t>(65535, tasks.size() - off);
    std::vector<GemmTask> part(tasks.begin() + off, tasks.begin() + off + cnt);
    DBuf d = upload(part, ctx->stream);
    dim3 grid(maxtiles, (unsigned)cnt, nz);
    const GemmTask* dt = d.as<GemmTask>();
    double* fc = fc_ptr(ctx, ctx->gemm_fp32 ? KID_GEMM_F32 : ctx->gemm_kid);
    ProfScope ps(ctx, ctx->gemm_fp32 ? KID_GEMM_F32 : ctx->gemm_kid);
    const int sp = split ? 1 : 0;
    if (tc) {
      launch_gemm_tc(ctx, ta, tb, grid, dt, kchunk, sp, fc);
    } else {
      if (!ta && !tb) k_gemm<false, false, double><<<grid, 256, 0, ctx->stream>>>(dt, kchunk, sp, te, fc);
      else if (ta && !tb) k_gemm<true, false, double><<<grid, 256, 0, ctx->stream>>>(dt, kchunk, sp, te, fc);
      else if (!ta && tb) k_gemm<false, true, double><<<grid, 256, 0, ctx->stream>>>(dt, kchunk, sp, te, fc);
      else k_gemm<true, true, double><<<grid, 256, 0, ctx->stream>>>(dt, kchunk, sp, te, fc);
    }
    check_launch("k_gemm");
  }
}

void splitk_reduce(sp_ctx* ctx, const std::vector<GemmTask>& tasks, int kchunk) {
  int64_t maxe = 1;
  for (const auto& t : tasks) maxe = std::max<int64_t>(maxe, (int64_t)t.m * t.n);
  for (size_t off = 0; off < tasks.size(); off += 65535) {
    const size_t cnt = std::min<size_t>(65535, tasks.size() - off);
    std::vector<GemmTask> part(tasks.begin() + off, tasks.begin() + off + cnt);
    DBuf d = upload(part, ctx->stream);
    const int gx = (int)std::min<int64_t>((maxe + 255) / 256, 1024);
    k_splitk_reduce<<<dim3(gx, (unsigned)cnt), 256, 0, ctx->stream>>>(d.as<GemmTask>(), kchunk);
    check_launch("k_splitk_reduce");
  }
}

// Tasks with a static k above this are cut into k ranges of at most this
// many rows (binary64 path): a coupling V^T X over a block of n/2 rows would
// otherwise walk its whole k range in one CTA -- a chain of n/32 dependent
// 16-deep k stages -- while the grid, sized from the rank capacities, looks
// large enough to skip the split-k below.
constexpr int kLongK = 512;
}  // namespace

void gemm_batched(sp_ctx* ctx, bool ta, bool tb, const std::vector<GemmTask>& tasks_in, int ksplit) {
  if (tasks_in.empty()) return;
  std::vector<GemmTask> tasks;
  tasks.reserve(tasks_in.size());
  int maxk = 0;
  for (const auto& t : tasks_in) {
    if (t.m <= 0 || t.n <= 0) continue;
    tasks.push_back(t);
    maxk = std::max(maxk, t.k);
    ctx->flops += 2.0 * t.m * (double)t.n * (double)t.k;
  }
  if (tasks.empty()) return;
  const bool tc = ctx->gemm_fp32;
  // long static k ranges: sub-tasks of at most kLongK rows, each writing its
  // own workspace slot; every task of the launch goes through the workspace
  // (one slot when not cut) and a second kernel sums a task's slots in order
  bool longk = false;
  if (!tc && ksplit <= 0)
    for (const auto& t : tasks) longk |= (!t.pk && t.k > kLongK);
  if (longk) {
    auto nsub = [](const GemmTask& t) { return (!t.pk && t.k > kLongK) ? (t.k + kLongK - 1) / kLongK : 1; };
    size_t tot = 0;
    for (const auto& t : tasks) tot += (size_t)nsub(t) * t.m * t.n;
    DBuf ws(tot * sizeof(double) + 16, ctx->stream);
    double* w = ws.as<double>();
    std::vector<GemmTask> sub, red;
    int maxtiles = 0, kch = 1;
    for (const auto& t : tasks) {
      const int ns = nsub(t);
      GemmTask r = t;
      r.W = w;
      r.nsplit = ns;
      red.push_back(r);
      for (int z = 0; z < ns; ++z) {
        GemmTask s = t;
        if (ns > 1) {
          const int kb = z * kLongK;
          s.k = std::min(kLongK, t.k - kb);
          s.A = ta ? t.A + kb : t.A + (int64_t)kb * t.lda;
          s.B = tb ? t.B + (int64_t)kb * t.ldb : t.B + kb;
        }
        s.W = w + (size_t)z * t.m * t.n;
        sub.push_back(s);
        kch = std::max(kch, s.k);
        maxtiles = std::max(maxtiles, ((t.m + kGT - 1) / kGT) * ((t.n + kGT - 1) / kGT));
      }
      w += (size_t)ns * t.m * t.n;
    }
    gemm_launch(ctx, ta, tb, sub, maxtiles, kGT, 1, kch, true, false);
    splitk_reduce(ctx, red, kch);
    return;
  }
  int maxtiles = 0;
  for (const auto& t : tasks) maxtiles = std::max(maxtiles, ((t.m + kGT - 1) / kGT) * ((t.n + kGT - 1) / kGT));
  int nz = 1, kchunk = std::max(maxk, 1);
  // binary64 runs at about 8 GFLOP/s per SM on this part, so a GEMM spread
  // over a few CTAs is compute-bound on a few SMs.  Small problems (fewer
  // 64 x 64 tiles than SMs) are laid out in 16 x 16 tiles instead, and k is
  // split (chunks of at least 32, resp. 64) until the grid covers the GPU.
  // The mixed-precision scope runs on the tensor cores in 128 x 64 tiles.
  int te = kGT;
  if (tc) {
    maxtiles = 0;
    for (const auto& t : tasks)
      maxtiles = std::max(maxtiles, ((t.m + gemm_tc_tile_rows() - 1) / gemm_tc_tile_rows()) *
                                        ((t.n + gemm_tc_tile_cols() - 1) / gemm_tc_tile_cols()));
  }
  int64_t ctas = (int64_t)maxtiles * (int64_t)tasks.size();
  if (!tc && ctx->small_tiles && ksplit <= 0 && ctas < ctx->num_sms) {
    te = 16;
    maxtiles = 0;
    for (const auto& t : tasks) maxtiles = std::max(maxtiles, ((t.m + 15) / 16) * ((t.n + 15) / 16));
    ctas = (int64_t)maxtiles * (int64_t)tasks.size();
  }
  const int kmin = (te == kGT || tc) ? 64 : 32;
  if (ksplit <= 0) {
    if (maxk >= 2 * kmin && ctas < 2 * ctx->num_sms) {
      nz = (int)std::min<int64_t>((4 * ctx->num_sms + ctas - 1) / ctas, maxk / kmin);
      nz = std::max(nz, 1);
    }
  } else {
    nz = std::max(1, ksplit);
  }
  if (nz > 1) {
    kchunk = ((maxk + nz - 1) / nz + kGK - 1) / kGK * kGK;
    nz = (maxk + kchunk - 1) / kchunk;
  }
  // split k: every chunk writes its partial tile into the task's workspace
  // slots (nz static m x n slots), a second kernel sums them in order
  DBuf ws;
  if (nz > 1) {
    size_t tot = 0;
    for (const auto& t : tasks) tot += (size_t)nz * t.m * t.n;
    ws = DBuf(tot * sizeof(double) + 16, ctx->stream);
    double* w = ws.as<double>();
    for (auto& t : tasks) {
      t.W = w;
      w += (size_t)nz * t.m * t.n;
    }
  }
  for (const auto& t : tasks)
    if (nz > 1 && !t.W) fail(SP_EINTERNAL, "split-k GEMM without a workspace");
  gemm_launch(ctx, ta, tb, tasks, maxtiles, te, nz, kchunk, nz > 1, tc);
  if (nz > 1) splitk_reduce(ctx, tasks, kchunk);
}

void axpby_batched(sp_ctx* ctx, const std::vector<AxpbyTask>& tasks) {
  if (tasks.empty()) return;
  int64_t maxe = 1;
  for (const auto& t : tasks) maxe = std::max<int64_t>(maxe, (int64_t)t.m * t.n);
  for (size_t off = 0; off < tasks.size(); off += 65535) {
    const size_t cnt = std::min<size_t>(65535, tasks.size() - off);
    std::vector<AxpbyTask> part(tasks.begin() + off, tasks.begin() + off + cnt);
    DBuf d = upload(part, ctx->stream);
    const int gx = (int)std::min<int64_t>((maxe + 255) / 256, 1024);
    k_axpby<<<dim3(gx, (unsigned)cnt), 256, 0, ctx->stream>>>(d.as<AxpbyTask>());
    check_launch("k_axpby");
  }
}

void zero_tail_batched(sp_ctx* ctx, const std::vector<ZeroTailTask>& tasks) {
  if (tasks.empty()) return;
  int64_t maxe = 1;
  for (const auto& t : tasks) maxe = std::max<int64_t>(maxe, (int64_t)t.m * t.cap);
  for (size_t off = 0; off < tasks.size(); off += 65535) {
    const size_t cnt = std::min<size_t>(65535, tasks.size() - off);
    std::vector<ZeroTailTask> part(tasks.begin() + off, tasks.begin() + off + cnt);
    DBuf d = upload(part, ctx->stream);
    const int gx = (int)std::min<int64_t>((maxe + 255) / 256, 1024);
    k_zero_tail<<<dim3(gx, (unsigned)cnt), 256, 0, ctx->stream>>>(d.as<ZeroTailTask>());
    check_launch("k_zero_tail");
  }
}

void check_finite(sp_ctx* ctx, const double* p, size_t count) {
  if (!p || count == 0) return;
  const int grid = (int)std::min<size_t>((count + 255) / 256, (size_t)ctx->num_sms * 8);
  k_nonfinite<<<grid, 256, 0, ctx->stream>>>(p, count, ctx->d_flags);
  check_launch("k_nonfinite");
}

void leaf_potrf(sp_ctx* ctx, const std::vector<LeafTask>& tasks) {
  if (tasks.empty()) return;
  for (const auto& t : tasks) ctx->flops += (double)t.n * t.n * t.n / 3.0;
  DBuf d = upload(tasks, ctx->stream);
  int nmax = 1;
  for (const auto& t : tasks) nmax = std::max(nmax, t.n);
  const size_t sm = (size_t)nmax * (kPW + 1) * sizeof(double);
  ensure_dynamic_smem(reinterpret_cast<const void*>(k_leaf_potrf), sm);
  ProfScope ps(ctx, KID_POTRF);
  k_leaf_potrf<<<(unsigned)tasks.size(), 1024, sm, ctx->stream>>>(d.as<LeafTask>(), ctx->d_flags,
                                                                   fc_ptr(ctx, KID_POTRF));
  check_launch("k_leaf_potrf");
}

bool leaf_chol_inv(sp_ctx* ctx, const std::vector<LeafTask>& tasks) {
  if (tasks.empty()) return true;
  for (const auto& t : tasks)
    if (t.n > kCMaxN || !t.X) return false;
  for (const auto& t : tasks) ctx->flops += 2.0 * (double)t.n * t.n * t.n / 3.0;
  for (size_t off = 0; off < tasks.size(); off += 65535) {
    const size_t cnt = std::min<size_t>(65535, tasks.size() - off);
    std::vector<LeafTask> part(tasks.begin() + off, tasks.begin() + off + cnt);
    DBuf d = upload(part, ctx->stream);
    ProfScope ps(ctx, KID_LEAF_CLUSTER);
    k_leaf_chol_inv_cluster<<<dim3(kCC, (unsigned)cnt), 256, sizeof(ClusterSmem), ctx->stream>>>(
        d.as<LeafTask>(), ctx->d_flags, fc_ptr(ctx, KID_LEAF_CLUSTER), fc_ptr(ctx, KID_LEAF_CLUSTER));
    check_launch("k_leaf_chol_inv_cluster");
  }
  return true;
}

void leaf_inverse_batched(sp_ctx* ctx, const std::vector<LeafTask>& tasks) {
  if (tasks.empty()) return;
  int maxn = 0;
  for (const auto& t : tasks) {
    if (t.n > kInvRows * 256) fail(SP_EINVAL, "leaf inverse: leaf larger than 1024 rows");
    maxn = std::max(maxn, t.n);
  }
  const bool staged = maxn <= kInvSmemRows;
  const size_t sm = staged ? (size_t)maxn * (maxn + 1) / 2 * sizeof(double) : 0;
  if (staged) ensure_dynamic_smem(reinterpret_cast<const void*>(k_leaf_inv_smem), sm);
  for (size_t off = 0; off < tasks.size(); off += 65535) {
    const size_t cnt = std::min<size_t>(65535, tasks.size() - off);
    std::vector<LeafTask> part(tasks.begin() + off, tasks.begin() + off + cnt);
    DBuf d = upload(part, ctx->stream);
    dim3 grid((maxn + kInvCols - 1) / kInvCols, (unsigned)cnt);
    ProfScope ps(ctx, KID_LEAF_INV);
    if (staged) {
      k_leaf_inv_smem<<<grid, 256, sm, ctx->stream>>>(d.as<LeafTask>(), fc_ptr(ctx, KID_LEAF_INV));
      check_launch("k_leaf_inv_smem");
    } else {
      k_leaf_inv<<<grid, 256, 0, ctx->stream>>>(d.as<LeafTask>(), fc_ptr(ctx, KID_LEAF_INV));
      check_launch("k_leaf_inv");
    }
  }
}

void configure_blas_kernels() {
  configure_dynamic_smem(reinterpret_cast<const void*>(k_leaf_chol_inv_cluster));
  configure_dynamic_smem(reinterpret_cast<const void*>(k_leaf_potrf));
  configure_dynamic_smem(reinterpret_cast<const void*>(k_leaf_inv_smem));
}

}  // namespace sp
