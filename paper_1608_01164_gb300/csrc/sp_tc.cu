// sp_tc.cu -- the mixed-precision GEMMs on the 5th-generation tensor cores.
//
// The late Cholesky-based / Newton-Schulz steps of the mixed-precision modes
// (residual form, see sp_api.cu) run their dense products C = alpha op(A)
// op(B) + beta C on the tensor cores with binary32 accumulation (not part of
// the paper: a precision growth direction).  Here
// every binary64 operand x is split into three bfloat16 slices
//   x1 = bf16(x), x2 = bf16(x - x1), x3 = bf16(x - x1 - x2)
// (the residuals taken in binary32 after one rounding of x to binary32), so
// x = x1 + x2 + x3 to about 2^-24 relative, and the product keeps the six
// slice products of order up to 2^-16:
//   A B ~ A1 B1 + A1 B2 + A2 B1 + A1 B3 + A2 B2 + A3 B1,
// all accumulated by tcgen05.mma (kind::f16, bf16 x bf16 -> f32) into one
// FP32 accumulator in tensor memory: binary32-level accuracy.
//
// CTA tile: 128 rows x 64 columns of C (UMMA M = 128, N = 64, cta_group::1),
// k in chunks of 16.  128 threads stage the six operand slices of a chunk
// into shared memory in the canonical no-swizzle K-major layout (8-row x
// 16-byte core matrices), double-buffered; one thread issues the six MMAs and
// commits them to the stage's mbarrier; the epilogue reads the accumulator
// with tcgen05.ld (warp w owns lanes 32w..32w+31 = rows) and applies alpha,
// beta (or writes the k chunk's partial tile for the ordered split-k sum).
// Every mbarrier wait is bounded: on expiry the kernel sets the timeout flag,
// waits once more (bounded), frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "sp_internal.h"

namespace sp {
namespace {

constexpr int kTM = 128;  // tile rows (UMMA M)
constexpr int kTN = 64;   // tile columns (UMMA N), TMEM columns
constexpr int kTK = 16;   // k per MMA (bf16)
constexpr int kASlice = kTM * kTK * 2;  // bytes of one A slice (4 KB)
constexpr int kBSlice = kTN * kTK * 2;  // bytes of one B slice (2 KB)
constexpr int kStage = 3 * kASlice + 3 * kBSlice;
constexpr long kWaitLimit = 1l << 24;  // try_wait polls before a wait gives up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor, no swizzle: K-adjacent core matrices LBO
// bytes apart, 8-row groups SBO bytes apart
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // fixed constant 0b001 in bits 46-48
  return d;
}

// byte offset of (row r, k) in a rows x 16 bf16 K-major tile: core matrix
// (r / 8, k / 8) at (r / 8) * 256 + (k / 8) * 128, row r % 8 at 16 B steps
__device__ __forceinline__ int tile_off(int r, int k) { return (r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

__device__ __forceinline__ int dsz(int s, const int* p) {
  if (p) {
    int v = *p;
    v = v < 0 ? 0 : v;
    return v < s ? v : s;
  }
  return s;
}

__device__ __forceinline__ void split3(double x, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
  const float f = (float)x;
  a = __float2bfloat16_rn(f);
  const float r1 = f - __bfloat162float(a);
  b = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(b);
  c = __float2bfloat16_rn(r2);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  for (long it = 0; it < kWaitLimit && !done; ++it)
    asm volatile(
        "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
  return done != 0;
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(128) k_gemm_tc(const GemmTask* __restrict__ tasks, int kchunk, int split,
                                                 double* fc, int* flags) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  const GemmTask t = tasks[blockIdx.y];
  const int m = dsz(t.m, t.pm), n = dsz(t.n, t.pn), k = dsz(t.k, t.pk);
  const int tiles_m = (m + kTM - 1) / kTM;
  const int tile = blockIdx.x;
  if (tile >= tiles_m * ((n + kTN - 1) / kTN)) return;  // whole CTA exits before any tcgen05 op
  const int row0 = (tile % tiles_m) * kTM, col0 = (tile / tiles_m) * kTN;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(k, kbeg + kchunk);
  if (kbeg >= kend && blockIdx.z > 0) return;
  const int nch = kend > kbeg ? (kend - kbeg + kTK - 1) / kTK : 0;
  const int tid = threadIdx.x, warp = tid >> 5;
  // align the dynamic buffer to 1 KB inside the allocation
  unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  // D f32, A and B bf16, both K-major, N = 64, M = 128
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTN >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
  bool ok = true;
  for (int ci = 0; ci < nch && ok; ++ci) {
    const int s = ci & 1;
    unsigned char* st = base + s * kStage;
    // the MMAs that read this stage two chunks ago must be done (one vote for
    // the whole CTA keeps the barriers below uniform)
    if (ci >= 2) ok = __syncthreads_and(mbar_wait(smem_u32(&mbar[s]), (uint32_t)(((ci - 2) >> 1) & 1)));
    if (!ok) break;
    const int kb = kbeg + ci * kTK;
    // A: element (r, kk) of op(A) = A(r, kk) (or A^T)
    for (int e = tid; e < kTM * kTK; e += 128) {
      int r, kk;
      if (!TA) { r = e % kTM; kk = e / kTM; } else { kk = e % kTK; r = e / kTK; }
      const int gr = row0 + r, gk = kb + kk;
      double v = 0.0;
      if (gr < m && gk < kend) v = TA ? t.A[gk + (int64_t)gr * t.lda] : t.A[gr + (int64_t)gk * t.lda];
      __nv_bfloat16 x1, x2, x3;
      split3(v, x1, x2, x3);
      const int o = tile_off(r, kk);
      *reinterpret_cast<__nv_bfloat16*>(st + o) = x1;
      *reinterpret_cast<__nv_bfloat16*>(st + kASlice + o) = x2;
      *reinterpret_cast<__nv_bfloat16*>(st + 2 * kASlice + o) = x3;
    }
    // B: element (kk, c) of op(B), stored as row c of the N x K operand
    unsigned char* sb = st + 3 * kASlice;
    for (int e = tid; e < kTN * kTK; e += 128) {
      int c, kk;
      if (!TB) { kk = e % kTK; c = e / kTK; } else { c = e % kTN; kk = e / kTN; }
      const int gc = col0 + c, gk = kb + kk;
      double v = 0.0;
      if (gc < n && gk < kend) v = TB ? t.B[gc + (int64_t)gk * t.ldb] : t.B[gk + (int64_t)gc * t.ldb];
      __nv_bfloat16 x1, x2, x3;
      split3(v, x1, x2, x3);
      const int o = tile_off(c, kk);
      *reinterpret_cast<__nv_bfloat16*>(sb + o) = x1;
      *reinterpret_cast<__nv_bfloat16*>(sb + kBSlice + o) = x2;
      *reinterpret_cast<__nv_bfloat16*>(sb + 2 * kBSlice + o) = x3;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = smem_u32(st), b0 = smem_u32(sb);
      // slice pairs (i, j) with i + j <= 4 (1-based): 11, 12, 21, 13, 22, 31
      const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const uint64_t ad = sdesc(a0 + pa[q] * kASlice, 128, 256);
        const uint64_t bd = sdesc(b0 + pb[q] * kBSlice, 128, 256);
        const uint32_t acc = (ci > 0 || q > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&mbar[s]))
                   : "memory");
    }
  }
  // all MMAs done: the last commit covers every earlier one
  if (ok && nch > 0)
    ok = __syncthreads_and(mbar_wait(smem_u32(&mbar[(nch - 1) & 1]), (uint32_t)(((nch - 1) >> 1) & 1)));
  if (!ok) {
    if (tid == 0) atomicOr(&flags[FLAG_TIMEOUT], 1);
    if (nch > 0) (void)mbar_wait(smem_u32(&mbar[(nch - 1) & 1]), (uint32_t)(((nch - 1) >> 1) & 1));
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    const int row = row0 + 32 * warp + (tid & 31);
    double* W = split ? t.W + (size_t)blockIdx.z * (size_t)t.m * (size_t)t.n : nullptr;
#pragma unroll 1
    for (int c0 = 0; c0 < kTN; c0 += 16) {
      uint32_t v[16];
      if (nch > 0) {
        const uint32_t ta = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0u;
      }
      if (row < m) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int gc = col0 + c0 + j;
          if (gc < n) {
            const double val = t.alpha * (double)__uint_as_float(v[j]);
            if (W) {
              W[row + (int64_t)gc * t.m] = val;
            } else {
              double* p = t.C + row + (int64_t)gc * t.ldc;
              *p = (t.beta == 0.0) ? val : val + t.beta * (*p);
            }
          }
        }
      }
    }
    if (fc && tid == 0)
      atomicAdd(fc, 2.0 * (double)min(kTM, m - row0) * (double)min(kTN, n - col0) * (double)(kend - kbeg));
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTN));
}

}  // namespace

size_t gemm_tc_smem() { return 2 * (size_t)kStage + 1024; }
int gemm_tc_tile_rows() { return kTM; }
int gemm_tc_tile_cols() { return kTN; }

void launch_gemm_tc(sp_ctx* ctx, bool ta, bool tb, dim3 grid, const GemmTask* tasks, int kchunk, int split,
                    double* fc) {
  const size_t sm = gemm_tc_smem();
  if (!ta && !tb) k_gemm_tc<false, false><<<grid, 128, sm, ctx->stream>>>(tasks, kchunk, split, fc, ctx->d_flags);
  else if (ta && !tb) k_gemm_tc<true, false><<<grid, 128, sm, ctx->stream>>>(tasks, kchunk, split, fc, ctx->d_flags);
  else if (!ta && tb) k_gemm_tc<false, true><<<grid, 128, sm, ctx->stream>>>(tasks, kchunk, split, fc, ctx->d_flags);
  else k_gemm_tc<true, true><<<grid, 128, sm, ctx->stream>>>(tasks, kchunk, split, fc, ctx->d_flags);
  check_launch("k_gemm_tc");
}

void configure_tc_kernels() {
  configure_dynamic_smem(reinterpret_cast<const void*>(k_gemm_tc<false, false>));
  configure_dynamic_smem(reinterpret_cast<const void*>(k_gemm_tc<true, false>));
  configure_dynamic_smem(reinterpret_cast<const void*>(k_gemm_tc<false, true>));
  configure_dynamic_smem(reinterpret_cast<const void*>(k_gemm_tc<true, true>));
}

}  // namespace sp
