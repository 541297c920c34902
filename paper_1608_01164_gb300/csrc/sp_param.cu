// sp_param.cu -- inertia counts and the QDWH start parameters.
//
// The paper starts QDWH with alpha ~ ||A||_2 and l0 ~ sigma_min(A/alpha)
// (Sec. 5, Eq. (param_estimation)).  QDWH needs alpha >= ||A - mu I||_2 and
// l0 <= sigma_min((A - mu I)/alpha); both follow from eigenvalue brackets, and
// brackets follow from inertia counts nu(sigma) = #{lambda < sigma}
// (Sylvester's law of inertia on A - sigma I = L D L^T).  Tridiagonal: one
// thread per shift runs the Sturm recurrence d_i = (a_i - sigma) -
// e_{i-1}^2 / d_{i-1}.  Banded, 2 <= b <= 80: one warp per shift runs the
// unpivoted banded LDL^T with the (b+1)^2 Schur window in shared memory; wider
// bands: one thread per shift with the last b columns of L in a ring.  A count
// is a sequential chain of n dependent steps, so many shifts run side by side.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "sp_internal.h"

namespace sp {
namespace {

// widest band handled by the warp-per-shift count (4 windows of (b+1)^2 doubles
// per 128-thread CTA must fit in shared memory)
constexpr int kWarpInertiaMaxB = 80;

// Algorithmic work of one inertia count: tridiagonal, per row a shift, a
// square, a divide and a subtraction; banded (LDL^T of bandwidth b), per row
// b(b+1)/2 Schur updates of 3 flops, the b multipliers and the pivot.
__host__ __device__ inline double inertia_flops(int64_t n, int b) {
  if (b <= 0) return (double)n;
  if (b == 1) return 4.0 * (double)n;
  return (double)n * (1.5 * b * (b + 1.0) + b + 1.0);
}

__global__ void k_inertia(const double* __restrict__ ab, int64_t ldab, int64_t n, int b,
                          const double* __restrict__ shifts, int nshift, int64_t* __restrict__ counts, double pivmin,
                          double* __restrict__ ring, double* fc) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nshift) return;
  if (fc) atomicAdd(fc, inertia_flops(n, b));
  const double sigma = shifts[t];
  int64_t cnt = 0;
  if (b == 1) {
    double d = 1.0;
    for (int64_t i = 0; i < n; ++i) {
      const double e = (i == 0) ? 0.0 : ab[1 + (i - 1) * ldab];
      d = (ab[i * ldab] - sigma) - ((i == 0) ? 0.0 : e * e / d);
      if (fabs(d) < pivmin) d = -pivmin;
      cnt += d < 0.0;
    }
  } else if (b == 0) {
    for (int64_t i = 0; i < n; ++i) cnt += ab[i * ldab] < sigma;
  } else {
    // ring: column k of L (entries L(k+1..k+b, k)) at slot k % b, plus D_k
    double* Lr = ring + (size_t)t * (b * b + b);
    double* Dr = Lr + b * b;
    for (int64_t j = 0; j < n; ++j) {
      double dj = ab[j * ldab] - sigma;
      const int64_t k0 = j - b > 0 ? j - b : 0;
      for (int64_t k = k0; k < j; ++k) {
        const double l = Lr[(k % b) * b + (j - k - 1)];
        dj -= l * l * Dr[k % b];
      }
      if (fabs(dj) < pivmin) dj = -pivmin;
      cnt += dj < 0.0;
      const double inv = 1.0 / dj;
      double* Lj = Lr + (j % b) * b;
      for (int64_t i = j + 1; i <= j + b; ++i) {
        double s = (i < n) ? ab[(i - j) + j * ldab] : 0.0;
        const int64_t kk0 = i - b > 0 ? i - b : 0;
        for (int64_t k = kk0; k < j; ++k) s -= Lr[(k % b) * b + (i - k - 1)] * Lr[(k % b) * b + (j - k - 1)] * Dr[k % b];
        Lj[i - j - 1] = s * inv;
      }
      Dr[j % b] = dj;
    }
  }
  counts[t] = cnt;
}

// Banded LDL^T count with one warp per shift (b >= 2).  The trailing
// (b+1) x (b+1) window of the Schur complement of A - sigma I is kept, both
// triangles, in shared memory as a ring over row/column indices (global index
// r lives in slot r mod (b+1)).  Step j: pivot d_j = S(j, j); every lane
// updates its share of the b^2 entries S(r, c) -= S(r, j) S(c, j) / d_j,
// r, c in (j, j+b]; then row/column j+b+1 of A enters the slot of j.  Same
// arithmetic as the per-thread ring above, summed in a different order.
__global__ void __launch_bounds__(128) k_inertia_warp(const double* __restrict__ ab, int64_t ldab, int64_t n, int b,
                                                      const double* __restrict__ shifts, int nshift,
                                                      int64_t* __restrict__ counts, double pivmin, double* fc) {
  extern __shared__ double win_all[];
  const int W = b + 1;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int t = blockIdx.x * (blockDim.x >> 5) + wib;
  if (t >= nshift) return;  // whole warps exit together
  if (fc && lane == 0) atomicAdd(fc, inertia_flops(n, b));
  double* S = win_all + (size_t)wib * W * W;
  const double sigma = shifts[t];
  // window rows/columns 0..b
  for (int e = lane; e < W * W; e += 32) {
    const int r = e / W, c = e % W;
    double v = 0.0;
    if (r < n && c < n) {
      const int hi = r > c ? r : c, lo = r > c ? c : r;
      if (hi - lo <= b) v = ab[(hi - lo) + (int64_t)lo * ldab];
      if (r == c) v -= sigma;
    }
    S[e] = v;
  }
  __syncwarp();
  int64_t cnt = 0;
  int sj = 0;  // slot of row j
  for (int64_t j = 0; j < n; ++j) {
    double d = S[sj * W + sj];
    if (fabs(d) < pivmin) d = -pivmin;
    cnt += d < 0.0;
    double inv = 0.0;
    if (lane == 0) inv = 1.0 / d;  // one divide per step, not 32
    inv = __shfl_sync(0xffffffffu, inv, 0);
    const int lim = (int)((n - 1 - j) < b ? (n - 1 - j) : b);  // rows j+1..j+lim exist
    for (int e = lane; e < lim * lim; e += 32) {
      const int ro = e / lim + 1, co = e % lim + 1;
      int sr = sj + ro, sc = sj + co;
      if (sr >= W) sr -= W;
      if (sc >= W) sc -= W;
      S[sr * W + sc] -= S[sr * W + sj] * S[sc * W + sj] * inv;
    }
    __syncwarp();
    // row/column j+b+1 of A - sigma I into slot sj
    const int64_t r = j + b + 1;
    if (r < n) {
      for (int co = lane; co <= b; co += 32) {
        const int64_t c = j + 1 + co;  // c in [j+1, r]
        double v = ab[(r - c) + c * ldab];
        if (c == r) v -= sigma;
        int sc = sj + 1 + co;
        if (sc >= W) sc -= W;
        S[sj * W + sc] = v;
        S[sc * W + sj] = v;
      }
    }
    __syncwarp();
    sj = (sj + 1 == W) ? 0 : sj + 1;
  }
  if (lane == 0) counts[t] = cnt;
}

__global__ void k_gershgorin(const double* __restrict__ ab, int64_t ldab, int64_t n, int b, double* out) {
  double lo = 1e300, hi = -1e300;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double r = 0.0;
    for (int d = 1; d <= b; ++d) {
      if (i + d < n) r += fabs(ab[d + i * ldab]);
      if (i - d >= 0) r += fabs(ab[d + (i - d) * ldab]);
    }
    lo = fmin(lo, ab[i * ldab] - r);
    hi = fmax(hi, ab[i * ldab] + r);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    const int w = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    out[2 * w] = lo;
    out[2 * w + 1] = hi;
  }
}

__global__ void k_absmax(const double* __restrict__ ab, int64_t ldab, int64_t n, int b, double* out) {
  double m = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int d = 0; d <= b; ++d)
      if (i + d < n) m = fmax(m, fabs(ab[d + i * ldab]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) out[blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32] = m;
}

// ---- no-allocation variant: scratch in a file-scope device array ----------
// Layout: [0, 512) absmax partials of k_absmax, [512] pivmin, [520, ...)
// per-shift LDL^T rings.
__device__ __align__(256) double g_noalloc_scratch[SP_NOALLOC_SCRATCH_DOUBLES];

__global__ void k_pivmin_from_partials(double* scratch, int nparts) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double amax = 1.0;
    for (int i = 0; i < nparts; ++i) amax = fmax(amax, scratch[i]);
    scratch[512] = DBL_MIN * amax * amax;
  }
}

// The scratch is written (per-shift rings) and read back by the same thread,
// so it is a plain pointer: no const/__restrict__ that would allow loads
// through the read-only data path.
__global__ void k_inertia_noalloc(const double* __restrict__ ab, int64_t ldab, int64_t n, int b,
                                  const double* __restrict__ shifts, int nshift, int64_t* __restrict__ counts,
                                  double* scratch) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nshift) return;
  const double pivmin = scratch[512];
  const double sigma = shifts[t];
  int64_t cnt = 0;
  if (b == 1) {
    double d = 1.0;
    for (int64_t i = 0; i < n; ++i) {
      const double e = (i == 0) ? 0.0 : ab[1 + (i - 1) * ldab];
      d = (ab[i * ldab] - sigma) - ((i == 0) ? 0.0 : e * e / d);
      if (fabs(d) < pivmin) d = -pivmin;
      cnt += d < 0.0;
    }
  } else if (b == 0) {
    for (int64_t i = 0; i < n; ++i) cnt += ab[i * ldab] < sigma;
  } else {
    double* Lr = scratch + 520 + (size_t)t * (b * b + b);
    double* Dr = Lr + b * b;
    for (int64_t j = 0; j < n; ++j) {
      double dj = ab[j * ldab] - sigma;
      const int64_t k0 = j - b > 0 ? j - b : 0;
      for (int64_t k = k0; k < j; ++k) {
        const double l = Lr[(k % b) * b + (j - k - 1)];
        dj -= l * l * Dr[k % b];
      }
      if (fabs(dj) < pivmin) dj = -pivmin;
      cnt += dj < 0.0;
      const double inv = 1.0 / dj;
      double* Lj = Lr + (j % b) * b;
      for (int64_t i = j + 1; i <= j + b; ++i) {
        double s = (i < n) ? ab[(i - j) + j * ldab] : 0.0;
        const int64_t kk0 = i - b > 0 ? i - b : 0;
        for (int64_t k = kk0; k < j; ++k) s -= Lr[(k % b) * b + (i - k - 1)] * Lr[(k % b) * b + (j - k - 1)] * Dr[k % b];
        Lj[i - j - 1] = s * inv;
      }
      Dr[j % b] = dj;
    }
  }
  counts[t] = cnt;
}

}  // namespace

// Device address of the no-allocation scratch on the current device, looked
// up once per device (the host-side symbol is only a stand-in).
double* noalloc_scratch_ptr() {
  static std::mutex mu;
  static double* ptrs[64] = {};
  int dev = 0;
  check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= 64) fail(SP_EINVAL, "device ordinal out of range for the no-allocation scratch");
  std::lock_guard<std::mutex> lk(mu);
  if (!ptrs[dev]) {
    void* p = nullptr;
    check_cuda(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(no-allocation scratch)");
    ptrs[dev] = static_cast<double*>(p);
  }
  return ptrs[dev];
}

void inertia_counts_noalloc(sp_ctx* ctx, int64_t n, int b, const double* ab_dev, int64_t ldab, int nshift,
                            const double* shifts_dev, int64_t* counts_dev) {
  const size_t need = 520 + (b > 1 ? (size_t)nshift * ((size_t)b * b + b) : 0);
  if (need > (size_t)SP_NOALLOC_SCRATCH_DOUBLES)
    fail(SP_EINVAL, "sp_inertia_noalloc: nshift * (b*b + b) + 520 = " + std::to_string(need) +
                        " doubles exceeds the scratch of " + std::to_string(SP_NOALLOC_SCRATCH_DOUBLES));
  if (nshift <= 0) return;
  double* scratch = noalloc_scratch_ptr();
  k_absmax<<<64, 256, 0, ctx->stream>>>(ab_dev, ldab, n, b, scratch);
  check_launch("k_absmax");
  k_pivmin_from_partials<<<1, 32, 0, ctx->stream>>>(scratch, 64 * (256 / 32));
  check_launch("k_pivmin_from_partials");
  k_inertia_noalloc<<<(nshift + 63) / 64, 64, 0, ctx->stream>>>(ab_dev, ldab, n, b, shifts_dev, nshift, counts_dev,
                                                                scratch);
  check_launch("k_inertia_noalloc");
}

// counts_dev[i] = #{lambda < shifts_dev[i]} (device arrays)
void inertia_counts(sp_ctx* ctx, int64_t n, int b, const double* ab_dev, int64_t ldab, int nshift,
                    const double* shifts_dev, int64_t* counts_dev) {
  if (nshift <= 0) return;
  // pivmin = DBL_MIN * max(1, max|a_ij|^2)
  const int gb = 64, tb = 256;
  DBuf part((size_t)gb * (tb / 32) * sizeof(double), ctx->stream);
  k_absmax<<<gb, tb, 0, ctx->stream>>>(ab_dev, ldab, n, b, part.as<double>());
  check_launch("k_absmax");
  std::vector<double> h(gb * (tb / 32));
  check_cuda(cudaMemcpyAsync(h.data(), part.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "cp");
  check_cuda(cudaStreamSynchronize(ctx->stream), "sync");
  double amax = 1.0;
  for (double v : h) amax = std::max(amax, v);
  const double pivmin = DBL_MIN * amax * amax;
  if (b >= 2 && b <= kWarpInertiaMaxB) {
    const size_t sm = (size_t)4 * (b + 1) * (b + 1) * sizeof(double);
    ensure_dynamic_smem(reinterpret_cast<const void*>(k_inertia_warp), sm);
    ProfScope ps(ctx, KID_INERTIA);
    k_inertia_warp<<<(nshift + 3) / 4, 128, sm, ctx->stream>>>(ab_dev, ldab, n, b, shifts_dev, nshift, counts_dev,
                                                               pivmin, fc_ptr(ctx, KID_INERTIA));
    check_launch("k_inertia_warp");
    return;
  }
  DBuf ring(b > 1 ? (size_t)nshift * (b * b + b) * sizeof(double) : 16, ctx->stream);
  ProfScope ps(ctx, KID_INERTIA);
  k_inertia<<<(nshift + 63) / 64, 64, 0, ctx->stream>>>(ab_dev, ldab, n, b, shifts_dev, nshift, counts_dev, pivmin,
                                                        ring.as<double>(), fc_ptr(ctx, KID_INERTIA));
  check_launch("k_inertia");
}

// Gershgorin interval of the band (device input), synchronising.
void gershgorin(sp_ctx* ctx, int64_t n, int b, const double* ab_dev, int64_t ldab, double* lo, double* hi) {
  const int gb = 64, tb = 256;
  DBuf part((size_t)gb * (tb / 32) * 2 * sizeof(double), ctx->stream);
  k_gershgorin<<<gb, tb, 0, ctx->stream>>>(ab_dev, ldab, n, b, part.as<double>());
  check_launch("k_gershgorin");
  std::vector<double> h(gb * (tb / 32) * 2);
  check_cuda(cudaMemcpyAsync(h.data(), part.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "cp");
  check_cuda(cudaStreamSynchronize(ctx->stream), "sync");
  double l = 1e300, u = -1e300;
  for (size_t i = 0; i < h.size(); i += 2) {
    l = std::min(l, h[i]);
    u = std::max(u, h[i + 1]);
  }
  *lo = l;
  *hi = u;
}

// Host-side multisection driver: evaluates counts at a batch of shifts.
static std::vector<int64_t> counts_at(sp_ctx* ctx, int64_t n, int b, const double* ab_dev, int64_t ldab,
                                      const std::vector<double>& x) {
  DBuf sx = upload(x, ctx->stream);
  DBuf cn(x.size() * sizeof(int64_t) + 8, ctx->stream);
  inertia_counts(ctx, n, b, ab_dev, ldab, (int)x.size(), sx.as<double>(), cn.as<int64_t>());
  std::vector<int64_t> h(x.size());
  check_cuda(cudaMemcpyAsync(h.data(), cn.p, h.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream), "cp");
  check_cuda(cudaStreamSynchronize(ctx->stream), "sync");
  return h;
}

// Brackets [x_k, y_k) of lambda_k for each requested k (1-based) by
// multisection: count(x) < k <= count(y).  rel: stop when y - x <= rel*scale.
static void bracket(sp_ctx* ctx, int64_t n, int b, const double* ab_dev, int64_t ldab, const std::vector<int64_t>& ks,
                    double glo, double ghi, double rel, std::vector<double>& xs, std::vector<double>& ys) {
  const int P = 255;  // interior points per bracket and round
  const size_t K = ks.size();
  xs.assign(K, glo);
  ys.assign(K, ghi);
  const double scale = std::max({1.0, std::fabs(glo), std::fabs(ghi)});
  for (int round = 0; round < 12; ++round) {
    std::vector<double> pts;
    std::vector<size_t> owner;
    for (size_t k = 0; k < K; ++k) {
      if (ys[k] - xs[k] <= rel * scale) continue;
      for (int p = 1; p <= P; ++p) {
        pts.push_back(xs[k] + (ys[k] - xs[k]) * p / (P + 1));
        owner.push_back(k);
      }
    }
    if (pts.empty()) break;
    std::vector<int64_t> c = counts_at(ctx, n, b, ab_dev, ldab, pts);
    for (size_t t = 0; t < pts.size(); ++t) {
      const size_t k = owner[t];
      if (c[t] >= ks[k]) ys[k] = std::min(ys[k], pts[t]);
      else xs[k] = std::max(xs[k], pts[t]);
    }
  }
}

void locate_shift(sp_ctx* ctx, int64_t n, int b, const double* ab_dev, int64_t ldab, int64_t nu, double* mu,
                  double* lam_nu_hi, double* lam_nu1_lo) {
  double glo, ghi;
  gershgorin(ctx, n, b, ab_dev, ldab, &glo, &ghi);
  const double pad = 1e-12 * std::max({1.0, std::fabs(glo), std::fabs(ghi)});
  glo -= pad;
  ghi += pad;
  if (nu <= 0) {
    std::vector<double> x, y;
    bracket(ctx, n, b, ab_dev, ldab, {1}, glo, ghi, 1e-3, x, y);
    *mu = x[0] - 1.0;
    *lam_nu_hi = *mu;
    *lam_nu1_lo = x[0];
    return;
  }
  if (nu >= n) {
    std::vector<double> x, y;
    bracket(ctx, n, b, ab_dev, ldab, {n}, glo, ghi, 1e-3, x, y);
    *mu = y[0] + 1.0;
    *lam_nu_hi = y[0];
    *lam_nu1_lo = *mu;
    return;
  }
  std::vector<double> x, y;
  bracket(ctx, n, b, ab_dev, ldab, {nu, nu + 1}, glo, ghi, 1e-15, x, y);
  *lam_nu_hi = y[0];
  *lam_nu1_lo = x[1];
  *mu = 0.5 * (y[0] + x[1]);
  std::vector<int64_t> c = counts_at(ctx, n, b, ab_dev, ldab, {*mu});
  if (c[0] != nu) fail(SP_EINVAL, "no shift separates lambda_nu and lambda_nu+1 at working precision");
}

// alpha >= ||A - mu I||_2 from brackets of the extreme eigenvalues, l0 from
// the largest d on a geometric then linear grid with count(mu-d) == count(mu)
// == count(mu+d) (no eigenvalue within distance d of mu).
void qdwh_start(sp_ctx* ctx, int64_t n, int b, const double* ab_dev, int64_t ldab, double mu, double* alpha,
                double* l0) {
  double glo, ghi;
  gershgorin(ctx, n, b, ab_dev, ldab, &glo, &ghi);
  const double pad = 1e-12 * std::max({1.0, std::fabs(glo), std::fabs(ghi)});
  glo -= pad;
  ghi += pad;
  std::vector<double> x, y;
  bracket(ctx, n, b, ab_dev, ldab, {1, n}, glo, ghi, 2e-3, x, y);
  const double lam_min_lo = x[0], lam_max_hi = y[1];
  const double a = std::max(mu - lam_min_lo, lam_max_hi - mu) * (1.0 + 1e-10);
  // distance to the spectrum
  std::vector<double> pts;
  std::vector<double> ds;
  pts.push_back(mu);
  for (int k = 0; k <= 60; ++k) {
    const double d = a * std::ldexp(1.0, -k);
    ds.push_back(d);
    pts.push_back(mu - d);
    pts.push_back(mu + d);
  }
  std::vector<int64_t> c = counts_at(ctx, n, b, ab_dev, ldab, pts);
  const int64_t nu = c[0];
  double dgood = 0.0;
  for (size_t k = 0; k < ds.size(); ++k) {
    if (c[1 + 2 * k] == nu && c[2 + 2 * k] == nu) {
      dgood = ds[k];
      break;
    }
  }
  if (dgood == 0.0) fail(SP_EINVAL, "mu is (numerically) an eigenvalue: no gap found");
  // refine between dgood and 2 dgood
  pts.clear();
  std::vector<double> lin;
  for (int p = 1; p <= 127; ++p) {
    const double d = dgood * (1.0 + p / 128.0);
    lin.push_back(d);
    pts.push_back(mu - d);
    pts.push_back(mu + d);
  }
  c = counts_at(ctx, n, b, ab_dev, ldab, pts);
  for (size_t p = 0; p < lin.size(); ++p) {
    if (c[2 * p] == nu && c[2 * p + 1] == nu) dgood = lin[p];
    else break;
  }
  *alpha = a;
  *l0 = std::min(dgood / a, 1.0);
}

void configure_param_kernels() { configure_dynamic_smem(reinterpret_cast<const void*>(k_inertia_warp)); }

}  // namespace sp
