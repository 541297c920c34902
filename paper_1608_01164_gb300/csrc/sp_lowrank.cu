// sp_lowrank.cu -- batched recompression of low-rank blocks.
//
// Every formatted HODLR operation (Table "complexity_HODLR": addition,
// multiplication, Cholesky, triangular solve) produces off-diagonal blocks as
// sums  sum_s U_s (scale_s V_s)^T  of low-rank terms.  The paper recompresses
// every such sum after each operation, dropping singular values below a fixed
// absolute threshold epsilon (Sec. 3.1.1; Sec. 5).  Here, per block:
//   1. gather the stacked factors  W_U = [U_1 .. U_S]  (m x R) and
//      W_V = [s_1 V_1 .. s_S V_S]  (q x R);
//   2. Householder QR of W_U and W_V; tall factors use a binary TSQR tree of
//      512-row chunks (tunable; every chunk and merge is one CTA), so a block of 50 000
//      rows spreads over many SMs.  A merge stacks its children's R factors
//      compactly: its row count and the children's row offsets follow from the
//      actual width R on the device, so no stage works on padding;
//   3. core  M = R_U R_V^T  (r_U x r_V, r = min(rows, R));
//   4. truncated SVD of M in one CTA (k_core_svd): column-pivoted QR stopped at
//      the truncation level, QR of the transposed trapezoid, one-sided Jacobi
//      on the kept triangle (pairs on lane groups);
//   5. keep the k singular values > tol, U = Q_U [U~_k S_k; 0],
//      V = Q_V [V~_k; 0] by applying the Householder reflectors back down the
//      tree.
// The segments' widths are ranks produced by earlier launches; one read-back
// per call (the only host synchronisation) sizes every buffer, chunk and slot
// by the actual width R; the kernels read the same widths on the device.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>

#include "sp_internal.h"

namespace sp {
namespace {


__device__ __forceinline__ int dwidth(int w, const int* p) {
  if (!p) return w;
  int v = *p;
  v = v < 0 ? 0 : v;
  return v < w ? v : w;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------- gather -------
struct GatherBlock {
  int m, q;
  int seg0, nseg;
  double* WU;  // m x Rmax (ld m)
  double* WV;  // q x Rmax (ld q)
  int Rmax;
  int* R;      // out: stacked width
  int* ru;     // out: min(m, R)
  int* rv;     // out: min(q, R)
};

// grid: (row chunks, segment slot, block).  Column offsets of a segment are the
// sum of the actual widths of the segments before it.
__global__ void k_gather(const GatherBlock* __restrict__ blocks, const Seg* __restrict__ segs, int maxseg) {
  const GatherBlock b = blocks[blockIdx.z];
  const int s = blockIdx.y;
  if (s >= b.nseg) return;
  int off = 0;
  for (int t = 0; t < s; ++t) off += dwidth(segs[b.seg0 + t].w, segs[b.seg0 + t].pw);
  const Seg g = segs[b.seg0 + s];
  const int w = dwidth(g.w, g.pw);
  if (blockIdx.x == 0 && s == 0 && threadIdx.x == 0) {
    int tot = 0;
    for (int t = 0; t < b.nseg; ++t) tot += dwidth(segs[b.seg0 + t].w, segs[b.seg0 + t].pw);
    *b.R = tot;
    *b.ru = min(b.m, tot);
    *b.rv = min(b.q, tot);
  }
  const int rows = max(b.m, b.q);
  const int r0 = blockIdx.x * 256;
  if (r0 >= rows) return;
  for (int e = threadIdx.x; e < 256 * w; e += blockDim.x) {
    const int i = r0 + (e & 255), c = e >> 8;
    if (i < b.m) b.WU[i + (int64_t)(off + c) * b.m] = g.U[i + (int64_t)c * g.ldu];
    if (i < b.q) b.WV[i + (int64_t)(off + c) * b.q] = g.scale * g.V[i + (int64_t)c * g.ldv];
  }
}

// Reads the device-resident widths the segments point at (one thread each).
__global__ void k_read_widths(const int* const* __restrict__ p, int cnt, int* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) out[i] = *p[i];
}

// ---------------------------------------------------------- Householder QR --
// Row counts of TSQR nodes.  A chunk has a static row count; a merge node
// stacks the R factors of its children, min(rows_t, R) rows each, so its row
// count (and every child's row offset in it) depends on the actual width R.
struct RowRule {
  int rows;         // chunk: its rows; merge: static capacity (R = Rmax)
  int nkid;         // 0: chunk; > 0: merge of nkid children
  int kid_rows[2];  // children's static row counts (merge)
  int npre;         // earlier siblings in the parent (0 or 1)
  int pre_rows;     // static row count of the earlier sibling
};

__device__ __forceinline__ int rule_rows(const RowRule& q, int R) {
  if (q.nkid == 0) return q.rows;
  int s = 0;
  for (int t = 0; t < q.nkid; ++t) s += min(q.kid_rows[t], R);
  return s;
}

__device__ __forceinline__ int rule_offset(const RowRule& q, int R) { return q.npre ? min(q.pre_rows, R) : 0; }

// In-place QR of the rows x R matrix J (R = *pR <= Rmax).  Householder vectors
// are stored below the diagonal with v_0 = 1 implicit, tau[j] their scalars.
// The upper-trapezoidal factor (nref x R, nref = min(rows, R), zeros below the
// diagonal) is written at row offset rule_offset of dst (ld_dst).
struct QrJob {
  double* J;
  int64_t ldj;
  RowRule rr;
  const int* pR;
  int Rmax;
  double* tau;
  double* dst;
  int64_t ld_dst;
};

__global__ void __launch_bounds__(256) k_qr(const QrJob* __restrict__ jobs, double* fc) {
  const QrJob jb = jobs[blockIdx.x];
  const int R = dwidth(jb.Rmax, jb.pR);
  const int rows = rule_rows(jb.rr, R);
  double* J = jb.J;
  const int64_t ld = jb.ldj;
  const int nref = min(rows, R);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __shared__ double red[32];
  __shared__ double s_tau;
  __shared__ double s_v0;
  for (int j = 0; j < nref; ++j) {
    // sigma = ||J(j+1:rows, j)||^2
    double part = 0.0;
    for (int i = j + 1 + threadIdx.x; i < rows; i += blockDim.x) {
      const double x = J[i + (int64_t)j * ld];
      part += x * x;
    }
    part = warp_sum(part);
    if (lane == 0) red[warp] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sigma = 0.0;
      for (int w = 0; w < nw; ++w) sigma += red[w];
      const double x0 = J[j + (int64_t)j * ld];
      if (sigma == 0.0) {
        s_tau = 0.0;
        s_v0 = 1.0;
      } else {
        const double mu = sqrt(x0 * x0 + sigma);
        const double v0 = (x0 <= 0.0) ? x0 - mu : -sigma / (x0 + mu);
        s_tau = 2.0 * v0 * v0 / (sigma + v0 * v0);
        s_v0 = 1.0 / v0;  // the reciprocal, taken once
        J[j + (int64_t)j * ld] = mu;
      }
      jb.tau[j] = s_tau;
    }
    __syncthreads();
    const double tau = s_tau;
    if (tau != 0.0) {
      const double inv = s_v0;
      for (int i = j + 1 + threadIdx.x; i < rows; i += blockDim.x) J[i + (int64_t)j * ld] *= inv;
      __syncthreads();
      for (int c = j + 1 + warp; c < R; c += nw) {
        double d = 0.0;
        for (int i = j + 1 + lane; i < rows; i += 32) d += J[i + (int64_t)j * ld] * J[i + (int64_t)c * ld];
        // read the pivot entry before the warp reduction (which synchronises
        // the warp), so no lane can read it after lane 0 has updated it
        const double jc = J[j + (int64_t)c * ld];
        d = warp_sum(d) + jc;
        const double f = tau * d;
        if (lane == 0) J[j + (int64_t)c * ld] = jc - f;
        for (int i = j + 1 + lane; i < rows; i += 32) J[i + (int64_t)c * ld] -= f * J[i + (int64_t)j * ld];
      }
    }
    __syncthreads();
  }
  if (fc && threadIdx.x == 0) {
    // per reflector j: norm (2 flops/row) + dot and axpy on R-j-1 columns (4 flops/row each)
    double f = 0.0;
    for (int j = 0; j < nref; ++j) f += (double)(rows - j) * (2.0 + 4.0 * (R - j - 1));
    atomicAdd(fc, f);
  }
  // the R factor: nref x R upper trapezoid at its row offset in dst
  double* dst = jb.dst + rule_offset(jb.rr, R);
  for (int64_t e = threadIdx.x; e < (int64_t)nref * R; e += blockDim.x) {
    const int i = (int)(e % nref), c = (int)(e / nref);
    dst[i + (int64_t)c * jb.ld_dst] = (i <= c) ? J[i + (int64_t)c * ld] : 0.0;
  }
}

// out = Q [S; 0] where Q = H_0 H_1 ... H_{r-1} are the reflectors of a QrJob
// (r = min(rows, R)); S: nref x k, read at row offset rule_offset(srule) of S
// (the node's slot in its parent's output).  A chunk (final output) writes
// rows x cap with columns >= k zero; a merge node writes only rows x k.
struct ApplyJob {
  const double* J;
  int64_t ldj;
  RowRule rr;
  RowRule srule;
  const int* pR;
  int Rmax;
  const double* tau;
  const double* S;
  int64_t lds;
  double* out;
  int64_t ldo;
  const int* pk;
  int cap;
};

__global__ void __launch_bounds__(256) k_apply_q(const ApplyJob* __restrict__ jobs, double* fc) {
  const ApplyJob jb = jobs[blockIdx.x];
  const int R = dwidth(jb.Rmax, jb.pR);
  const int rows = rule_rows(jb.rr, R);
  const int nref = min(rows, R);
  const int k = dwidth(jb.cap, jb.pk);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double* O = jb.out;
  const int64_t ldo = jb.ldo;
  const double* S = jb.S + rule_offset(jb.srule, R);
  const int wcols = jb.rr.nkid == 0 ? jb.cap : k;
  for (int64_t e = threadIdx.x; e < (int64_t)rows * wcols; e += blockDim.x) {
    const int i = (int)(e % rows), c = (int)(e / rows);
    double v = 0.0;
    if (c < k && i < nref) v = S[i + (int64_t)c * jb.lds];
    O[i + (int64_t)c * ldo] = v;
  }
  __syncthreads();
  const double* J = jb.J;
  const int64_t ld = jb.ldj;
  if (fc && threadIdx.x == 0) {
    double f = 0.0;
    for (int j = 0; j < nref; ++j) f += 4.0 * (double)(rows - j) * k;
    atomicAdd(fc, f);
  }
  for (int j = nref - 1; j >= 0; --j) {
    const double tau = jb.tau[j];
    if (tau != 0.0) {
      for (int c = warp; c < k; c += nw) {
        double d = 0.0;
        for (int i = j + 1 + lane; i < rows; i += 32) d += J[i + (int64_t)j * ld] * O[i + (int64_t)c * ldo];
        const double oj = O[j + (int64_t)c * ldo];  // read before the synchronising reduction
        d = warp_sum(d) + oj;
        const double f = tau * d;
        if (lane == 0) O[j + (int64_t)c * ldo] = oj - f;
        for (int i = j + 1 + lane; i < rows; i += 32) O[i + (int64_t)c * ldo] -= f * J[i + (int64_t)j * ld];
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ Jacobi SVD ----
struct SvdJob {
  const double* M;  // ru x rv core (ld Rmax)
  const int* pru;
  const int* prv;
  int Rmax;
  double* G;        // work (Rmax x Rmax)
  double* Vacc;     // work (Rmax x Rmax)
  double* W3;       // work (Rmax x Rmax)
  double* SU;       // Rmax x cap: U~ Sigma (ru rows)
  double* SV;       // Rmax x cap: V~ (rv rows)
  int* pk;          // out: kept rank
  int cap;
};

__device__ __forceinline__ void rr_pair(int round, int p, int P, int& i, int& j) {
  // round-robin tournament: player P-1 fixed, the others rotate
  if (p == 0) {
    i = P - 1;
    j = round;
  } else {
    i = (round + p) % (P - 1);
    j = (round - p + P - 1) % (P - 1);
  }
}

// Block-wide argmax of v[c], c in [c0, c1) (v in shared memory); returns the
// index (ties -> smallest) in *out_idx and the value in *out_val.
__device__ void block_argmax(const double* v, int c0, int c1, double* red_v, int* red_i, int* out_idx,
                             double* out_val) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double best = -1.0;
  int bi = c1;
  for (int c = c0 + threadIdx.x; c < c1; c += blockDim.x)
    if (v[c] > best) {
      best = v[c];
      bi = c;
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) {
      best = ov;
      bi = oi;
    }
  }
  if (lane == 0) {
    red_v[warp] = best;
    red_i[warp] = bi;
  }
  __syncthreads();
  if (warp == 0) {  // the per-warp candidates, reduced by one warp
    double b = lane < nw ? red_v[lane] : -1.0;
    int ib = lane < nw ? red_i[lane] : c1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, b, o);
      const int oi = __shfl_xor_sync(0xffffffffu, ib, o);
      if (ov > b || (ov == b && oi < ib)) {
        b = ov;
        ib = oi;
      }
    }
    if (lane == 0) {
      *out_idx = ib;
      *out_val = b;
    }
  }
  __syncthreads();
}

// Householder reflector for column j of X (rows j..rows-1), stored in place
// below the diagonal (v_0 = 1 implicit); returns tau (0: identity).  All
// threads call it; the caller synchronises before using the column.
__device__ double make_reflector(double* X, int64_t ld, int j, int rows, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __shared__ double s_tau;
  __shared__ double s_v0;
  double part = 0.0;
  for (int i = j + 1 + threadIdx.x; i < rows; i += blockDim.x) {
    const double x = X[i + (int64_t)j * ld];
    part = fma(x, x, part);
  }
  part = warp_sum(part);
  if (lane == 0) red[warp] = part;
  __syncthreads();
  if (warp == 0) {
    // the per-warp partials summed by one warp (a fixed order) instead of
    // one thread's serial sum, then the reflector's scalars (R's diagonal
    // mu >= 0, as in k_qr)
    const double sigma = warp_sum(lane < nw ? red[lane] : 0.0);
    const double x0 = X[j + (int64_t)j * ld];
    if (lane == 0) {
      if (sigma == 0.0) {
        s_tau = 0.0;
        s_v0 = 1.0;
      } else {
        const double mu = sqrt(x0 * x0 + sigma);
        const double v0 = (x0 <= 0.0) ? x0 - mu : -sigma / (x0 + mu);
        s_tau = 2.0 * v0 * v0 / (sigma + v0 * v0);
        s_v0 = 1.0 / v0;  // the reciprocal, taken once
        X[j + (int64_t)j * ld] = mu;
      }
    }
  }
  __syncthreads();
  const double tau = s_tau;
  if (tau != 0.0) {
    const double inv = s_v0;
    for (int i = j + 1 + threadIdx.x; i < rows; i += blockDim.x) X[i + (int64_t)j * ld] *= inv;
  }
  __syncthreads();
  return tau;
}

// Y(j:rows, c) -= tau v (v^T Y(j:rows, c)) for columns c in [c0, c1) of Y, v =
// reflector j stored in V (column j, v_0 = 1); one warp per column.  With
// nrm != null also stores ||Y(j+1:rows, c)||^2 in nrm[c] (pivoting norms).
__device__ void apply_reflector(const double* V, int64_t ldv, int j, int rows, double tau, double* Y, int64_t ldy,
                                int c0, int c1, double* nrm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = c0 + warp; c < c1; c += nw) {
    double* y = Y + (int64_t)c * ldy;
    const double* v = V + (int64_t)j * ldv;
    if (tau != 0.0) {
      double d = 0.0;
      for (int i = j + 1 + lane; i < rows; i += 32) d = fma(v[i], y[i], d);
      const double yj = y[j];  // read before the synchronising reduction
      d = warp_sum(d) + yj;
      const double f = tau * d;
      if (lane == 0) y[j] = yj - f;
      for (int i = j + 1 + lane; i < rows; i += 32) y[i] -= f * v[i];
    }
    if (nrm) {
      double q = 0.0;
      for (int i = j + 1 + lane; i < rows; i += 32) q = fma(y[i], y[i], q);
      q = warp_sum(q);
      if (lane == 0) nrm[c] = q;
    }
  }
}

// One-sided (Hestenes) Jacobi sweeps on the rp columns of B (ld ldb),
// accumulating the rotations into J, round-robin pair order.  A pair is
// handled by a group of G lanes (G = 8, 16 or 32 by rp), so one warp works on
// 32/G pairs at once: for small cores the reductions and the rotation's
// parameters, not the dot products, are most of a pair's binary64 work.  A
// pair is rotated when g^2 > eps^2 a b; stops after a sweep without rotation
// or after max_sweeps.  All threads of the CTA call it.  Returns the flops of
// the tests and rotations counted by each group's first lane (0 elsewhere).
template <typename T>
__device__ double jacobi_sweeps(T* B, T* J, int ldb, int rp, T eps, int max_sweeps, int* s_rot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int G = rp <= 16 ? 8 : (rp <= 48 ? 16 : 32);
  const int ppw = 32 / G, grp = lane / G, gl = lane % G;
  const int P = rp + (rp & 1);
  const int npairs = P / 2;
  double fl = 0.0;
  for (int sweep = 0; sweep < max_sweeps && rp > 1; ++sweep) {
    if (threadIdx.x == 0) *s_rot = 0;
    __syncthreads();
    int rotated = 0;
    for (int round = 0; round < P - 1; ++round) {
      for (int base = warp * ppw; base < npairs; base += nw * ppw) {  // uniform within the warp
        const int pp = base + grp;
        int i = 0, jj = 0;
        bool valid = pp < npairs;
        if (valid) {
          rr_pair(round, pp, P, i, jj);
          valid = i < rp && jj < rp;
        }
        if (!valid) i = jj = 0;
        T* gi = B + (int64_t)i * ldb;
        T* gj = B + (int64_t)jj * ldb;
        T a = 0, b = 0, g = 0;
        if (valid)
          for (int r = gl; r < rp; r += G) {
            const T x = gi[r], y = gj[r];
            a = fma(x, x, a);
            b = fma(y, y, b);
            g = fma(x, y, g);
          }
        for (int o = G >> 1; o > 0; o >>= 1) {  // within the group
          a += __shfl_xor_sync(0xffffffffu, a, o);
          b += __shfl_xor_sync(0xffffffffu, b, o);
          g += __shfl_xor_sync(0xffffffffu, g, o);
        }
        if (valid && gl == 0) fl += 6.0 * rp;
        if (valid && g != (T)0 && g * g > eps * eps * a * b) {
          if (gl == 0) fl += 12.0 * rp;
          // tan(theta) = t = sign(d) e / (|d| + h), d = b - a, e = 2g,
          // h = sqrt(d^2 + e^2) (the smaller root of t^2 + 2 (d/e) t - 1);
          // by the half-angle formulas cos(theta) = (|d| + h) w and
          // sin(theta) = sign(d) e w with w = 1 / sqrt(2 h (|d| + h)): two
          // reciprocal square roots on the chain, no division
          const T d = b - a, e = (T)2 * g;
          const T hq = fma(d, d, e * e);
          T cs, sn;
          if (hq > (T)1e-280 && hq < (T)1e280) {
            const T h = hq * rsqrt(hq);
            const T y = fabs(d) + h;
            const T w = rsqrt((T)2 * h * y);
            cs = y * w;
            sn = (d >= (T)0 ? e : -e) * w;
          } else {  // extreme ranges: the quotient form
            const T zeta = d / e;
            const T t = (zeta >= (T)0 ? (T)1 : (T)-1) / (fabs(zeta) + sqrt((T)1 + zeta * zeta));
            cs = (T)1 / sqrt((T)1 + t * t);
            sn = cs * t;
          }
          T* ji = J + (int64_t)i * ldb;
          T* jj2 = J + (int64_t)jj * ldb;
          for (int r = gl; r < rp; r += G) {
            const T x = gi[r], y = gj[r];
            gi[r] = cs * x - sn * y;
            gj[r] = sn * x + cs * y;
            const T u = ji[r], v = jj2[r];
            ji[r] = cs * u - sn * v;
            jj2[r] = sn * u + cs * v;
          }
          rotated = 1;
        }
      }
      __syncthreads();
    }
    if (rotated) *s_rot = 1;
    __syncthreads();
    const int any = *s_rot;
    __syncthreads();
    if (!any) break;
  }
  return fl;
}


// Truncated SVD of the r_U x r_V core M = R_U R_V^T (one CTA per core):
//  1. column-pivoted Householder QR  M P = Q1 [R11 R12; 0 R22], stopped when
//     every remaining column norm is <= 1e-3 tol / sqrt(cols), so the dropped
//     ||R22||_F <= 1e-3 tol;  r' = rows kept;
//  2. Householder QR of the transpose of the r' x cols trapezoid T: T^T = Q2 R2;
//  3. one-sided Jacobi on B = R2^T (r' x r'):  B J = U~ Sigma;
//  4. M ~= (Q1 U~ Sigma)(P Q2 J)^T: keep sigma > tol, apply the reflectors.
// Cost O(r' r_U r_V) instead of O(r_U^3) for a core of numerical rank r'.
__global__ void __launch_bounds__(1024) k_core_svd(const SvdJob* __restrict__ jobs, double tol, int* flags,
                                                   double* fc) {
  const SvdJob jb = jobs[blockIdx.x];
  const int ru = *jb.pru, rv = *jb.prv;
  const int ld = jb.Rmax;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double* M = const_cast<double*>(jb.M);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* nrm = reinterpret_cast<double*>(smem_raw);  // Rmax
  double* tau1 = nrm + ld;                            // Rmax
  double* tau2 = tau1 + ld;                           // Rmax
  double* sig = tau2 + ld;                            // Rmax
  int* perm = reinterpret_cast<int*>(sig + ld);       // Rmax
  int* perm2 = perm + ld;                             // Rmax
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ int s_p;
  __shared__ double s_max;
  __shared__ int s_rot;
  __shared__ int s_k;
  double nflop = 0.0;   // block-level stages, counted by thread 0
  double nflopw = 0.0;  // Jacobi work, counted by the first lane of each pair group
  // ---- 1. column-pivoted QR of M
  for (int c = warp; c < rv; c += nw) {
    double q = 0.0;
    for (int i = lane; i < ru; i += 32) q = fma(M[i + (int64_t)c * ld], M[i + (int64_t)c * ld], q);
    q = warp_sum(q);
    if (lane == 0) {
      nrm[c] = q;
      perm[c] = c;
    }
  }
  __syncthreads();
  const double thr = 1e-3 * tol / sqrt((double)(rv > 0 ? rv : 1));
  const double thr2 = thr * thr;
  int rp = 0;
  const int rmin = ru < rv ? ru : rv;
  for (int j = 0; j < rmin; ++j) {
    // remaining norm of column c counts rows j..ru-1
    block_argmax(nrm, j, rv, red_v, red_i, &s_p, &s_max);
    if (s_max <= thr2) break;
    const int p = s_p;
    if (p != j) {
      for (int i = threadIdx.x; i < ru; i += blockDim.x) {
        const double t = M[i + (int64_t)j * ld];
        M[i + (int64_t)j * ld] = M[i + (int64_t)p * ld];
        M[i + (int64_t)p * ld] = t;
      }
      if (threadIdx.x == 0) {
        const double t = nrm[j];
        nrm[j] = nrm[p];
        nrm[p] = t;
        const int q = perm[j];
        perm[j] = perm[p];
        perm[p] = q;
      }
    }
    __syncthreads();
    const double tau = make_reflector(M, ld, j, ru, red_v);
    if (threadIdx.x == 0) tau1[j] = tau;
    apply_reflector(M, ld, j, ru, tau, M, ld, j + 1, rv, nrm);
    nflop += 6.0 * (double)(ru - j) * (rv - j);
    __syncthreads();
    rp = j + 1;
  }
  // ---- 2. A2 = T^T (rv x rp), T = rows 0..rp-1 of the upper trapezoid
  double* A2 = jb.G;
  for (int64_t e = threadIdx.x; e < (int64_t)rv * rp; e += blockDim.x) {
    const int c = (int)(e % rv), i = (int)(e / rv);
    A2[c + (int64_t)i * ld] = (i <= c) ? M[i + (int64_t)c * ld] : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < rp; ++j) {
    const double tau = make_reflector(A2, ld, j, rv, red_v);
    if (threadIdx.x == 0) tau2[j] = tau;
    apply_reflector(A2, ld, j, rv, tau, A2, ld, j + 1, rp, nullptr);
    nflop += 4.0 * (double)(rv - j) * (rp - j);
    __syncthreads();
  }
  // ---- 3. Jacobi on B = R2^T (rp x rp), J accumulated
  double* B = jb.Vacc;
  double* J = jb.W3;
  for (int64_t e = threadIdx.x; e < (int64_t)rp * rp; e += blockDim.x) {
    const int i = (int)(e % rp), c = (int)(e / rp);
    B[i + (int64_t)c * ld] = (c <= i) ? A2[c + (int64_t)i * ld] : 0.0;
    J[i + (int64_t)c * ld] = (i == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  nflopw += jacobi_sweeps<double>(B, J, ld, rp, 1e-15, 60, &s_rot);
  // ---- 4. singular values, order, truncation
  for (int c = warp; c < rp; c += nw) {
    double a = 0.0;
    for (int r = lane; r < rp; r += 32) a = fma(B[r + (int64_t)c * ld], B[r + (int64_t)c * ld], a);
    a = warp_sum(a);
    if (lane == 0) sig[c] = sqrt(a);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < rp; c += blockDim.x) {
    int pos = 0;
    const double sc = sig[c];
    for (int d = 0; d < rp; ++d) pos += (sig[d] > sc) || (sig[d] == sc && d < c);
    perm2[pos] = c;
  }
  if (threadIdx.x == 0) {
    int k = 0;
    for (int c = 0; c < rp; ++c) k += sig[c] > tol;
    if (k > jb.cap) {
      atomicOr(&flags[FLAG_RANK], 1);
      k = jb.cap;
    }
    s_k = k;
    *jb.pk = k;
  }
  __syncthreads();
  const int k = s_k;
  // S_U = Q1 [B(:, perm2) ; 0]  (ru rows, k columns; the applies read no more)
  for (int64_t e = threadIdx.x; e < (int64_t)ru * k; e += blockDim.x) {
    const int r = (int)(e % ru), p = (int)(e / ru);
    jb.SU[r + (int64_t)p * ld] = (r < rp) ? B[r + (int64_t)perm2[p] * ld] : 0.0;
  }
  __syncthreads();
  for (int j = rp - 1; j >= 0; --j) {
    apply_reflector(M, ld, j, ru, tau1[j], jb.SU, ld, 0, k, nullptr);
    __syncthreads();
  }
  // W = Q2 [J(:, perm2); 0] (rv rows) in B's buffer, then S_V = P W
  double* W = B;
  for (int64_t e = threadIdx.x; e < (int64_t)ld * k; e += blockDim.x) {
    const int r = (int)(e % ld), p = (int)(e / ld);
    W[r + (int64_t)p * ld] = (r < rp) ? J[r + (int64_t)perm2[p] * ld] : 0.0;
  }
  __syncthreads();
  for (int j = rp - 1; j >= 0; --j) {
    apply_reflector(A2, ld, j, rv, tau2[j], W, ld, 0, k, nullptr);
    __syncthreads();
  }
  for (int64_t e = threadIdx.x; e < (int64_t)rv * k; e += blockDim.x) {
    const int r = (int)(e % rv), p = (int)(e / rv);
    jb.SV[perm[r] + (int64_t)p * ld] = W[r + (int64_t)p * ld];
  }
  if (fc) {
    if (threadIdx.x == 0) nflop += 4.0 * rp * ((double)ru + rv) * k;  // the two reflector applications
    const double f = (threadIdx.x == 0 ? nflop : 0.0) + nflopw;
    if (f > 0.0) atomicAdd(fc, f);
  }
}

// -------------------------------------------------------------- planning ----
struct TreePlan {
  // QR jobs by level (level 0 = chunks); apply jobs in reverse order
  std::vector<std::vector<QrJob>> qr;
  std::vector<std::vector<ApplyJob>> app;
};

}  // namespace

// Builds the TSQR tree of one side (rows x Rmax matrix W, device width pR),
// leaving the final R factor in `rdst` (ld ldr) and arranging for Q [S; 0]
// (S with ld ldr) to be written into `out` (rows x cap, ld ldo).  Each merge
// stacks two children's R factors (at most min(rows_t, Rmax) rows each).
static void plan_side(double* W, int64_t ldw, int rows, const int* pR, int Rmax, double* rdst, int64_t ldr,
                      const double* S, const int* pk, int cap, double* out, int64_t ldo,
                      std::vector<std::vector<QrJob>>& qrl, std::vector<std::vector<ApplyJob>>& apl,
                      std::vector<DBuf>& keep, cudaStream_t st, int chunk_rows) {
  // chunks of at least 2 Rmax rows, so that a merge (<= 2 Rmax rows) is never
  // taller than a chunk
  const int kChunk = std::max(chunk_rows, (2 * Rmax + 31) / 32 * 32);
  struct Node {
    double* J;
    int64_t ldj;
    RowRule rr;
    double* tau;
    int parent;       // index into the next level, -1 for the root
    int slot;         // 0 or 1 within the parent
    double* app_out;  // apply output (merge: own buffer, chunk: out + row)
    int64_t ldapp;
  };
  auto chunk_rule = [](int r) { return RowRule{r, 0, {0, 0}, 0, 0}; };
  std::vector<std::vector<Node>> lv;
  std::vector<Node> l0;
  const int nch = rows <= kChunk ? 1 : (rows + kChunk - 1) / kChunk;
  for (int c = 0; c < nch; ++c) {
    const int r0 = c * kChunk;
    const int rr = std::min(kChunk, rows - r0);
    l0.push_back(Node{W + r0, ldw, chunk_rule(rr), nullptr, -1, 0, out + r0, ldo});
  }
  lv.push_back(l0);
  while (lv.back().size() > 1) {
    std::vector<Node>& cur = lv.back();
    std::vector<Node> nxt;
    for (size_t i = 0; i < cur.size(); i += 2) {
      const int nchild = (i + 1 < cur.size()) ? 2 : 1;
      RowRule m{0, nchild, {0, 0}, 0, 0};
      for (int t = 0; t < nchild; ++t) {
        m.kid_rows[t] = cur[i + t].rr.rows;
        m.rows += std::min(cur[i + t].rr.rows, Rmax);
      }
      keep.emplace_back((size_t)m.rows * Rmax * sizeof(double) + 16, st);
      double* Mb = keep.back().as<double>();
      nxt.push_back(Node{Mb, m.rows, m, nullptr, -1, 0, nullptr, 0});
      for (int t = 0; t < nchild; ++t) {
        cur[i + t].parent = (int)nxt.size() - 1;
        cur[i + t].slot = t;
        if (t == 1) {
          cur[i + t].rr.npre = 1;
          cur[i + t].rr.pre_rows = cur[i].rr.rows;
        }
      }
    }
    lv.push_back(nxt);
  }
  // taus, QR jobs, apply buffers
  qrl.resize(std::max(qrl.size(), lv.size()));
  apl.resize(std::max(apl.size(), lv.size()));
  for (size_t l = 0; l < lv.size(); ++l) {
    for (auto& nd : lv[l]) {
      keep.emplace_back((size_t)Rmax * sizeof(double) + 16, st);
      nd.tau = keep.back().as<double>();
      if (l > 0) {
        keep.emplace_back((size_t)nd.rr.rows * cap * sizeof(double) + 16, st);
        nd.app_out = keep.back().as<double>();
        nd.ldapp = nd.rr.rows;
      }
    }
  }
  const size_t depth = lv.size();
  for (size_t l = 0; l < depth; ++l) {
    for (auto& nd : lv[l]) {
      const bool root = (l + 1 == depth);
      double* dst = root ? rdst : lv[l + 1][nd.parent].J;
      const int64_t ldd = root ? ldr : lv[l + 1][nd.parent].ldj;
      // the node's own row rule carries its offset in the parent (npre/pre_rows)
      qrl[l].push_back(QrJob{nd.J, nd.ldj, nd.rr, pR, Rmax, nd.tau, dst, ldd});
      const double* Sin = root ? S : lv[l + 1][nd.parent].app_out;
      const int64_t lds = root ? ldr : lv[l + 1][nd.parent].ldapp;
      // apply levels run from the top: store at index (depth-1-l)
      apl[depth - 1 - l].push_back(ApplyJob{nd.J, nd.ldj, nd.rr, nd.rr, pR, Rmax, nd.tau, Sin, lds, nd.app_out,
                                            nd.ldapp, pk, cap});
    }
  }
}

void recompress(sp_ctx* ctx, const std::vector<LrBlock>& blocks, double tol) {
  if (blocks.empty()) return;
  cudaStream_t st = ctx->stream;
  const int nb = (int)blocks.size();
  std::vector<Seg> segs;
  std::vector<GatherBlock> gb(nb);
  std::vector<int> Rmax(nb), Rs(nb);
  // Exact stacked widths: the segments' widths live on the device (ranks
  // produced by earlier launches); read them once so that every buffer, chunk
  // and slot below is sized by the actual width instead of the capacities.
  std::vector<const int*> wptr;
  for (const LrBlock& b : blocks)
    for (const Seg& sg : b.segs)
      if (sg.pw) wptr.push_back(sg.pw);
  std::vector<int> wval(wptr.size());
  if (!wptr.empty()) {
    DBuf dp = upload(wptr, st);
    DBuf dv(wptr.size() * sizeof(int) + 16, st);
    k_read_widths<<<(unsigned)((wptr.size() + 255) / 256), 256, 0, st>>>(dp.as<const int*>(), (int)wptr.size(),
                                                                           dv.as<int>());
    check_launch("k_read_widths");
    check_cuda(cudaMemcpyAsync(wval.data(), dv.p, wval.size() * sizeof(int), cudaMemcpyDeviceToHost, st), "widths");
    const auto t0 = std::chrono::steady_clock::now();
    check_cuda(cudaStreamSynchronize(st), "sync");
    if (ctx->profiling) {
      ctx->ms[KID_HOST_WAIT] += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      ctx->launches[KID_HOST_WAIT] += 1;
    }
  }
  size_t wsz = 0, csz = 0;
  int maxseg = 1, maxrows = 1, maxR = 1;
  size_t wi = 0;
  for (int t = 0; t < nb; ++t) {
    const LrBlock& b = blocks[t];
    int R = 0;
    for (const Seg& sg : b.segs) {
      int w = sg.w;
      if (sg.pw) w = std::min(sg.w, std::max(wval[wi++], 0));
      R += w;
    }
    Rmax[t] = std::max(R, 1);
    // R factors, core and SVD work have at most min(max(m, q), R) rows
    Rs[t] = std::max(1, std::min(std::max(b.m, b.q), Rmax[t]));
    wsz += (size_t)(b.m + b.q) * Rmax[t];
    csz += 2 * (size_t)Rs[t] * Rmax[t] + (size_t)Rs[t] * Rs[t] + 2 * (size_t)Rs[t] * b.cap;
    maxseg = std::max(maxseg, (int)b.segs.size());
    maxrows = std::max(maxrows, std::max(b.m, b.q));
    maxR = std::max(maxR, Rs[t]);
    ctx->flops += 4.0 * (double)(b.m + b.q) * Rmax[t] * Rmax[t];
  }
  std::vector<DBuf> keep;
  DBuf wbuf(wsz * sizeof(double) + 64, st);
  check_cuda(cudaMemsetAsync(wbuf.p, 0, wsz * sizeof(double) + 64, st), "memset workspace");
  DBuf cbuf(csz * sizeof(double) + 64, st);
  DBuf ibuf((size_t)nb * 4 * sizeof(int) + 64, st);
  double* wp = wbuf.as<double>();
  double* cp = cbuf.as<double>();
  int* ip = ibuf.as<int>();
  struct Side {
    double* W;
    int rows;
    double* Rdst;
  };
  std::vector<SvdJob> svd(nb);
  std::vector<std::vector<QrJob>> qrl;
  std::vector<std::vector<ApplyJob>> apl;
  std::vector<GemmTask> core;
  for (int t = 0; t < nb; ++t) {
    const LrBlock& b = blocks[t];
    const int Rm = Rmax[t];
    GatherBlock& g = gb[t];
    g.m = b.m;
    g.q = b.q;
    g.seg0 = (int)segs.size();
    g.nseg = (int)b.segs.size();
    for (const Seg& s : b.segs) segs.push_back(s);
    g.WU = wp;
    wp += (size_t)b.m * Rm;
    g.WV = wp;
    wp += (size_t)b.q * Rm;
    g.Rmax = Rm;
    g.R = ip + 4 * t;
    g.ru = ip + 4 * t + 1;
    g.rv = ip + 4 * t + 2;
    const int Rr = Rs[t];
    double* RU = cp;  // Rr x Rm, ld Rr
    cp += (size_t)Rr * Rm;
    double* RV = cp;
    cp += (size_t)Rr * Rm;
    double* M = cp;  // Rr x Rr
    cp += (size_t)Rr * Rr;
    double* SU = cp;  // Rr x cap
    cp += (size_t)Rr * b.cap;
    double* SV = cp;
    cp += (size_t)Rr * b.cap;
    plan_side(g.WU, b.m, b.m, g.R, Rm, RU, Rr, SU, b.rank_out, b.cap, b.Uout, b.ldu_out, qrl, apl, keep, st, ctx->tsqr_chunk);
    plan_side(g.WV, b.q, b.q, g.R, Rm, RV, Rr, SV, b.rank_out, b.cap, b.Vout, b.ldv_out, qrl, apl, keep, st, ctx->tsqr_chunk);
    // M = R_U R_V^T (ru x rv, inner dimension R)
    core.push_back(gt(RU, Rr, RV, Rr, M, Rr, Rr, Rr, Rm, 1.0, 0.0, g.ru, g.rv, g.R));
    keep.emplace_back((size_t)Rr * Rr * 3 * sizeof(double) + 16, st);
    double* Gw = keep.back().as<double>();
    svd[t] = SvdJob{M, g.ru, g.rv, Rr, Gw, Gw + (size_t)Rr * Rr, Gw + 2 * (size_t)Rr * Rr, SU, SV, b.rank_out, b.cap};
  }
  // 1. gather
  {
    DBuf dseg = upload(segs, st);
    DBuf dgb = upload(gb, st);
    for (int off = 0; off < nb; off += 65535) {
      const int cnt = std::min(65535, nb - off);
      dim3 grid((maxrows + 255) / 256, maxseg, cnt);
      ProfScope ps(ctx, KID_GATHER);
      k_gather<<<grid, 256, 0, st>>>(dgb.as<GatherBlock>() + off, dseg.as<Seg>(), maxseg);
      check_launch("k_gather");
    }
  }
  // 2. QR levels bottom-up
  for (auto& lvl : qrl) {
    if (lvl.empty()) continue;
    DBuf d = upload(lvl, st);
    ProfScope ps(ctx, KID_QR);
    k_qr<<<(unsigned)lvl.size(), 256, 0, st>>>(d.as<QrJob>(), fc_ptr(ctx, KID_QR));
    check_launch("k_qr");
  }
  // 3. cores
  gemm_batched(ctx, false, true, core);
  // 4. truncated SVD of every core (rank-revealing QR, then Jacobi on the
  // kept triangle)
  {
    DBuf d = upload(svd, st);
    const size_t sm = (size_t)maxR * (4 * sizeof(double) + 2 * sizeof(int)) + 64;
    ensure_dynamic_smem(reinterpret_cast<const void*>(k_core_svd), sm);
    ProfScope ps(ctx, KID_CORE_SVD);
    // small cores: fewer warps make the ~rp barrier-separated stages cheaper
    const int threads = maxR <= 64 ? 256 : (maxR <= 160 ? 512 : 1024);
    k_core_svd<<<(unsigned)nb, threads, sm, st>>>(d.as<SvdJob>(), tol, ctx->d_flags, fc_ptr(ctx, KID_CORE_SVD));
    check_launch("k_core_svd");
  }
  // 5. apply reflectors top-down
  for (auto& lvl : apl) {
    if (lvl.empty()) continue;
    DBuf d = upload(lvl, st);
    ProfScope ps(ctx, KID_APPLYQ);
    k_apply_q<<<(unsigned)lvl.size(), 256, 0, st>>>(d.as<ApplyJob>(), fc_ptr(ctx, KID_APPLYQ));
    check_launch("k_apply_q");
  }
}

void configure_lowrank_kernels() { configure_dynamic_smem(reinterpret_cast<const void*>(k_core_svd)); }

}  // namespace sp
