// sp_lowrank.cu -- batched recompression of low-rank blocks.
//
// Every formatted HODLR operation (Table "complexity_HODLR": addition,
// multiplication, Cholesky, triangular solve) produces off-diagonal blocks as
// sums  sum_s U_s (scale_s V_s)^T  of low-rank terms.  The paper truncates them
// with an absolute tolerance epsilon ("repeated recompression with the absolute
// truncation tolerance", Sec. 5; Sec. 3.1.1).  Here, per block:
//   1. gather the stacked factors  W_U = [U_1 .. U_S]  (m x R) and
//      W_V = [s_1 V_1 .. s_S V_S]  (q x R);
//   2. Householder QR of W_U and W_V; tall factors use a binary TSQR tree of
//      row chunks (every chunk and merge is one CTA), so a block of 50 000 rows
//      spreads over many SMs;
//   3. core  M = R_U R_V^T  (r_U x r_V, r = min(rows, R));
//   4. one-sided (Hestenes) Jacobi SVD of M in one CTA, round-robin pair order;
//   5. keep the k singular values > tol, U = Q_U [U~_k S_k; 0],
//      V = Q_V [V~_k; 0] by applying the Householder reflectors back down the
//      tree.
// All sizes except the static upper bounds are device-resident (ranks produced
// by earlier launches), so the whole pipeline is enqueued without a host sync.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "sp_internal.h"

namespace sp {
namespace {

// shared memory available to the SVD kernel's working set (bytes)
constexpr size_t kSvdSmemMax = 200 * 1024;

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

// ---------------------------------------------------------- Householder QR --
// In-place QR of the rows x R matrix J (R = *pR <= Rmax).  Householder vectors
// are stored below the diagonal with v_0 = 1 implicit, tau[j] their scalars.
// The upper-trapezoidal factor is copied to dst (Rmax x Rmax slot, ld_dst),
// zero elsewhere in the slot.
struct QrJob {
  double* J;
  int64_t ldj;
  int rows;
  const int* pR;
  int Rmax;
  double* tau;
  double* dst;
  int64_t ld_dst;
};

__global__ void __launch_bounds__(256) k_qr(const QrJob* __restrict__ jobs, double* fc) {
  const QrJob jb = jobs[blockIdx.x];
  const int R = dwidth(jb.Rmax, jb.pR);
  const int rows = jb.rows;
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
        s_v0 = v0;
        J[j + (int64_t)j * ld] = mu;
      }
      jb.tau[j] = s_tau;
    }
    __syncthreads();
    const double tau = s_tau;
    if (tau != 0.0) {
      const double inv = 1.0 / s_v0;
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
  // copy R (nref x R upper trapezoid) into the Rmax x Rmax slot
  for (int64_t e = threadIdx.x; e < (int64_t)jb.Rmax * jb.Rmax; e += blockDim.x) {
    const int i = (int)(e % jb.Rmax), c = (int)(e / jb.Rmax);
    double v = 0.0;
    if (i < nref && c < R && i <= c) v = J[i + (int64_t)c * ld];
    jb.dst[i + (int64_t)c * jb.ld_dst] = v;
  }
}

// out = Q [S; 0] where Q = H_0 H_1 ... H_{r-1} are the reflectors of a QrJob
// (r = min(rows, R)); S: Rmax x k slot (rows beyond min(rows,R) ignored);
// out: rows x cap, columns >= k set to zero.
struct ApplyJob {
  const double* J;
  int64_t ldj;
  int rows;
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
  const int rows = jb.rows;
  const int nref = min(rows, R);
  const int k = dwidth(jb.cap, jb.pk);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double* O = jb.out;
  const int64_t ldo = jb.ldo;
  for (int64_t e = threadIdx.x; e < (int64_t)rows * jb.cap; e += blockDim.x) {
    const int i = (int)(e % rows), c = (int)(e / rows);
    double v = 0.0;
    if (c < k && i < nref) v = jb.S[i + (int64_t)c * jb.lds];
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

// One CTA (32 warps) per core.  When rows*cols + cols*cols doubles fit in
// shared memory (SMEM = true) the working matrix G and the accumulated right
// rotations V live there; otherwise in the global work buffers.  Each round of
// the round-robin ordering has P/2 disjoint column pairs, processed by the
// warps concurrently (one warp per pair: three dot products, then the
// rotation of both columns of G and V).
template <bool SMEM>
__global__ void __launch_bounds__(1024) k_jacobi_svd(const SvdJob* __restrict__ jobs, double tol, int* flags,
                                                     double* fc) {
  const SvdJob jb = jobs[blockIdx.x];
  const int ru = *jb.pru, rv = *jb.prv;
  const bool tr = rv > ru;
  const int rows = tr ? rv : ru, cols = tr ? ru : rv;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sig = reinterpret_cast<double*>(smem_raw);
  int* perm = reinterpret_cast<int*>(sig + jb.Rmax);
  double* G;
  double* V;
  int ldg, ldv;
  if (SMEM) {
    G = sig + jb.Rmax + (jb.Rmax + 1) / 2;  // after sig (Rmax doubles) and perm (Rmax ints)
    V = G + (size_t)rows * cols;
    ldg = rows;
    ldv = cols;
  } else {
    G = jb.G;
    V = jb.Vacc;
    ldg = jb.Rmax;
    ldv = jb.Rmax;
  }
  __shared__ int s_rot;
  __shared__ int s_k;
  const int ldm = jb.Rmax;
  for (int64_t e = threadIdx.x; e < (int64_t)rows * cols; e += blockDim.x) {
    const int i = (int)(e % rows), c = (int)(e / rows);
    G[i + (int64_t)c * ldg] = tr ? jb.M[c + (int64_t)i * ldm] : jb.M[i + (int64_t)c * ldm];
  }
  for (int64_t e = threadIdx.x; e < (int64_t)cols * cols; e += blockDim.x) {
    const int i = (int)(e % cols), c = (int)(e / cols);
    V[i + (int64_t)c * ldv] = (i == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int P = cols + (cols & 1);
  const double eps = 1e-15;
  double nflop = 0.0;
  for (int sweep = 0; sweep < 60 && cols > 1; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    int rotated = 0;
    for (int round = 0; round < P - 1; ++round) {
      for (int p = warp; p < P / 2; p += nw) {
        int i, j;
        rr_pair(round, p, P, i, j);
        if (i >= cols || j >= cols) continue;
        double* gi = G + (int64_t)i * ldg;
        double* gj = G + (int64_t)j * ldg;
        double a = 0.0, b = 0.0, g = 0.0;
        for (int r = lane; r < rows; r += 32) {
          const double x = gi[r], y = gj[r];
          a = fma(x, x, a);
          b = fma(y, y, b);
          g = fma(x, y, g);
        }
        a = warp_sum(a);
        b = warp_sum(b);
        g = warp_sum(g);
        nflop += 6.0 * rows;
        if (g != 0.0 && fabs(g) > eps * sqrt(a * b)) {
          nflop += 6.0 * rows + 6.0 * cols;
          const double zeta = (b - a) / (2.0 * g);
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double cs = rsqrt(1.0 + t * t), sn = cs * t;
          for (int r = lane; r < rows; r += 32) {
            const double x = gi[r], y = gj[r];
            gi[r] = cs * x - sn * y;
            gj[r] = sn * x + cs * y;
          }
          double* vi = V + (int64_t)i * ldv;
          double* vj = V + (int64_t)j * ldv;
          for (int r = lane; r < cols; r += 32) {
            const double x = vi[r], y = vj[r];
            vi[r] = cs * x - sn * y;
            vj[r] = sn * x + cs * y;
          }
          rotated = 1;
        }
      }
      __syncthreads();
    }
    if (rotated && lane == 0) s_rot = 1;
    __syncthreads();
    if (!s_rot) break;
    __syncthreads();
  }
  if (fc && lane == 0 && nflop > 0.0) atomicAdd(fc, nflop);
  // singular values = column norms
  for (int c = warp; c < cols; c += nw) {
    double a = 0.0;
    for (int r = lane; r < rows; r += 32) {
      const double x = G[r + (int64_t)c * ldg];
      a = fma(x, x, a);
    }
    a = warp_sum(a);
    if (lane == 0) sig[c] = sqrt(a);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < cols; c += blockDim.x) {
    int pos = 0;
    const double sc = sig[c];
    for (int d = 0; d < cols; ++d) pos += (sig[d] > sc) || (sig[d] == sc && d < c);
    perm[pos] = c;
  }
  if (threadIdx.x == 0) {
    int k = 0;
    for (int c = 0; c < cols; ++c) k += sig[c] > tol;
    if (k > jb.cap) {
      atomicOr(&flags[FLAG_RANK], 1);
      k = jb.cap;
    }
    s_k = k;
    *jb.pk = k;
  }
  __syncthreads();
  const int k = s_k;
  const int ld = jb.Rmax;
  for (int64_t e = threadIdx.x; e < (int64_t)ld * jb.cap; e += blockDim.x) {
    const int r = (int)(e % ld), p = (int)(e / ld);
    double u = 0.0, v = 0.0;
    if (p < k) {
      const int c = perm[p];
      const double s = sig[c];
      if (!tr) {
        if (r < ru) u = G[r + (int64_t)c * ldg];
        if (r < rv) v = V[r + (int64_t)c * ldv];
      } else {
        if (r < ru) u = V[r + (int64_t)c * ldv] * s;
        if (r < rv) v = (s > 0.0) ? G[r + (int64_t)c * ldg] / s : 0.0;
      }
    }
    jb.SU[r + (int64_t)p * ld] = u;
    jb.SV[r + (int64_t)p * ld] = v;
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
// leaving the final R factor in `rdst` (Rmax x Rmax, ld Rmax) and arranging
// for Q [S; 0] to be written into `out` (rows x cap, ld ldo).
static void plan_side(double* W, int64_t ldw, int rows, const int* pR, int Rmax, double* rdst, const double* S,
                      const int* pk, int cap, double* out, int64_t ldo, std::vector<std::vector<QrJob>>& qrl,
                      std::vector<std::vector<ApplyJob>>& apl, std::vector<DBuf>& keep, cudaStream_t st) {
  const int CH = std::max(256, ((4 * Rmax + 31) / 32) * 32);
  struct Node {
    double* J;
    int64_t ldj;
    int rows;
    double* tau;
    int parent;       // index into nodes, -1 for root
    int slot;         // row slot in the parent's matrix
    int64_t out_row;  // for leaves: row offset in `out`
    double* app_out;  // apply output buffer (internal: own temp, leaf: out + row)
    int64_t ldapp;
  };
  std::vector<std::vector<Node>> lv;
  // level 0: chunks
  std::vector<Node> l0;
  const int nch = rows <= CH ? 1 : (rows + CH - 1) / CH;
  for (int c = 0; c < nch; ++c) {
    const int r0 = c * CH;
    const int rr = std::min(CH, rows - r0);
    l0.push_back(Node{W + r0, ldw, rr, nullptr, -1, 0, r0, out + r0, ldo});
  }
  lv.push_back(l0);
  while (lv.back().size() > 1) {
    std::vector<Node>& cur = lv.back();
    std::vector<Node> nxt;
    for (size_t i = 0; i < cur.size(); i += 2) {
      const int nchild = (i + 1 < cur.size()) ? 2 : 1;
      const int mrows = nchild * Rmax;
      keep.emplace_back((size_t)mrows * Rmax * sizeof(double), st);
      double* Mb = keep.back().as<double>();
      nxt.push_back(Node{Mb, mrows, mrows, nullptr, -1, 0, 0, nullptr, 0});
      for (int t = 0; t < nchild; ++t) {
        cur[i + t].parent = (int)nxt.size() - 1;
        cur[i + t].slot = t;
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
        keep.emplace_back((size_t)nd.rows * cap * sizeof(double) + 16, st);
        nd.app_out = keep.back().as<double>();
        nd.ldapp = nd.rows;
      }
    }
  }
  for (size_t l = 0; l < lv.size(); ++l) {
    for (auto& nd : lv[l]) {
      double* dst;
      int64_t ldd;
      if (l + 1 < lv.size()) {
        Node& par = lv[l + 1][nd.parent];
        dst = par.J + (int64_t)nd.slot * Rmax;
        ldd = par.ldj;
      } else {
        dst = rdst;
        ldd = Rmax;
      }
      qrl[l].push_back(QrJob{nd.J, nd.ldj, nd.rows, pR, Rmax, nd.tau, dst, ldd});
      const double* Sin;
      int64_t lds;
      if (l + 1 < lv.size()) {
        Node& par = lv[l + 1][nd.parent];
        Sin = par.app_out + (int64_t)nd.slot * Rmax;
        lds = par.ldapp;
      } else {
        Sin = S;
        lds = Rmax;
      }
      // apply levels are run from the top: store at index (depth-1-l)
      const size_t depth = lv.size();
      apl[depth - 1 - l].push_back(ApplyJob{nd.J, nd.ldj, nd.rows, pR, Rmax, nd.tau, Sin, lds, nd.app_out,
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
  std::vector<int> Rmax(nb);
  size_t wsz = 0, csz = 0;
  int maxseg = 1, maxrows = 1, maxR = 1;
  for (int t = 0; t < nb; ++t) {
    const LrBlock& b = blocks[t];
    int R = 0;
    for (const Seg& s : b.segs) R += s.w;
    Rmax[t] = std::max(R, 1);
    wsz += (size_t)(b.m + b.q) * Rmax[t];
    csz += (size_t)Rmax[t] * Rmax[t] * 3 + 2 * (size_t)Rmax[t] * b.cap;
    maxseg = std::max(maxseg, (int)b.segs.size());
    maxrows = std::max(maxrows, std::max(b.m, b.q));
    maxR = std::max(maxR, Rmax[t]);
    for (const Seg& s : b.segs) {
      ctx->flops += 4.0 * (double)(b.m + b.q) * Rmax[t] * Rmax[t];
      (void)s;
    }
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
    double* RU = cp;
    cp += (size_t)Rm * Rm;
    double* RV = cp;
    cp += (size_t)Rm * Rm;
    double* M = cp;
    cp += (size_t)Rm * Rm;
    double* SU = cp;
    cp += (size_t)Rm * b.cap;
    double* SV = cp;
    cp += (size_t)Rm * b.cap;
    plan_side(g.WU, b.m, b.m, g.R, Rm, RU, SU, b.rank_out, b.cap, b.Uout, b.ldu_out, qrl, apl, keep, st);
    plan_side(g.WV, b.q, b.q, g.R, Rm, RV, SV, b.rank_out, b.cap, b.Vout, b.ldv_out, qrl, apl, keep, st);
    // M = R_U R_V^T (ru x rv, inner dimension R)
    core.push_back(gt(RU, Rm, RV, Rm, M, Rm, Rm, Rm, Rm, 1.0, 0.0, g.ru, g.rv, g.R));
    keep.emplace_back((size_t)Rm * Rm * 2 * sizeof(double) + 16, st);
    double* Gw = keep.back().as<double>();
    svd[t] = SvdJob{M, g.ru, g.rv, Rm, Gw, Gw + (size_t)Rm * Rm, SU, SV, b.rank_out, b.cap};
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
  // 4. SVD + truncation: cores whose working set fits in shared memory take
  // the shared-memory kernel, the rest the global-memory one
  {
    std::vector<SvdJob> small, large;
    int maxR_small = 1, maxR_large = 1;
    size_t need_small = 0;
    for (int t = 0; t < nb; ++t) {
      const size_t R = (size_t)Rmax[t];
      const size_t bytes = R * (sizeof(double) + sizeof(int)) + 2 * R * R * sizeof(double) + 64;
      if (bytes <= kSvdSmemMax) {
        small.push_back(svd[t]);
        maxR_small = std::max(maxR_small, Rmax[t]);
        need_small = std::max(need_small, bytes);
      } else {
        large.push_back(svd[t]);
        maxR_large = std::max(maxR_large, Rmax[t]);
      }
    }
    ProfScope ps(ctx, KID_JACOBI);
    if (!small.empty()) {
      DBuf d = upload(small, st);
      check_cuda(cudaFuncSetAttribute(k_jacobi_svd<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kSvdSmemMax),
                 "smem attr");
      k_jacobi_svd<true><<<(unsigned)small.size(), 1024, need_small, st>>>(d.as<SvdJob>(), tol, ctx->d_flags,
                                                                            fc_ptr(ctx, KID_JACOBI));
      check_launch("k_jacobi_svd");
    }
    if (!large.empty()) {
      DBuf d = upload(large, st);
      const size_t sm = (size_t)maxR_large * (sizeof(double) + sizeof(int)) + 64;
      if (sm > 48 * 1024)
        check_cuda(cudaFuncSetAttribute(k_jacobi_svd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                   "smem attr");
      k_jacobi_svd<false><<<(unsigned)large.size(), 1024, sm, st>>>(d.as<SvdJob>(), tol, ctx->d_flags,
                                                                     fc_ptr(ctx, KID_JACOBI));
      check_launch("k_jacobi_svd");
    }
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

}  // namespace sp
