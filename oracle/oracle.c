/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the hQDWH spectral projector
 * of Kressner & Susnjara, "Fast computation of spectral projectors of banded
 * matrices" (arXiv 1608.01164).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library links, includes or
 * calls this file; only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code with the CUDA path.
 *
 * Every matrix is column-major (Fortran order) with an explicit leading
 * dimension.  Every routine is a direct transcription of a textbook
 * definition or of the paper's algorithm, with no blocking or reordering.
 *
 * Contents (paper passages in brackets):
 *   orc_sturm_count        inertia of a symmetric tridiagonal matrix
 *                          (Sylvester + LDL^T recurrence) [Sec. 1: lambda_nu < mu < lambda_nu+1]
 *   orc_band_ldl_count     inertia of a symmetric banded matrix by an
 *                          unpivoted banded LDL^T in long double
 *   orc_householder_tridiag, orc_tridiag_qr, orc_eigh
 *                          dense symmetric eigensolver (Householder reduction,
 *                          implicit symmetric QR with Wilkinson shift)
 *                          -> Pi = V_nu V_nu^T  [Sec. 2, polar/sign relation]
 *   orc_jacobi_eig_ld      cyclic two-sided Jacobi in long double (an
 *                          independent brute-force eigensolver for n <= 64)
 *   orc_qdwh_h, orc_qdwh_params
 *                          QDWH dynamic weights [Eq. (qdwh_parameters_abc)]
 *   orc_qdwh_dense         dense QDWH: QR-based step(s) [Eq. (qdwh_qr_reccur)]
 *                          then Cholesky-based steps [Eq. (qdwh_chol_reccur)],
 *                          stopped when |1 - l_k| <= delta [Sec. 2.1]
 *   orc_fastqr_replay      dense replay of the fast QR of [cA; I]
 *                          [Algorithm 1 (b = 1) and Algorithm 2 (b > 1)]
 */
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

/* ------------------------------------------------------------------------ */
/* Inertia counts                                                            */
/* ------------------------------------------------------------------------ */

/* Number of eigenvalues of the symmetric tridiagonal T (diagonal a[0..n-1],
 * off-diagonal e[0..n-2]) that are strictly smaller than sigma.
 * T - sigma I = L D L^T with d_0 = a_0 - sigma and
 * d_i = (a_i - sigma) - e_{i-1}^2 / d_{i-1}; by Sylvester's law of inertia the
 * count is the number of negative d_i.  A pivot that is exactly or nearly zero
 * is replaced by -pivmin (Kahan's safeguard), which counts sigma as lying just
 * above the corresponding eigenvalue. */
long orc_sturm_count(long n, const double* a, const double* e, double sigma) {
  double emax2 = 1.0;
  for (long i = 0; i + 1 < n; ++i) {
    double t = e[i] * e[i];
    if (t > emax2) emax2 = t;
  }
  const double pivmin = DBL_MIN * emax2;
  long count = 0;
  double d = 1.0;
  for (long i = 0; i < n; ++i) {
    double off = (i == 0) ? 0.0 : e[i - 1] * e[i - 1] / d;
    d = (a[i] - sigma) - off;
    if (fabs(d) < pivmin) d = -pivmin;
    if (d < 0.0) ++count;
  }
  return count;
}

/* Number of eigenvalues < sigma of the symmetric banded matrix given in lower
 * band storage ab[(i-j) + j*ldab] = A(i,j), 0 <= i-j <= b.  Computes the
 * unpivoted banded factorisation A - sigma I = L D L^T in long double and
 * counts negative pivots (Sylvester).  A vanishing pivot is replaced by
 * -pivmin, as in the tridiagonal recurrence.  For b = 1 this is the same
 * recurrence as orc_sturm_count. */
long orc_band_ldl_count(long n, long b, const double* ab, long ldab, double sigma) {
  long double* L = (long double*)calloc((size_t)(b + 1) * (size_t)n, sizeof(long double));
  long double* D = (long double*)calloc((size_t)n, sizeof(long double));
  if (!L || !D) { free(L); free(D); return -1; }
  long double amax = 1.0L;
  for (long j = 0; j < n; ++j)
    for (long k = 0; k <= b && j + k < n; ++k) {
      long double t = fabsl((long double)ab[IDX(k, j, ldab)]);
      if (t > amax) amax = t;
    }
  const long double pivmin = (long double)DBL_MIN * amax * amax;
  long count = 0;
  /* L stored in band form: L[(i-j) + j*(b+1)] = L(i,j) for 1 <= i-j <= b. */
  for (long j = 0; j < n; ++j) {
    long double dj = (long double)ab[IDX(0, j, ldab)] - (long double)sigma;
    for (long k = (j - b > 0 ? j - b : 0); k < j; ++k) {
      long double l = L[IDX(j - k, k, b + 1)];
      dj -= l * l * D[k];
    }
    if (fabsl(dj) < pivmin) dj = -pivmin;
    D[j] = dj;
    if (dj < 0) ++count;
    for (long i = j + 1; i <= j + b && i < n; ++i) {
      long double s = (long double)ab[IDX(i - j, j, ldab)];
      for (long k = (i - b > 0 ? i - b : 0); k < j; ++k)
        s -= L[IDX(i - k, k, b + 1)] * L[IDX(j - k, k, b + 1)] * D[k];
      L[IDX(i - j, j, b + 1)] = s / dj;
    }
  }
  free(L);
  free(D);
  return count;
}

/* Dense symmetric matrix from lower band storage, shifted by -mu. */
void orc_band_to_dense(long n, long b, const double* ab, long ldab, double mu, double* A, long lda) {
  for (long j = 0; j < n; ++j)
    for (long i = 0; i < n; ++i) A[IDX(i, j, lda)] = 0.0;
  for (long j = 0; j < n; ++j)
    for (long k = 0; k <= b && j + k < n; ++k) {
      double v = ab[IDX(k, j, ldab)];
      A[IDX(j + k, j, lda)] = v;
      A[IDX(j, j + k, lda)] = v;
    }
  for (long j = 0; j < n; ++j) A[IDX(j, j, lda)] -= mu;
}

/* ------------------------------------------------------------------------ */
/* Dense symmetric eigensolver                                               */
/* ------------------------------------------------------------------------ */

/* Householder reduction of the symmetric A (n x n, lower and upper parts both
 * referenced and destroyed) to tridiagonal form T = Q^T A Q.  On return d, e
 * hold T's diagonal and sub-diagonal and Q (n x n) the accumulated product of
 * reflectors H_0 H_1 ... H_{n-3}. */
void orc_householder_tridiag(long n, double* A, long lda, double* d, double* e, double* Q, long ldq) {
  for (long j = 0; j < n; ++j)
    for (long i = 0; i < n; ++i) Q[IDX(i, j, ldq)] = (i == j) ? 1.0 : 0.0;
  double* v = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* p = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (long k = 0; k + 2 < n; ++k) {
    long m = n - k - 1; /* length of x = A(k+1:n-1, k) */
    double sigma = 0.0;
    for (long i = 1; i < m; ++i) sigma += A[IDX(k + 1 + i, k, lda)] * A[IDX(k + 1 + i, k, lda)];
    double x0 = A[IDX(k + 1, k, lda)];
    if (sigma == 0.0) continue; /* already tridiagonal in this column */
    double mu = sqrt(x0 * x0 + sigma);
    /* v = x - ||x|| e_1 (first entry formed without cancellation), scaled so v_0 = 1. */
    double v0 = (x0 <= 0.0) ? x0 - mu : -sigma / (x0 + mu);
    double beta = 2.0 * v0 * v0 / (sigma + v0 * v0);
    v[0] = 1.0;
    for (long i = 1; i < m; ++i) v[i] = A[IDX(k + 1 + i, k, lda)] / v0;
    /* p = beta * A22 v */
    for (long i = 0; i < m; ++i) {
      double s = 0.0;
      for (long jj = 0; jj < m; ++jj) s += A[IDX(k + 1 + i, k + 1 + jj, lda)] * v[jj];
      p[i] = beta * s;
    }
    /* w = p - (beta/2)(p^T v) v, stored in p */
    double pv = 0.0;
    for (long i = 0; i < m; ++i) pv += p[i] * v[i];
    double half = 0.5 * beta * pv;
    for (long i = 0; i < m; ++i) p[i] -= half * v[i];
    /* A22 -= v w^T + w v^T */
    for (long jj = 0; jj < m; ++jj)
      for (long i = 0; i < m; ++i)
        A[IDX(k + 1 + i, k + 1 + jj, lda)] -= v[i] * p[jj] + p[i] * v[jj];
    /* new column k below the diagonal: (||x||, 0, ..., 0), since the
     * reflector built from v = x - ||x|| e_1 maps x to ||x|| e_1. */
    double alpha = mu;
    A[IDX(k + 1, k, lda)] = alpha;
    A[IDX(k, k + 1, lda)] = alpha;
    for (long i = 1; i < m; ++i) {
      A[IDX(k + 1 + i, k, lda)] = 0.0;
      A[IDX(k, k + 1 + i, lda)] = 0.0;
    }
    /* Q(:, k+1:n) <- Q(:, k+1:n) (I - beta v v^T) */
    for (long i = 0; i < n; ++i) {
      double s = 0.0;
      for (long jj = 0; jj < m; ++jj) s += Q[IDX(i, k + 1 + jj, ldq)] * v[jj];
      s *= beta;
      for (long jj = 0; jj < m; ++jj) Q[IDX(i, k + 1 + jj, ldq)] -= s * v[jj];
    }
  }
  for (long i = 0; i < n; ++i) d[i] = A[IDX(i, i, lda)];
  for (long i = 0; i + 1 < n; ++i) e[i] = A[IDX(i + 1, i, lda)];
  free(v);
  free(p);
}

/* Implicit symmetric QR iteration with Wilkinson shift on the tridiagonal
 * (d, e); the rotations are accumulated into the columns of Z (rows 0..nz-1),
 * so on return T = Z^T A Z with T diagonal when Z enters as the reduction's
 * Q.  Returns 0 on success, -1 if an unreduced block fails to converge. */
int orc_tridiag_qr(long n, double* d, double* e, long nz, double* Z, long ldz) {
  const double eps = DBL_EPSILON * 0.5;
  long hi = n - 1;
  long iter = 0, maxiter = 60 * (n > 1 ? n : 1);
  while (hi > 0) {
    if (fabs(e[hi - 1]) <= eps * (fabs(d[hi - 1]) + fabs(d[hi])) || e[hi - 1] == 0.0) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    long lo = hi - 1;
    while (lo > 0 && !(fabs(e[lo - 1]) <= eps * (fabs(d[lo - 1]) + fabs(d[lo])) || e[lo - 1] == 0.0)) --lo;
    if (lo > 0) e[lo - 1] = 0.0;
    if (++iter > maxiter) return -1;
    /* Wilkinson shift: eigenvalue of the trailing 2x2 closer to d[hi]. */
    double delta = 0.5 * (d[hi - 1] - d[hi]);
    double f = e[hi - 1];
    double sgn = (delta >= 0.0) ? 1.0 : -1.0;
    double shift = d[hi] - f * f / (delta + sgn * hypot(delta, f));
    double x = d[lo] - shift, z = e[lo];
    double bulge = 0.0;
    for (long k = lo; k < hi; ++k) {
      double r = hypot(x, z);
      double c = (r == 0.0) ? 1.0 : x / r;
      double s = (r == 0.0) ? 0.0 : z / r;
      if (k > lo) e[k - 1] = r;
      double a0 = d[k], a1 = d[k + 1], g = e[k];
      d[k] = c * c * a0 + 2.0 * c * s * g + s * s * a1;
      d[k + 1] = s * s * a0 - 2.0 * c * s * g + c * c * a1;
      e[k] = c * s * (a1 - a0) + (c * c - s * s) * g;
      if (k + 1 < hi) {
        double g2 = e[k + 1];
        bulge = s * g2;
        e[k + 1] = c * g2;
        x = e[k];
        z = bulge;
      }
      for (long i = 0; i < nz; ++i) {
        double zk = Z[IDX(i, k, ldz)], zk1 = Z[IDX(i, k + 1, ldz)];
        Z[IDX(i, k, ldz)] = c * zk + s * zk1;
        Z[IDX(i, k + 1, ldz)] = -s * zk + c * zk1;
      }
    }
  }
  return 0;
}

/* Sort eigenpairs ascending (selection sort on w, swapping columns of V). */
static void sort_eigenpairs(long n, double* w, double* V, long ldv) {
  for (long i = 0; i < n; ++i) {
    long m = i;
    for (long j = i + 1; j < n; ++j)
      if (w[j] < w[m]) m = j;
    if (m != i) {
      double t = w[i]; w[i] = w[m]; w[m] = t;
      for (long r = 0; r < n; ++r) {
        double u = V[IDX(r, i, ldv)];
        V[IDX(r, i, ldv)] = V[IDX(r, m, ldv)];
        V[IDX(r, m, ldv)] = u;
      }
    }
  }
}

/* Eigen-decomposition of the dense symmetric A (destroyed): A = V diag(w) V^T,
 * w ascending.  Returns 0 on success. */
int orc_eigh(long n, double* A, long lda, double* w, double* V, long ldv) {
  double* e = (double*)calloc((size_t)(n > 1 ? n : 1), sizeof(double));
  orc_householder_tridiag(n, A, lda, w, e, V, ldv);
  int rc = orc_tridiag_qr(n, w, e, n, V, ldv);
  free(e);
  if (rc == 0) sort_eigenpairs(n, w, V, ldv);
  return rc;
}

/* Eigen-decomposition of a symmetric tridiagonal matrix (a, e) directly. */
int orc_eigh_tridiag(long n, const double* a, const double* e, double* w, double* V, long ldv) {
  double* ee = (double*)calloc((size_t)(n > 1 ? n : 1), sizeof(double));
  for (long i = 0; i < n; ++i) w[i] = a[i];
  for (long i = 0; i + 1 < n; ++i) ee[i] = e[i];
  for (long j = 0; j < n; ++j)
    for (long i = 0; i < n; ++i) V[IDX(i, j, ldv)] = (i == j) ? 1.0 : 0.0;
  int rc = orc_tridiag_qr(n, w, ee, n, V, ldv);
  free(ee);
  if (rc == 0) sort_eigenpairs(n, w, V, ldv);
  return rc;
}

/* Spectral projector onto the eigenvalues < mu of the dense symmetric A:
 * Pi = V_nu V_nu^T.  A is not modified.  Returns nu (or -1 on failure). */
long orc_projector(long n, const double* A, long lda, double mu, double* P, long ldp, double* w_out) {
  double* B = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  double* V = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  double* w = (double*)malloc(sizeof(double) * (size_t)n);
  for (long j = 0; j < n; ++j)
    for (long i = 0; i < n; ++i) B[IDX(i, j, n)] = A[IDX(i, j, lda)];
  long nu = -1;
  if (orc_eigh(n, B, n, w, V, n) == 0) {
    nu = 0;
    while (nu < n && w[nu] < mu) ++nu;
    for (long j = 0; j < n; ++j)
      for (long i = 0; i < n; ++i) {
        double s = 0.0;
        for (long k = 0; k < nu; ++k) s += V[IDX(i, k, n)] * V[IDX(j, k, n)];
        P[IDX(i, j, ldp)] = s;
      }
    if (w_out)
      for (long i = 0; i < n; ++i) w_out[i] = w[i];
  }
  free(B);
  free(V);
  free(w);
  return nu;
}

/* Cyclic two-sided Jacobi method in long double for the symmetric A
 * (n <= a few hundred; intended for n <= 64).  Textbook rotation choice:
 * theta = (a_qq - a_pp) / (2 a_pq), t = sign(theta)/(|theta| + sqrt(theta^2+1)).
 * On return w (unsorted -> sorted ascending) and V (columns = eigenvectors).
 * Returns the number of sweeps, or -1 if 100 sweeps did not converge. */
int orc_jacobi_eig_ld(long n, const double* A, long lda, double* w, double* V, long ldv) {
  long double* M = (long double*)malloc(sizeof(long double) * (size_t)n * (size_t)n);
  long double* Z = (long double*)malloc(sizeof(long double) * (size_t)n * (size_t)n);
  for (long j = 0; j < n; ++j)
    for (long i = 0; i < n; ++i) {
      M[IDX(i, j, n)] = (long double)A[IDX(i, j, lda)];
      Z[IDX(i, j, n)] = (i == j) ? 1.0L : 0.0L;
    }
  /* A sweep rotates every pair (p, q) whose a_pq is not negligible
   * (|a_pq| > eps_ld sqrt(|a_pp a_qq|)); negligible entries are set to zero.
   * The iteration stops after a sweep with no rotation. */
  int sweeps = 0;
  for (; sweeps < 100; ++sweeps) {
    long rotations = 0;
    for (long p = 0; p < n - 1; ++p)
      for (long q = p + 1; q < n; ++q) {
        long double apq = M[IDX(p, q, n)];
        if (fabsl(apq) <= LDBL_EPSILON * sqrtl(fabsl(M[IDX(p, p, n)] * M[IDX(q, q, n)])) || apq == 0.0L) {
          M[IDX(p, q, n)] = 0.0L;
          M[IDX(q, p, n)] = 0.0L;
          continue;
        }
        ++rotations;
        long double theta = (M[IDX(q, q, n)] - M[IDX(p, p, n)]) / (2.0L * apq);
        long double t = (theta >= 0 ? 1.0L : -1.0L) / (fabsl(theta) + sqrtl(theta * theta + 1.0L));
        long double c = 1.0L / sqrtl(t * t + 1.0L), s = t * c;
        for (long k = 0; k < n; ++k) { /* columns p, q */
          long double mkp = M[IDX(k, p, n)], mkq = M[IDX(k, q, n)];
          M[IDX(k, p, n)] = c * mkp - s * mkq;
          M[IDX(k, q, n)] = s * mkp + c * mkq;
        }
        for (long k = 0; k < n; ++k) { /* rows p, q */
          long double mpk = M[IDX(p, k, n)], mqk = M[IDX(q, k, n)];
          M[IDX(p, k, n)] = c * mpk - s * mqk;
          M[IDX(q, k, n)] = s * mpk + c * mqk;
        }
        for (long k = 0; k < n; ++k) {
          long double zkp = Z[IDX(k, p, n)], zkq = Z[IDX(k, q, n)];
          Z[IDX(k, p, n)] = c * zkp - s * zkq;
          Z[IDX(k, q, n)] = s * zkp + c * zkq;
        }
      }
    if (rotations == 0) break;
  }
  for (long i = 0; i < n; ++i) w[i] = (double)M[IDX(i, i, n)];
  for (long j = 0; j < n; ++j)
    for (long i = 0; i < n; ++i) V[IDX(i, j, ldv)] = (double)Z[IDX(i, j, n)];
  sort_eigenpairs(n, w, V, ldv);
  free(M);
  free(Z);
  return sweeps < 100 ? sweeps : -1;
}

/* ------------------------------------------------------------------------ */
/* QDWH scalar recurrence [Sec. 2.1]                                         */
/* ------------------------------------------------------------------------ */

/* h(l) = sqrt(1+g) + 0.5 sqrt(8 - 4g + 8(2-l^2)/(l^2 sqrt(1+g))),
 * g = cbrt(4(1-l^2)/l^4). */
double orc_qdwh_h(double l) {
  double l2 = l * l;
  double g = cbrt(4.0 * (1.0 - l2) / (l2 * l2));
  double s = sqrt(1.0 + g);
  return s + 0.5 * sqrt(8.0 - 4.0 * g + 8.0 * (2.0 - l2) / (l2 * s));
}

/* a = h(l), b = (a-1)^2/4, c = a+b-1, and the next lower bound
 * l' = l (a + b l^2) / (1 + c l^2). */
void orc_qdwh_params(double l, double* a, double* b, double* c, double* lnext) {
  double aa = orc_qdwh_h(l);
  double bb = 0.25 * (aa - 1.0) * (aa - 1.0);
  double cc = aa + bb - 1.0;
  *a = aa;
  *b = bb;
  *c = cc;
  *lnext = l * (aa + bb * l * l) / (1.0 + cc * l * l);
}

/* ------------------------------------------------------------------------ */
/* Dense kernels used by the dense QDWH                                      */
/* ------------------------------------------------------------------------ */

/* C = alpha * op(A) op(B) + beta C with op = transpose when ta/tb != 0. */
static void gemm(int ta, int tb, long m, long n, long k, double alpha, const double* A, long lda,
                 const double* B, long ldb, double beta, double* C, long ldc) {
  for (long j = 0; j < n; ++j)
    for (long i = 0; i < m; ++i) {
      double s = 0.0;
      for (long p = 0; p < k; ++p) {
        double x = ta ? A[IDX(p, i, lda)] : A[IDX(i, p, lda)];
        double y = tb ? B[IDX(j, p, ldb)] : B[IDX(p, j, ldb)];
        s += x * y;
      }
      C[IDX(i, j, ldc)] = alpha * s + (beta == 0.0 ? 0.0 : beta * C[IDX(i, j, ldc)]);
    }
}

/* Householder QR of the m x n matrix M (m >= n, destroyed): on return Q holds
 * the first n columns of the orthogonal factor (m x n) and R the n x n upper
 * triangle. */
static void householder_qr_thin(long m, long n, double* M, long ldm, double* Q, long ldq, double* R, long ldr) {
  double* tau = (double*)calloc((size_t)n, sizeof(double));
  for (long k = 0; k < n; ++k) {
    double sigma = 0.0;
    for (long i = k + 1; i < m; ++i) sigma += M[IDX(i, k, ldm)] * M[IDX(i, k, ldm)];
    double x0 = M[IDX(k, k, ldm)];
    if (sigma == 0.0) { tau[k] = 0.0; continue; }
    double mu = sqrt(x0 * x0 + sigma);
    double v0 = (x0 <= 0.0) ? x0 - mu : -sigma / (x0 + mu);
    tau[k] = 2.0 * v0 * v0 / (sigma + v0 * v0);
    for (long i = k + 1; i < m; ++i) M[IDX(i, k, ldm)] /= v0; /* v below the unit */
    M[IDX(k, k, ldm)] = mu; /* v = x - ||x|| e_1 maps x to ||x|| e_1 */
    for (long j = k + 1; j < n; ++j) {
      double s = M[IDX(k, j, ldm)];
      for (long i = k + 1; i < m; ++i) s += M[IDX(i, k, ldm)] * M[IDX(i, j, ldm)];
      s *= tau[k];
      M[IDX(k, j, ldm)] -= s;
      for (long i = k + 1; i < m; ++i) M[IDX(i, j, ldm)] -= s * M[IDX(i, k, ldm)];
    }
  }
  for (long j = 0; j < n; ++j)
    for (long i = 0; i < n; ++i) R[IDX(i, j, ldr)] = (i <= j) ? M[IDX(i, j, ldm)] : 0.0;
  /* Q = H_0 ... H_{n-1} [I_n; 0], accumulated backwards. */
  for (long j = 0; j < n; ++j)
    for (long i = 0; i < m; ++i) Q[IDX(i, j, ldq)] = (i == j) ? 1.0 : 0.0;
  for (long k = n - 1; k >= 0; --k) {
    if (tau[k] == 0.0) continue;
    for (long j = k; j < n; ++j) {
      double s = Q[IDX(k, j, ldq)];
      for (long i = k + 1; i < m; ++i) s += M[IDX(i, k, ldm)] * Q[IDX(i, j, ldq)];
      s *= tau[k];
      Q[IDX(k, j, ldq)] -= s;
      for (long i = k + 1; i < m; ++i) Q[IDX(i, j, ldq)] -= s * M[IDX(i, k, ldm)];
    }
  }
  free(tau);
}

/* Upper Cholesky factor W (W^T W = Z) of the SPD matrix Z; returns 0 or the
 * 1-based index of the first non-positive pivot. */
static long cholesky_upper(long n, const double* Z, long ldz, double* W, long ldw) {
  for (long j = 0; j < n; ++j)
    for (long i = 0; i < n; ++i) W[IDX(i, j, ldw)] = 0.0;
  for (long j = 0; j < n; ++j) {
    double s = Z[IDX(j, j, ldz)];
    for (long k = 0; k < j; ++k) s -= W[IDX(k, j, ldw)] * W[IDX(k, j, ldw)];
    if (!(s > 0.0)) return j + 1;
    double wjj = sqrt(s);
    W[IDX(j, j, ldw)] = wjj;
    for (long i = j + 1; i < n; ++i) {
      double t = Z[IDX(j, i, ldz)];
      for (long k = 0; k < j; ++k) t -= W[IDX(k, j, ldw)] * W[IDX(k, i, ldw)];
      W[IDX(j, i, ldw)] = t / wjj;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Dense QDWH                                                                */
/* ------------------------------------------------------------------------ */

/* Dense QDWH for the symmetric nonsingular A (n x n, not modified) [Sec. 2.1]:
 *   X_0 = A / alpha; while |1 - l_k| > delta: a_k, b_k, c_k from l_k;
 *   QR-based step   X <- (b/c) X + (1/sqrt c)(a - b/c) Q1 Q2^T,
 *                   [sqrt(c) X; I] = [Q1; Q2] R                  (Eq. qdwh_qr_reccur)
 *   or Cholesky step Z = I + c X^T X, W = chol(Z),
 *                   X <- (b/c) X + (a - b/c)(X W^{-1}) W^{-T}     (Eq. qdwh_chol_reccur)
 *   l_{k+1} = l_k (a + b l_k^2) / (1 + c l_k^2).
 * Step policy: if qr_policy >= 1, the first qr_policy steps are QR-based
 * (the paper's choice is exactly one, Sec. 2.2); if qr_policy == -1, QR-based
 * steps are used while c_k > 100 (the switching rule the paper compares
 * against).  Outputs the final iterate U (n x n), and per-iteration
 * parameters (arrays of length >= maxit): l_hist[k] = l_k, a/b/c_hist,
 * kind_hist[k] = 1 for QR, 2 for Cholesky; optionally the first iterate X1.
 * Returns the number of iterations, or -1 on a Cholesky breakdown / too many
 * iterations. */
int orc_qdwh_dense(long n, const double* A, long lda, double alpha, double l0, double delta, int qr_policy,
                   int maxit, double* U, long ldu, double* l_hist, double* a_hist, double* b_hist,
                   double* c_hist, int* kind_hist, double* X1, long ldx1) {
  size_t nn = (size_t)n * (size_t)n;
  double* X = (double*)malloc(sizeof(double) * nn);
  double* T1 = (double*)malloc(sizeof(double) * nn * 2);
  double* T2 = (double*)malloc(sizeof(double) * nn * 2);
  double* T3 = (double*)malloc(sizeof(double) * nn);
  for (long j = 0; j < n; ++j)
    for (long i = 0; i < n; ++i) X[IDX(i, j, n)] = A[IDX(i, j, lda)] / alpha;
  double l = l0;
  int k = 0;
  int rc = 0;
  while (fabs(1.0 - l) > delta) {
    if (k >= maxit) { rc = -1; break; }
    double a, b, c, lnext;
    orc_qdwh_params(l, &a, &b, &c, &lnext);
    l_hist[k] = l; a_hist[k] = a; b_hist[k] = b; c_hist[k] = c;
    int use_qr = (qr_policy >= 1) ? (k < qr_policy) : (qr_policy == -1 && c > 100.0);
    kind_hist[k] = use_qr ? 1 : 2;
    if (use_qr) {
      /* M = [sqrt(c) X; I] (2n x n) in T1; thin Q in T2 (2n x n); R in T3. */
      double sc = sqrt(c);
      for (long j = 0; j < n; ++j)
        for (long i = 0; i < n; ++i) {
          T1[IDX(i, j, 2 * n)] = sc * X[IDX(i, j, n)];
          T1[IDX(n + i, j, 2 * n)] = (i == j) ? 1.0 : 0.0;
        }
      householder_qr_thin(2 * n, n, T1, 2 * n, T2, 2 * n, T3, n);
      /* T3 <- Q1 Q2^T */
      gemm(0, 1, n, n, n, 1.0, T2, 2 * n, T2 + n, 2 * n, 0.0, T3, n);
      double w1 = b / c, w2 = (a - b / c) / sc;
      for (size_t t = 0; t < nn; ++t) X[t] = w1 * X[t] + w2 * T3[t];
    } else {
      /* Z = I + c X^T X in T1 (n x n); W in T2 (n x n). */
      gemm(1, 0, n, n, n, c, X, n, X, n, 0.0, T1, n);
      for (long i = 0; i < n; ++i) T1[IDX(i, i, n)] += 1.0;
      if (cholesky_upper(n, T1, n, T2, n) != 0) { rc = -1; break; }
      /* Y W = X  -> rows of Y by forward substitution on W^T: Y(:,j) */
      for (long r = 0; r < n; ++r) /* row r of Y */
        for (long j = 0; j < n; ++j) {
          double s = X[IDX(r, j, n)];
          for (long q = 0; q < j; ++q) s -= T3[IDX(r, q, n)] * T2[IDX(q, j, n)];
          T3[IDX(r, j, n)] = s / T2[IDX(j, j, n)];
        }
      /* V W^T = Y -> V(:, j) for j = n-1 .. 0 */
      for (long r = 0; r < n; ++r)
        for (long j = n - 1; j >= 0; --j) {
          double s = T3[IDX(r, j, n)];
          for (long q = j + 1; q < n; ++q) s -= T1[IDX(r, q, n)] * T2[IDX(j, q, n)];
          T1[IDX(r, j, n)] = s / T2[IDX(j, j, n)];
        }
      double w1 = b / c, w2 = a - b / c;
      for (size_t t = 0; t < nn; ++t) X[t] = w1 * X[t] + w2 * T1[t];
    }
    if (k == 0 && X1)
      for (long j = 0; j < n; ++j)
        for (long i = 0; i < n; ++i) X1[IDX(i, j, ldx1)] = X[IDX(i, j, n)];
    l = lnext;
    ++k;
  }
  for (long j = 0; j < n; ++j)
    for (long i = 0; i < n; ++i) U[IDX(i, j, ldu)] = X[IDX(i, j, n)];
  free(X);
  free(T1);
  free(T2);
  free(T3);
  return rc == 0 ? k : -1;
}

/* ------------------------------------------------------------------------ */
/* Dense replay of the fast QR of [cA; I]  [Algorithms 1 and 2]              */
/* ------------------------------------------------------------------------ */

/* A Givens rotation acting on the ordered row pair (p, q) of R: its 2x2 block
 * [[c, s], [-s, c]] maps (R(p,col), R(q,col)) = (f, g) to (r, 0) with
 * r = hypot(f, g) >= 0.  The same rotation multiplies Q from the right:
 * Q(:,p) <- c Q(:,p) + s Q(:,q), Q(:,q) <- -s Q(:,p) + c Q(:,q). */
typedef struct {
  double* R; long ldr; long rcols;
  double* Q; long ldq; long qrows;
  long* P; long* Qi; double* C; double* S;
  long count;
} replay_t;

static void replay_rot(replay_t* st, long p, long q, long col) {
  double f = st->R[IDX(p, col, st->ldr)], g = st->R[IDX(q, col, st->ldr)];
  double r = hypot(f, g);
  double c = (r == 0.0) ? 1.0 : f / r;
  double s = (r == 0.0) ? 0.0 : g / r;
  for (long j = 0; j < st->rcols; ++j) {
    double x = st->R[IDX(p, j, st->ldr)], y = st->R[IDX(q, j, st->ldr)];
    st->R[IDX(p, j, st->ldr)] = c * x + s * y;
    st->R[IDX(q, j, st->ldr)] = -s * x + c * y;
  }
  st->R[IDX(q, col, st->ldr)] = 0.0; /* exact zero by construction */
  if (st->Q)
    for (long i = 0; i < st->qrows; ++i) {
      double x = st->Q[IDX(i, p, st->ldq)], y = st->Q[IDX(i, q, st->ldq)];
      st->Q[IDX(i, p, st->ldq)] = c * x + s * y;
      st->Q[IDX(i, q, st->ldq)] = -s * x + c * y;
    }
  if (st->P) {
    st->P[st->count] = p;
    st->Qi[st->count] = q;
    st->C[st->count] = c;
    st->S[st->count] = s;
  }
  st->count++;
}

/* Fast QR decomposition of [scale * A; I] for the symmetric banded A given in
 * lower band storage (bandwidth b >= 1; b = 1 is Algorithm 1, which is
 * Algorithm 2 with b = 1).  R (2n x n, ldr >= 2n) receives the reduced matrix,
 * Q (2n x 2n, ldq >= 2n, may be NULL) the accumulated orthogonal factor.  If
 * P is non-NULL the rotations are recorded in order: pair (P[t], Qi[t]) of
 * 0-based row indices, cosine C[t], sine S[t].  Row n of the stacked matrix is
 * the paper's row n+1, and so on.  Returns the number of rotations.
 *
 * Step i (1-based) of Algorithm 2:
 *   alpha_{i,i}:  rows (n+1, n+i), annihilate R(n+i, i)
 *   alpha_{i,j}:  annihilate R(n+i, j) against row n+j, j = i+1..min(n, i+b-1)
 *   beta_i:       rows (i, n+1), annihilate R(n+1, i)
 *   gamma_{i,j}:  rows (i, j), annihilate R(j, i), j = i+1..min(n, i+b), i < n
 * Step 1 consists of beta_1 and gamma_{1,j} only. */
long orc_fastqr_replay(long n, long b, const double* ab, long ldab, double scale, double* R, long ldr,
                       double* Q, long ldq, long* P, long* Qi, double* C, double* S) {
  replay_t st;
  st.R = R; st.ldr = ldr; st.rcols = n;
  st.Q = Q; st.ldq = ldq; st.qrows = 2 * n;
  st.P = P; st.Qi = Qi; st.C = C; st.S = S; st.count = 0;
  for (long j = 0; j < n; ++j)
    for (long i = 0; i < 2 * n; ++i) R[IDX(i, j, ldr)] = 0.0;
  for (long j = 0; j < n; ++j)
    for (long k = 0; k <= b && j + k < n; ++k) {
      double v = scale * ab[IDX(k, j, ldab)];
      R[IDX(j + k, j, ldr)] = v;
      R[IDX(j, j + k, ldr)] = v;
    }
  for (long i = 0; i < n; ++i) R[IDX(n + i, i, ldr)] = 1.0;
  if (Q)
    for (long j = 0; j < 2 * n; ++j)
      for (long i = 0; i < 2 * n; ++i) Q[IDX(i, j, ldq)] = (i == j) ? 1.0 : 0.0;
  for (long i = 1; i <= n; ++i) {
    long ci = i - 1; /* 0-based column / row index of step i */
    if (i >= 2) {
      replay_rot(&st, n, n + ci, ci); /* alpha_{i,i} */
      long jmax = (n < b + i - 1) ? n : b + i - 1;
      for (long j = i + 1; j <= jmax; ++j) replay_rot(&st, n + (j - 1), n + ci, j - 1); /* alpha_{i,j} */
    }
    replay_rot(&st, ci, n, ci); /* beta_i */
    if (i < n) {
      long jmax = (n < b + i) ? n : b + i;
      for (long j = i + 1; j <= jmax; ++j) replay_rot(&st, ci, j - 1, ci); /* gamma_{i,j} */
    }
  }
  return st.count;
}
