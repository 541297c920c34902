"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test ties an oracle routine to something other than itself: a closed
form, an independent algorithm, a library routine, or an exact invariant.
"""
import math

import numpy as np
import pytest

import oracle
import sp_inputs


def laplace_eigs(n):
    k = np.arange(1, n + 1)
    return 2.0 - 2.0 * np.cos(k * math.pi / (n + 1))


# ------------------------------------------------------------- inertia ----

def test_sturm_count_laplace_closed_form():
    """nu(sigma) on tridiag(-1,2,-1) matches the closed-form eigenvalues
    lambda_k = 2 - 2 cos(k pi/(n+1)) (Sec. 6.2, 1D Laplace) at every gap."""
    n = 200
    lam = laplace_eigs(n)
    ab = sp_inputs.laplace(n)
    assert oracle.sturm_count(ab, lam[0] - 1.0) == 0
    assert oracle.sturm_count(ab, lam[-1] + 1.0) == n
    for k in range(1, n):
        sigma = 0.5 * (lam[k - 1] + lam[k])
        assert oracle.sturm_count(ab, sigma) == k


def test_laplace_mu_is_two():
    """n = 1024: cos(512 pi/1025) = -cos(513 pi/1025), so the midpoint of
    lambda_512 and lambda_513 is exactly 2 and nu(2) = 512."""
    ab = sp_inputs.laplace(1024)
    assert oracle.sturm_count(ab, 2.0) == 512
    sh = oracle.locate_mu(ab, 512)
    assert abs(sh.mu - 2.0) < 1e-12
    lam = laplace_eigs(1024)
    tol = 1e-14  # the closed-form cosines are themselves rounded
    assert sh.lam_nu[0] - tol <= lam[511] < sh.lam_nu[1] + tol
    assert sh.lam_nu1[0] - tol <= lam[512] < sh.lam_nu1[1] + tol


@pytest.mark.parametrize("b", [2, 4, 8])
def test_band_ldl_count_vs_library_eigvalsh(b):
    """Banded inertia (unpivoted LDL^T, long double) against LAPACK's
    eigenvalues of the same dense matrix at shifts between eigenvalues."""
    n = 240
    ab = sp_inputs.normal_band(n, b, seed=11 + b)
    A = sp_inputs.dense_from_band(ab)
    w = np.linalg.eigvalsh(A)
    rng = np.random.default_rng(b)
    for k in rng.choice(np.arange(1, n), size=40, replace=False):
        sigma = 0.5 * (w[k - 1] + w[k])
        if w[k] - w[k - 1] < 1e-9:
            continue
        assert oracle.band_count(ab, sigma) == k


def test_band_count_monotone_and_extremes():
    ab = sp_inputs.uniform_band(300, 3, seed=5)
    lo, hi = oracle.gershgorin(ab)
    xs = np.linspace(lo - 0.1, hi + 0.1, 60)
    counts = [oracle.band_count(ab, x) for x in xs]
    assert counts[0] == 0 and counts[-1] == 300
    assert all(c1 <= c2 for c1, c2 in zip(counts, counts[1:]))


# ---------------------------------------------------------- eigensolver ----

def test_eigh_laplace_closed_form_vectors():
    """Eigenpairs of tridiag(-1,2,-1): v_k(j) = sqrt(2/(n+1)) sin(jk pi/(n+1))."""
    n = 128
    ab = sp_inputs.laplace(n)
    w, V = oracle.eigh_tridiag(ab)
    lam = laplace_eigs(n)
    assert np.max(np.abs(w - lam)) < 1e-13
    j = np.arange(1, n + 1)[:, None]
    k = np.arange(1, n + 1)[None, :]
    Vref = math.sqrt(2.0 / (n + 1)) * np.sin(j * k * math.pi / (n + 1))
    signs = np.sign(np.sum(V * Vref, axis=0))
    assert np.max(np.abs(V * signs - Vref)) < 1e-12


def test_eigh_dense_vs_jacobi_long_double():
    """Householder + implicit QR against cyclic Jacobi in long double (an
    independent algorithm) on random dense symmetric matrices, n <= 64."""
    rng = np.random.default_rng(7)
    for n in (1, 2, 5, 17, 64):
        M = rng.standard_normal((n, n))
        A = M + M.T
        w1, V1 = oracle.eigh(A)
        w2, V2 = oracle.jacobi_eigh_ld(A)
        assert np.max(np.abs(w1 - w2)) < 1e-12 * max(1.0, np.max(np.abs(w2)))
        # projectors onto the lower half agree (invariant to eigenvector signs)
        nu = n // 2
        if 0 < nu < n and w2[nu] - w2[nu - 1] > 1e-6:
            P1 = V1[:, :nu] @ V1[:, :nu].T
            P2 = V2[:, :nu] @ V2[:, :nu].T
            assert np.max(np.abs(P1 - P2)) < 1e-10


def test_eigh_dense_vs_lapack_and_residual():
    rng = np.random.default_rng(3)
    n = 300
    M = rng.standard_normal((n, n))
    A = 0.5 * (M + M.T)
    w, V = oracle.eigh(A)
    assert np.max(np.abs(w - np.linalg.eigvalsh(A))) < 1e-11
    assert np.max(np.abs(V.T @ V - np.eye(n))) < 1e-12
    assert np.max(np.abs(A @ V - V * w)) < 1e-11


def test_eigh_banded_path_matches_tridiagonal_path():
    """For a tridiagonal input the dense (Householder) path and the direct
    tridiagonal path give the same projector."""
    ab = sp_inputs.uniform_tridiag(150, seed=9)
    A = sp_inputs.dense_from_band(ab)
    P1, nu1, _ = oracle.projector_dense(A, 0.05)
    P2, nu2, _ = oracle.projector(ab, 0.05)
    assert nu1 == nu2 == oracle.sturm_count(ab, 0.05)
    assert np.max(np.abs(P1 - P2)) < 1e-9


# ------------------------------------------------------------ projector ----

def test_projector_laplace_closed_form_n1024():
    """Pi for tridiag(-1,2,-1), n = 1024, mu = 2 (nu = 512) against the
    Dirichlet-kernel closed form; Pi_jj = 1/2 and Pi_jl = 0 for even j-l != 0
    (A - 2I is bipartite, so sign(A - 2I) is odd)."""
    n = 1024
    ab = sp_inputs.laplace(n)
    P, nu, w = oracle.projector(ab, 2.0)
    assert nu == 512
    Pc = oracle.laplace_projector(n, nu)
    assert np.max(np.abs(P - Pc)) < 1e-11
    assert np.max(np.abs(np.diag(Pc) - 0.5)) < 1e-12
    d = np.subtract.outer(np.arange(n), np.arange(n))
    even_off = (d % 2 == 0) & (d != 0)
    assert np.max(np.abs(Pc[even_off])) < 1e-12


def test_projector_invariants_config0():
    """Workload 0 (n = 1024 uniform tridiagonal, nu = 512): trace Pi = nu,
    Pi^2 = Pi, A Pi = Pi A, Pi = Pi^T (to a small multiple of n u / gap)."""
    (name, ab, nu), = sp_inputs.workload(0)
    sh = oracle.locate_mu(ab, nu)
    P, nu2, w = oracle.projector(ab, sh.mu)
    assert nu2 == nu
    A = sp_inputs.dense_from_band(ab)
    assert abs(np.trace(P) - nu) < 1e-9
    assert np.max(np.abs(P @ P - P)) < 1e-11
    assert np.max(np.abs(A @ P - P @ A)) < 1e-11
    assert np.max(np.abs(P - P.T)) < 1e-14
    assert w[nu - 1] < sh.mu < w[nu]


# ------------------------------------------------------------ QDWH scalars -

@pytest.mark.parametrize("l", [0.9, 0.5, 0.1, 1e-3, 1e-6, 1e-10, 1e-15])
def test_dwh_weights_are_optimal(l):
    """The dynamic weights make f(x) = x(a + b x^2)/(1 + c x^2) map [l, 1]
    into [f(l), 1]: max f = 1 (attained at x = 1 and at an interior point),
    min f = f(l) = l_next (Sec. 2.1, recurrence for l_k)."""
    a, b, c, ln = oracle.qdwh_params(l)
    assert abs(c - (a + b - 1.0)) <= 1e-12 * c
    assert abs(b - 0.25 * (a - 1.0) ** 2) <= 1e-12 * b
    x = np.concatenate([np.geomspace(l, 1.0, 200001), np.linspace(l, 1.0, 200001)])
    f = x * (a + b * x * x) / (1.0 + c * x * x)
    assert f.max() <= 1.0 + 1e-12
    assert abs(f.min() - ln) <= 1e-12 * max(ln, 1e-300)
    interior = (x > 1.5 * l) & (x < 0.999)
    if interior.any() and l < 0.5:
        assert f[interior].max() > 1.0 - 1e-6


def test_dwh_residual_identity():
    """f(x) - x = (a - 1) x (1 - x^2) / (1 + c x^2), since b - c = 1 - a."""
    rng = np.random.default_rng(1)
    for l in (0.3, 1e-4):
        a, b, c, _ = oracle.qdwh_params(l)
        x = rng.uniform(l, 1.0, 1000)
        lhs = x * (a + b * x * x) / (1 + c * x * x) - x
        rhs = (a - 1.0) * x * (1.0 - x * x) / (1.0 + c * x * x)
        assert np.max(np.abs(lhs - rhs)) < 1e-9


@pytest.mark.parametrize("l0", [1e-1, 1e-4, 1e-6, 1e-10, 1e-16])
def test_schedule_at_most_six_iterations(l0):
    """At most 6 iterations for kappa <= 1e16 (Sec. 2.1); c_k decreases
    monotonically towards 3 (Sec. 2.2)."""
    sched = oracle.qdwh_schedule(l0, 1e-15)
    assert 1 <= len(sched) <= 6
    cs = [c for (_, _, _, c) in sched]
    assert all(c1 > c2 for c1, c2 in zip(cs, cs[1:]))
    assert cs[-1] > 3.0 - 1e-9 and cs[-1] < 3.5


# ------------------------------------------------------------ dense QDWH ---

def test_qdwh_dense_diagonal_is_scalar_map():
    """For a diagonal A every iterate is the scalar map applied entrywise; the
    limit is sign(A)."""
    lam = np.array([-1.0, -0.3, -1e-3, 2e-3, 0.5, 0.9])
    A = np.diag(lam)
    alpha = 1.0
    l0 = 1e-3
    res = oracle.qdwh_dense(A, alpha, l0, 1e-15, qr_policy=1)
    assert np.max(np.abs(res.U - np.diag(np.sign(lam)))) < 1e-14
    a, b, c, _ = oracle.qdwh_params(l0)
    x = lam / alpha
    f0 = x * (a + b * x * x) / (1 + c * x * x)
    assert np.max(np.abs(np.diag(res.X1) - f0)) < 1e-14
    assert np.max(np.abs(res.X1 - np.diag(np.diag(res.X1)))) < 1e-15


def test_qdwh_dense_eigenbasis_diagonal_and_projector():
    """In the eigenbasis of A the QDWH iterate is diagonal with the scalar map
    entries; (I - U)/2 matches Pi = V_nu V_nu^T."""
    (name, ab, nu), = sp_inputs.workload(0, n=200)
    sh = oracle.locate_mu(ab, nu)
    alpha, l0 = oracle.qdwh_start(sh)
    A = sp_inputs.dense_from_band(ab) - sh.mu * np.eye(200)
    res = oracle.qdwh_dense(A, alpha, l0, 1e-15, qr_policy=1)
    assert res.kind[0] == 1 and all(k == 2 for k in res.kind[1:])
    w, V = oracle.eigh(A)
    D = V.T @ res.X1 @ V
    a, b, c, _ = oracle.qdwh_params(l0)
    x = w / alpha
    assert np.max(np.abs(np.diag(D) - x * (a + b * x * x) / (1 + c * x * x))) < 1e-12
    assert np.max(np.abs(D - np.diag(np.diag(D)))) < 1e-12
    P, nu2, _ = oracle.projector(ab, sh.mu)
    e_id, e_tr, e_sp = oracle.error_measures(res.U, A, P, nu2)
    gap = min(abs(w[nu - 1]), abs(w[nu]))
    assert e_id < 1e-13 and e_tr < 1e-12
    assert e_sp < 1e-14 / gap + 1e-13


def test_qdwh_one_qr_vs_all_cholesky_agree_when_well_conditioned():
    """The QR-based and the Cholesky-based forms are the same recurrence
    (Eq. (reccur)); they agree when Z is well conditioned (|lambda| >= 0.2)."""
    n = 120
    rng = np.random.default_rng(12)
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = rng.uniform(0.2, 1.0, n) * np.where(np.arange(n) % 2 == 0, -1.0, 1.0)
    A = (Qm * lam) @ Qm.T
    A = 0.5 * (A + A.T)
    alpha, l0 = 1.0, 0.2
    r1 = oracle.qdwh_dense(A, alpha, l0, 1e-15, qr_policy=1)
    r0 = oracle.qdwh_dense(A, alpha, l0, 1e-15, qr_policy=0)
    assert r1.kind[0] == 1 and r0.kind[0] == 2
    assert np.max(np.abs(r1.X1 - r0.X1)) < 1e-13
    assert np.max(np.abs(r1.U - r0.U)) < 1e-13
    assert np.max(np.abs(r1.U - (Qm * np.sign(lam)) @ Qm.T)) < 1e-13


# ------------------------------------------------------------ fast QR ------

@pytest.mark.parametrize("n,b", [(2, 1), (7, 1), (40, 1), (6, 3), (33, 2), (50, 4), (64, 8)])
def test_fastqr_structure(n, b):
    """Algorithms 1/2: (2b+1)n - b^2 - b rotations; Q orthogonal; Q R equals
    [cA; I]; R upper triangular with upper bandwidth 2b; Q1 b-Hessenberg,
    Q2 upper triangular (Sec. 4.1-4.2)."""
    ab = sp_inputs.normal_band(n, b, seed=100 + n + b)
    c = 0.7
    fq = oracle.fastqr_replay(ab, c)
    assert len(fq.c) == oracle.fastqr_rotation_count(n, b)
    Q, R = fq.Q, fq.R
    assert np.max(np.abs(Q.T @ Q - np.eye(2 * n))) < 1e-13
    M = np.vstack([c * sp_inputs.dense_from_band(ab), np.eye(n)])
    assert np.max(np.abs(Q[:, :n] @ R[:n, :] - M)) < 1e-13
    assert np.max(np.abs(R[n:, :])) == 0.0
    assert np.max(np.abs(np.tril(R[:n, :], -1))) == 0.0
    assert np.max(np.abs(np.triu(R[:n, :], 2 * b + 1))) < 1e-300
    Q1, Q2 = Q[:n, :n], Q[n:, :n]
    assert np.max(np.abs(np.tril(Q1, -b - 1))) == 0.0
    assert np.max(np.abs(np.tril(Q2, -1))) == 0.0


def _numrank(M, tol=1e-12):
    if M.size == 0:
        return 0
    s = np.linalg.svd(M, compute_uv=False)
    return int(np.count_nonzero(s > tol * max(1.0, s[0])))


@pytest.mark.parametrize("n,b", [(60, 1), (48, 3)])
def test_fastqr_rank_theorems(n, b):
    """Theorems 4/6: Q(1:k, k+1:n) and Q(n+1:n+k, k+1:n) have rank <= 2b;
    Theorems 5/7: every off-diagonal block of Q1 Q2^T has rank <= 2b; for
    b = 1 the first iterate is HODLR with ranks <= 3 (Sec. 4.1)."""
    ab = sp_inputs.uniform_band(n, b, seed=2 * n + b)
    fq = oracle.fastqr_replay(ab, 1.3)
    Q = fq.Q
    Q1, Q2 = Q[:n, :n], Q[n:, :n]
    P = Q1 @ Q2.T
    A = sp_inputs.dense_from_band(ab)
    X1 = 0.4 * A + 0.9 * P
    for k in range(1, n):
        assert _numrank(Q[:k, k:n]) <= 2 * b
        assert _numrank(Q[n:n + k, k:n]) <= 2 * b
        assert _numrank(P[:k, k:]) <= 2 * b
        assert _numrank(P[k:, :k]) <= 2 * b
        if b == 1:
            assert _numrank(X1[:k, k:]) <= 3
            assert _numrank(X1[k:, :k]) <= 3


def test_fastqr_product_is_rational_function_and_matches_householder():
    """Q1 Q2^T = c A (I + c^2 A^2)^{-1} (from [cA; I] = Q R), and the QR-based
    first iterate built from the replayed rotations equals the dense QDWH's
    Householder-based X1 (the QR factor is unique up to column signs D and
    Q1 D D Q2^T = Q1 Q2^T)."""
    (name, ab, nu), = sp_inputs.workload(0, n=96)
    sh = oracle.locate_mu(ab, nu)
    alpha, l0 = oracle.qdwh_start(sh)
    n = 96
    ab_s = ab.copy()
    ab_s[:, 0] -= sh.mu
    a, b, c, _ = oracle.qdwh_params(l0)
    sc = math.sqrt(c)
    fq = oracle.fastqr_replay(ab_s, sc / alpha)
    Q1, Q2 = fq.Q[:n, :n], fq.Q[n:, :n]
    X0 = sp_inputs.dense_from_band(ab_s) / alpha
    P = Q1 @ Q2.T
    ref = sc * X0 @ np.linalg.inv(np.eye(n) + c * X0 @ X0)
    assert np.max(np.abs(P - ref)) < 1e-9
    X1 = (b / c) * X0 + (a - b / c) / sc * P
    res = oracle.qdwh_dense(X0 * alpha, alpha, l0, 1e-15, qr_policy=1)
    assert np.max(np.abs(X1 - res.X1)) < 1e-12


def test_dense_qdwh_accuracy_vs_gap_follows_paper():
    """Dense QDWH (one QR-based step) on the Sec. 6.1 tridiagonal matrices:
    the paper's table (tests/golden/dense_qdwh_one_qr_vs_gap.txt, n = 2000)
    shows e_trace and e_id at rounding level for every gap and e_SP growing
    like u/gap until the projector is lost at gap ~ u.  At n = 200: the same
    levels, e_SP within two orders of magnitude of the printed value where it
    is a rounding-level quantity, and the same growth."""
    import os
    rows = [list(map(float, ln.split())) for ln in
            open(os.path.join(os.path.dirname(__file__), "golden", "dense_qdwh_one_qr_vs_gap.txt"))
            if ln.strip() and not ln.startswith("#")]
    n = 200
    esp = []
    for gap, pt, pid, psp in rows:
        lam = sp_inputs.gap_spectrum(n, gap)
        ab = sp_inputs.prescribed_band(lam, 1)
        A = sp_inputs.dense_from_band(ab)
        res = oracle.qdwh_dense(A, 1.0, gap)
        Pref, nu, _ = oracle.projector(ab, 0.0)
        U = res.U
        e_tr = abs(np.trace(U) - (n - 2 * nu))
        e_id = oracle.sym_norm2(U @ U - np.eye(n))
        e_sp = oracle.sym_norm2(0.5 * (np.eye(n) - U) - Pref)
        assert e_tr <= 100 * max(pt, 1e-16) and e_id <= 100 * pid, (gap, e_tr, e_id)
        esp.append(e_sp)
        if gap >= 1e-5:
            assert psp / 100 <= e_sp <= psp * 100, (gap, e_sp, psp)
    assert esp[0] < esp[1] < esp[2] < esp[3]   # grows as the gap closes
    assert esp[2] <= 1e-5 and esp[3] >= 1e-5   # lost only when the gap reaches rounding level
