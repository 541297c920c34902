"""GPU parity tests: the CUDA path through the C ABI against the CPU oracle.

Tolerances: the projector's bar is ||Pi - Pi_oracle||_2 <= 1e-8 with the
trace equal to nu after rounding; exact operations (band ingest, structural
zeros) are compared bit for bit; formatted HODLR arithmetic against dense
binary64 products at a tolerance tied to the truncation tolerance.
"""
import math

import numpy as np
import pytest

import oracle
import sp_inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1608_01164_gb300 as sp  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sp.load()
    c = sp.sp_ctx_create(0)
    yield c
    sp.sp_ctx_destroy(c)


def dense(ctx, M, n):
    out = np.zeros((n, n), order="F")
    sp.sp_to_dense(ctx, M, 0, n, out, n)
    return out


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


class Handles:
    def __init__(self):
        self.h = []

    def __call__(self, x):
        self.h.append(x)
        return x

    def free(self):
        for x in self.h:
            sp.sp_hodlr_destroy(x)


@pytest.fixture
def keep():
    k = Handles()
    yield k
    k.free()


# ----------------------------------------------------------- band ingest ---

@pytest.mark.parametrize("n,b,leaf", [(1, 1, 2), (7, 1, 8), (37, 2, 8), (300, 1, 16), (513, 4, 32), (1000, 8, 64),
                                      (257, 16, 32)])
def test_band_roundtrip_exact(ctx, keep, n, b, leaf):
    """HODLR of a band is exact (Lemma 2: off-diagonal rank <= b)."""
    ab = sp_inputs.normal_band(n, b, seed=n + b)
    A = keep(sp.sp_hodlr_from_band(ctx, dev(ab), 0.37, leaf, 1e-10))
    D = dense(ctx, A, n)
    ref = sp_inputs.dense_from_band(ab) - 0.37 * np.eye(n)
    assert np.array_equal(D, ref)
    nn, levels, rmax, _ = sp.sp_hodlr_info(ctx, A)
    assert nn == n and (levels == 0 or rmax == b)


@pytest.mark.parametrize("n,b,leaf", [(513, 3, 32), (1000, 1, 64)])
def test_apply_and_trace(ctx, keep, n, b, leaf):
    ab = sp_inputs.normal_band(n, b, seed=5)
    A = keep(sp.sp_hodlr_from_band(ctx, dev(ab), 0.0, leaf, 1e-10))
    X = np.random.default_rng(0).standard_normal((n, 7))
    Xd = torch.from_numpy(np.asfortranarray(X).T.copy()).cuda()  # column-major (n x 7): memory of X^T row-major
    Yd = torch.zeros_like(Xd)
    sp.sp_apply(ctx, A, 7, Xd, n, Yd, n)
    torch.cuda.synchronize()
    Y = Yd.cpu().numpy().T
    Ad = sp_inputs.dense_from_band(ab)
    assert np.max(np.abs(Y - Ad @ X)) < 1e-12 * np.max(np.abs(Ad @ X))
    assert abs(sp.sp_trace(ctx, A) - np.trace(Ad)) < 1e-11


# ---------------------------------------------------- formatted arithmetic --

@pytest.mark.parametrize("n,b,leaf", [(400, 2, 32), (777, 5, 64)])
def test_add_mult_exact_ranks(ctx, keep, n, b, leaf):
    """Sums and products of banded matrices are banded (bandwidth 2b): the
    formatted results are exact up to rounding."""
    ab = sp_inputs.normal_band(n, b, seed=11)
    ab2 = sp_inputs.uniform_band(n, b, seed=12)
    A = keep(sp.sp_hodlr_from_band(ctx, dev(ab), 0.1, leaf, 1e-12))
    B = keep(sp.sp_hodlr_from_band(ctx, dev(ab2), -0.2, leaf, 1e-12))
    Ad = sp_inputs.dense_from_band(ab) - 0.1 * np.eye(n)
    Bd = sp_inputs.dense_from_band(ab2) + 0.2 * np.eye(n)
    C = keep(sp.sp_hodlr_add(ctx, 2.0, A, -3.0, B, 0.5))
    assert np.max(np.abs(dense(ctx, C, n) - (2 * Ad - 3 * Bd + 0.5 * np.eye(n)))) < 1e-12
    M = keep(sp.sp_hodlr_mult(ctx, A, B))
    ref = Ad @ Bd
    assert np.max(np.abs(dense(ctx, M, n) - ref)) < 1e-12 * np.max(np.abs(ref))
    assert sp.sp_hodlr_info(ctx, M)[2] <= 2 * b


@pytest.mark.parametrize("n,b,leaf", [(500, 2, 32), (1024, 1, 64)])
def test_cholesky_and_solves(ctx, keep, n, b, leaf):
    """H-Cholesky of Z = I + c A^2 (SPD) and the two formatted triangular
    solves L^{-1} X and L^{-T} L^{-1} X = Z^{-1} X used by the Cholesky-based
    QDWH step (Eq. (qdwh_chol_reccur))."""
    ab = sp_inputs.normal_band(n, b, seed=21)
    A = keep(sp.sp_hodlr_from_band(ctx, dev(ab), 0.0, leaf, 1e-12))
    Ad = sp_inputs.dense_from_band(ab)
    c = 0.37
    AA = keep(sp.sp_hodlr_mult(ctx, A, A))
    Z = keep(sp.sp_hodlr_add(ctx, c, AA, 0.0, None, 1.0))
    Zd = c * Ad @ Ad + np.eye(n)
    L = keep(sp.sp_hodlr_cholesky(ctx, Z))
    Ld = dense(ctx, L, n)
    assert np.max(np.abs(np.triu(Ld, 1))) == 0.0
    assert np.max(np.abs(Ld - np.linalg.cholesky(Zd))) < 1e-10
    Y = keep(sp.sp_hodlr_trsm(ctx, L, 0, A))
    assert np.max(np.abs(dense(ctx, Y, n) - np.linalg.solve(np.linalg.cholesky(Zd), Ad))) < 1e-9
    V = keep(sp.sp_hodlr_trsm(ctx, L, 1, Y))
    assert np.max(np.abs(dense(ctx, V, n) - np.linalg.solve(Zd, Ad))) < 1e-9


# ------------------------------------------------------- QR-based step -----

@pytest.mark.parametrize("n,b", [(2, 1), (50, 1), (301, 1), (200, 3), (257, 8), (130, 16)])
def test_givens_match_replay(ctx, n, b):
    """Algorithm 1/2 rotations, in order, against the oracle's dense replay."""
    ab = sp_inputs.normal_band(n, b, seed=31 + b)
    cnt = oracle.fastqr_rotation_count(n, b)
    cs = torch.zeros(2 * cnt, dtype=torch.float64, device="cuda")
    sp.sp_givens_generate(ctx, n, b, dev(ab), b + 1, 0.83, cs)
    torch.cuda.synchronize()
    h = cs.cpu().numpy()
    fq = oracle.fastqr_replay(ab, 0.83, want_q=False)
    assert len(fq.c) == cnt
    assert np.max(np.abs(h[0::2] - fq.c)) < 1e-12
    assert np.max(np.abs(h[1::2] - fq.s)) < 1e-12


@pytest.mark.parametrize("n,b,leaf", [(64, 1, 8), (300, 1, 32), (301, 3, 32), (256, 8, 32)])
def test_fastqr_factors_match_replay(ctx, keep, n, b, leaf):
    """Q1 and Q2 built directly in HODLR format (Remark construct_off,
    Theorems 4/6) against the dense replay's orthogonal factor."""
    ab = sp_inputs.uniform_band(n, b, seed=41 + n)
    A = keep(sp.sp_hodlr_from_band(ctx, dev(ab), 0.2, leaf, 1e-12))
    q1, q2 = sp.sp_fastqr_factors(ctx, A, 1.7)
    keep(q1)
    keep(q2)
    ab_s = ab.copy()
    ab_s[:, 0] -= 0.2
    fq = oracle.fastqr_replay(ab_s, 1.7)
    assert np.max(np.abs(dense(ctx, q1, n) - fq.Q[:n, :n])) < 1e-12
    assert np.max(np.abs(dense(ctx, q2, n) - fq.Q[n:, :n])) < 1e-12


# ------------------------------------------------- parameter estimation ----

@pytest.mark.parametrize("n,b", [(500, 1), (400, 4), (700, 16), (300, 33), (200, 90)])
def test_inertia_counts(ctx, n, b):
    ab = sp_inputs.normal_band(n, b, seed=51)
    w = np.linalg.eigvalsh(sp_inputs.dense_from_band(ab))
    shifts = np.concatenate([[w[0] - 1, w[-1] + 1], 0.5 * (w[1:] + w[:-1])[::7]])
    counts = np.zeros(len(shifts), dtype=np.int64)
    sp.sp_inertia(ctx, ab, shifts, counts)
    ref = np.array([oracle.band_count(ab, s) for s in shifts])
    assert np.array_equal(counts, ref)


@pytest.mark.parametrize("n,b,nu", [(1024, 1, 512), (600, 4, 200)])
def test_locate_shift_and_start(ctx, n, b, nu):
    ab = sp_inputs.normal_band(n, b, seed=61)
    mu, lam_nu_hi, lam_nu1_lo = sp.sp_locate_shift(ctx, ab, nu)
    w = np.linalg.eigvalsh(sp_inputs.dense_from_band(ab))
    assert w[nu - 1] < mu < w[nu]
    slack = 1e-13  # brackets converge to a few ulps; LAPACK's eigenvalues are rounded too
    assert w[nu - 1] - slack < lam_nu_hi <= mu <= lam_nu1_lo <= w[nu] + slack
    alpha, l0 = sp.sp_qdwh_start(ctx, ab, mu)
    assert alpha >= np.max(np.abs(w - mu)) and alpha <= 1.01 * np.max(np.abs(w - mu))
    smin = np.min(np.abs(w - mu)) / alpha
    assert 0.9 * smin <= l0 <= smin


# --------------------------------------------------------- the projector ---

def run_projector(ctx, keep, ab, mu, leaf, tol, opts=None):
    A = keep(sp.sp_hodlr_from_band(ctx, dev(ab), mu, leaf, tol))
    S, info = sp.sp_qdwh_sign(ctx, A, opts)
    keep(S)
    P = keep(sp.sp_projector(ctx, S))
    return A, S, P, info


def test_projector_workload0_vs_oracle(ctx, keep):
    """Workload 0: n = 1024 tridiagonal with U[-1,1] entries, nu = 512,
    leaf 64, tol 1e-10: ||Pi - Pi_oracle||_2 <= 1e-8 and trace = nu."""
    (name, ab, nu), = sp_inputs.workload(0)
    n = ab.shape[0]
    sh = oracle.locate_mu(ab, nu)
    A, S, P, info = run_projector(ctx, keep, ab, sh.mu, 64, 1e-10)
    Pd = dense(ctx, P, n)
    Pref, nu_ref, w = oracle.projector(ab, sh.mu)
    err = oracle.sym_norm2(Pd - Pref)
    tr = sp.sp_trace(ctx, P)
    assert nu_ref == nu and round(tr) == nu
    assert err <= 1e-8, err
    assert info.iters <= 6 and info.kind[0] == 1 and all(k == 2 for k in info.kind[1:info.iters])


def test_projector_laplace_closed_form(ctx, keep):
    """tridiag(-1,2,-1), n = 1024, mu = 2 against the closed-form projector."""
    n = 1024
    ab = sp_inputs.laplace(n)
    A, S, P, info = run_projector(ctx, keep, ab, 2.0, 64, 1e-10)
    Pd = dense(ctx, P, n)
    Pc = oracle.laplace_projector(n, n // 2)
    assert oracle.sym_norm2(Pd - Pc) <= 1e-8
    assert round(sp.sp_trace(ctx, P)) == n // 2


@pytest.mark.parametrize("n,b,nu,leaf", [(700, 4, 233, 32), (512, 8, 256, 64), (333, 2, 111, 16)])
def test_projector_banded_vs_oracle(ctx, keep, n, b, nu, leaf):
    ab = sp_inputs.normal_band(n, b, seed=71 + b, scale=1.0 / math.sqrt(b))
    sh = oracle.locate_mu(ab, nu)
    A, S, P, info = run_projector(ctx, keep, ab, sh.mu, leaf, 1e-10)
    Pd = dense(ctx, P, n)
    Pref, nu_ref, _ = oracle.projector(ab, sh.mu)
    assert oracle.sym_norm2(Pd - Pref) <= 1e-8
    assert round(sp.sp_trace(ctx, P)) == nu


def test_first_iterate_matches_dense_qdwh(ctx, keep):
    """X_1 of the QR-based step against the oracle's Householder-based X_1,
    with the same alpha and l0 (Eq. (qdwh_qr_reccur))."""
    (name, ab, nu), = sp_inputs.workload(0, n=300)
    n = 300
    sh = oracle.locate_mu(ab, nu)
    alpha, l0 = oracle.qdwh_start(sh)
    o = sp.sp_qdwh_opts_default()
    o.alpha, o.l0, o.max_iter = alpha, l0, 1
    A = keep(sp.sp_hodlr_from_band(ctx, dev(ab), sh.mu, 32, 1e-13))
    with pytest.raises(sp.SpError):
        sp.sp_qdwh_sign(ctx, A, o)  # max_iter = 1 is below the schedule's length
    o.max_iter = 10
    S, info = sp.sp_qdwh_sign(ctx, A, o)
    keep(S)
    res = oracle.qdwh_dense(sp_inputs.dense_from_band(ab) - sh.mu * np.eye(n), alpha, l0)
    assert info.iters == res.iters
    assert np.allclose(info.c[:info.iters], res.c, rtol=1e-14, atol=0)
    assert np.max(np.abs(dense(ctx, S, n) - res.U)) < 1e-10


@pytest.mark.parametrize("nu", [0, 64])
def test_projector_degenerate_spectrum_ends(ctx, keep, nu):
    """mu below the spectrum (nu = 0: P = 0) and above it (nu = n: P = I)."""
    n = 64
    ab = sp_inputs.uniform_tridiag(n, seed=81)
    sh = oracle.locate_mu(ab, nu)
    A, S, P, info = run_projector(ctx, keep, ab, sh.mu, 16, 1e-10)
    Pd = dense(ctx, P, n)
    ref = np.zeros((n, n)) if nu == 0 else np.eye(n)
    assert np.max(np.abs(Pd - ref)) < 1e-10


def test_single_leaf(ctx, keep):
    """n <= leaf: the HODLR is one dense leaf (L = 0)."""
    n = 40
    ab = sp_inputs.normal_band(n, 2, seed=91)
    sh = oracle.locate_mu(ab, 20)
    A, S, P, info = run_projector(ctx, keep, ab, sh.mu, 64, 1e-10)
    Pref, _, _ = oracle.projector(ab, sh.mu)
    assert oracle.sym_norm2(dense(ctx, P, n) - Pref) <= 1e-8
