"""Projectors beyond the oracle's reach, checked by invariants that hold at any
size: trace = nu exactly after rounding (nu from an inertia count),
idempotence P(Pv) = Pv, commutation A(Pv) = P(Av) and symmetry
<u, Pv> = <Pu, v> on seeded probe vectors (Sec. 2: Pi is the orthogonal
projector onto the eigenvectors of the eigenvalues below mu)."""
import numpy as np
import pytest

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


def band_matvec(ab, X):
    """Y = A X for the symmetric band A in lower band storage (ab[i, d] = A[i+d, i])."""
    n, w = ab.shape
    Y = ab[:, 0:1] * X
    for d in range(1, w):
        e = ab[: n - d, d:d + 1]
        Y[d:] += e * X[: n - d]
        Y[: n - d] += e * X[d:]
    return Y


def check_invariants(ctx, ab, nu, leaf, precision=None, nprobe=6, tol=1e-8, trunc=1e-10):
    n = ab.shape[0]
    mu, _, _ = sp.sp_locate_shift(ctx, ab, nu)
    A = sp.sp_hodlr_from_band(ctx, ab, mu, leaf, trunc)
    opts = sp.sp_qdwh_opts_default()
    if precision is not None:
        opts.precision = precision
    S, info = sp.sp_qdwh_sign(ctx, A, opts)
    P = sp.sp_projector(ctx, S)
    try:
        tr = sp.sp_trace(ctx, P)
        assert round(tr) == nu and abs(tr - nu) < 1e-6, (tr, nu)
        V = np.asfortranarray(sp_inputs.normal(4242, n * nprobe).reshape(nprobe, n).T)
        PV = np.zeros_like(V, order="F")
        sp.sp_apply(ctx, P, nprobe, V, n, PV, n)
        PPV = np.zeros_like(V, order="F")
        sp.sp_apply(ctx, P, nprobe, np.asfortranarray(PV), n, PPV, n)
        nv = np.linalg.norm(V)
        idem = np.linalg.norm(PPV - PV) / nv
        Ashift = ab.copy()
        Ashift[:, 0] -= mu
        AV = np.asfortranarray(band_matvec(Ashift, V))
        PAV = np.zeros_like(V, order="F")
        sp.sp_apply(ctx, P, nprobe, AV, n, PAV, n)
        APV = band_matvec(Ashift, PV)
        anorm = np.max(np.abs(Ashift).sum(axis=1)) * 2
        comm = np.linalg.norm(APV - PAV) / (anorm * nv)
        G = V.T @ PV
        sym = np.linalg.norm(G - G.T) / nv ** 2
        print(f"n={n}: trace - nu {tr - nu:.1e}, idempotence {idem:.1e}, commutation {comm:.1e}, symmetry {sym:.1e}")
        assert idem <= tol, idem
        assert comm <= tol, comm
        assert sym <= 1e-10, sym
        return info, idem, comm
    finally:
        for h in (A, S, P):
            sp.sp_hodlr_destroy(h)


def test_anderson_16384(ctx):
    (_, ab, nu), = sp_inputs.workload(1, n=16384)
    info, idem, comm = check_invariants(ctx, ab, nu, 128)
    print(f"Anderson n=16384: iters {info.iters} max rank {info.max_rank} idem {idem:.1e} comm {comm:.1e}")


def test_band8_16384(ctx):
    (_, ab, nu), = sp_inputs.workload(1, variant="band8", n=16384)
    info, idem, comm = check_invariants(ctx, ab, nu, 128)
    print(f"b=8 n=16384: iters {info.iters} max rank {info.max_rank} idem {idem:.1e} comm {comm:.1e}")


@pytest.mark.parametrize("trunc", [1e-10, 1e-12])
@pytest.mark.parametrize("precision", ["fp64", "mixed_ns"])
def test_tridiagonal_1e5(ctx, precision, trunc):
    """Paper-scale workload: n = 1e5, relative gap ~1e-6 (localised Anderson
    eigenvectors), at the workload's truncation tolerance 1e-10 and at 1e-12:
    the 1e-8 bar on every invariant."""
    (_, ab, nu), = sp_inputs.workload(4, n=100000)
    prec = sp.SP_FP64 if precision == "fp64" else sp.SP_MIXED_NS
    info, idem, comm = check_invariants(ctx, ab, nu, 256, prec, tol=1e-8, trunc=trunc)
    print(f"tridiagonal n=1e5 tol {trunc:g} {precision}: iters {info.iters} max rank {info.max_rank} "
          f"idem {idem:.1e} comm {comm:.1e}")


def test_band4_1e5(ctx):
    """Paper-scale banded workload: b = 4, N(0,1) entries, n = 1e5, nu = n/2,
    truncation tolerance 1e-10."""
    (_, ab, nu), = sp_inputs.workload(4, variant="band4", n=100000)
    info, idem, comm = check_invariants(ctx, ab, nu, 256, tol=1e-8, trunc=1e-10)
    print(f"b=4 n=1e5 tol 1e-10: iters {info.iters} max rank {info.max_rank} idem {idem:.1e} comm {comm:.1e}")


def test_band16_32768(ctx):
    """Mixed-precision workload's matrix in binary64: b = 16, N(0,1)/4, n = 32768."""
    ab = sp_inputs.normal_band(32768, 16, sp_inputs.workload_seed(2, 0), 0.25)
    info, idem, comm = check_invariants(ctx, ab, 16384, 128, tol=1e-8)
    print(f"b=16 n=32768: iters {info.iters} max rank {info.max_rank} idem {idem:.1e} comm {comm:.1e}")


def projector(ctx, ab, nu, leaf, trunc, precision):
    mu, _, _ = sp.sp_locate_shift(ctx, ab, nu)
    A = sp.sp_hodlr_from_band(ctx, ab, mu, leaf, trunc)
    opts = sp.sp_qdwh_opts_default()
    opts.precision = precision
    S, info = sp.sp_qdwh_sign(ctx, A, opts)
    P = sp.sp_projector(ctx, S)
    sp.sp_hodlr_destroy(A)
    sp.sp_hodlr_destroy(S)
    return P, info


def diff_norm2(ctx, P1, P2, n, steps=30, s=4, seed=99):
    """||P1 - P2||_2 by block power iteration on the symmetric difference
    (a lower bound that converges to the norm), through sp_apply."""
    X = np.asfortranarray(sp_inputs.normal(seed, n * s).reshape(s, n).T)
    est = 0.0
    for _ in range(steps):
        X, _ = np.linalg.qr(X)
        X = np.asfortranarray(X)
        Y1 = np.zeros_like(X, order="F")
        Y2 = np.zeros_like(X, order="F")
        sp.sp_apply(ctx, P1, s, X, n, Y1, n)
        sp.sp_apply(ctx, P2, s, X, n, Y2, n)
        X = Y1 - Y2
        est = max(est, float(np.max(np.linalg.norm(X, axis=0))))
    return est


@pytest.mark.parametrize("workload", ["tridiag", "band4"])
def test_mixed_vs_fp64_1e5(ctx, workload):
    """The mixed-precision forms against the binary64 form at n = 1e5:
    ||P_mixed - P_fp64||_2 <= 1e-8 (power iteration on the difference)."""
    (_, ab, nu), = sp_inputs.workload(4, variant="main" if workload == "tridiag" else "band4", n=100000)
    n = ab.shape[0]
    P64, _ = projector(ctx, ab, nu, 256, 1e-10, sp.SP_FP64)
    try:
        for prec in (sp.SP_MIXED_FP32, sp.SP_MIXED_NS):
            Pm, info = projector(ctx, ab, nu, 256, 1e-10, prec)
            try:
                d = diff_norm2(ctx, Pm, P64, n)
                print(f"{workload} n=1e5 precision {prec}: ||P_mixed - P_fp64||_2 ~ {d:.2e} ({info.iters} iters)")
                assert d <= 1e-8, d
            finally:
                sp.sp_hodlr_destroy(Pm)
    finally:
        sp.sp_hodlr_destroy(P64)


@pytest.mark.parametrize("n,leaf", [(98304, 256), (100000, 256)])
def test_qr_step_commutes_localised(ctx, n, leaf):
    """The QR-based first step alone (Eq. (qdwh_qr)) gives X1 = f(X0), a
    function of A: it must commute with A to rounding.  On the localised
    Anderson matrices at this size the nested-basis factors of Q2 are badly
    scaled; without rebalancing them the formatted product Q1 Q2^T lost its
    upper blocks (commutation 4e-5 at n = 98304)."""
    (_, ab, nu), = sp_inputs.workload(4, n=n)
    mu, _, _ = sp.sp_locate_shift(ctx, ab, nu)
    A = sp.sp_hodlr_from_band(ctx, ab, mu, leaf, 1e-12)
    opts = sp.sp_qdwh_opts_default()
    opts.delta = 0.999  # the scalar schedule stops after the first (QR-based) step
    S, info = sp.sp_qdwh_sign(ctx, A, opts)
    try:
        assert info.iters == 1 and info.kind[0] == 1
        V = np.asfortranarray(sp_inputs.normal(77, n * 4).reshape(4, n).T)
        SV = np.zeros_like(V, order="F")
        sp.sp_apply(ctx, S, 4, V, n, SV, n)
        Ash = ab.copy()
        Ash[:, 0] -= mu
        AV = np.asfortranarray(band_matvec(Ash, V))
        SAV = np.zeros_like(V, order="F")
        sp.sp_apply(ctx, S, 4, AV, n, SAV, n)
        comm = np.linalg.norm(band_matvec(Ash, SV) - SAV) / (np.max(np.abs(Ash).sum(axis=1)) * np.linalg.norm(V))
        print(f"n={n} leaf {leaf}: X1 commutation {comm:.1e}")
        assert comm <= 1e-13, comm
    finally:
        sp.sp_hodlr_destroy(A)
        sp.sp_hodlr_destroy(S)
