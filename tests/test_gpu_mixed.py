"""Mixed precision: late Cholesky-based steps in residual form with binary32
GEMM arithmetic, then binary64 Newton-Schulz polish; errors against the
binary64 oracle before and after the polish."""
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


def projector(ctx, ab, mu, leaf, precision, polish):
    A = sp.sp_hodlr_from_band(ctx, ab, mu, leaf, 1e-10)
    o = sp.sp_qdwh_opts_default()
    o.precision = precision
    o.polish_steps = polish
    S, info = sp.sp_qdwh_sign(ctx, A, o)
    P = sp.sp_projector(ctx, S)
    n = ab.shape[0]
    Pd = dense(ctx, P, n)
    tr = sp.sp_trace(ctx, P)
    for h in (A, S, P):
        sp.sp_hodlr_destroy(h)
    return Pd, tr, info


@pytest.mark.parametrize("name,n,b,leaf", [("band16", 1024, 16, 64), ("tridiag", 1024, 1, 64)])
def test_mixed_precision_error_before_and_after_polish(ctx, name, n, b, leaf):
    if b == 16:
        ab = sp_inputs.normal_band(n, 16, seed=2024, scale=1.0 / math.sqrt(16.0))
    else:
        (_, ab, _), = sp_inputs.workload(0, n=n)
    nu = n // 2
    sh = oracle.locate_mu(ab, nu)
    Pref, _, _ = oracle.projector(ab, sh.mu)
    P64, tr64, i64 = projector(ctx, ab, sh.mu, leaf, sp.SP_FP64, 0)
    Pm0, trm0, im0 = projector(ctx, ab, sh.mu, leaf, sp.SP_MIXED_FP32, 0)
    Pm1, trm1, im1 = projector(ctx, ab, sh.mu, leaf, sp.SP_MIXED_FP32, 1)
    e64 = oracle.sym_norm2(P64 - Pref)
    e0 = oracle.sym_norm2(Pm0 - Pref)
    e1 = oracle.sym_norm2(Pm1 - Pref)
    kinds = list(im1.kind[:im1.iters])
    assert 3 in kinds and kinds[0] == 1, kinds          # at least one mixed step ran
    assert e64 <= 1e-8
    assert e1 <= 1e-8, (e0, e1)                         # the bar, after the polish
    assert e0 <= 1e-5                                   # before the polish: binary32-level at worst
    assert round(tr64) == nu and round(trm1) == nu
    print(f"{name}: FP64 {e64:.2e}  mixed before polish {e0:.2e}  after polish {e1:.2e}")


@pytest.mark.parametrize("name,n,b,leaf", [("band16", 1024, 16, 64), ("tridiag", 1024, 1, 64)])
def test_mixed_newton_schulz_tail(ctx, name, n, b, leaf):
    """Late QDWH steps replaced by residual-form Newton-Schulz steps (binary32
    products): same bar against the binary64 oracle."""
    if b == 16:
        ab = sp_inputs.normal_band(n, 16, seed=2024, scale=1.0 / math.sqrt(16.0))
    else:
        (_, ab, _), = sp_inputs.workload(0, n=n)
    nu = n // 2
    sh = oracle.locate_mu(ab, nu)
    Pref, _, _ = oracle.projector(ab, sh.mu)
    Pn, trn, inn = projector(ctx, ab, sh.mu, leaf, sp.SP_MIXED_NS, 1)
    kinds = list(inn.kind[:inn.iters])
    assert kinds[0] == 1 and 4 in kinds and 3 not in kinds, kinds
    # the tail starts where 1 - l_k^2 <= 1e-2; every step before it is a Cholesky step
    first_ns = kinds.index(4)
    assert all(k == 2 for k in kinds[1:first_ns])
    assert all(k == 4 for k in kinds[first_ns:])
    assert 1.0 - inn.l[first_ns] ** 2 <= 1e-2
    e = oracle.sym_norm2(Pn - Pref)
    assert e <= 1e-8, e
    assert round(trn) == nu
    print(f"{name}: mixed Newton-Schulz tail {kinds} error {e:.2e}")


def test_mixed_rejects_bad_precision(ctx):
    ab = sp_inputs.uniform_band(64, 1, 3)
    A = sp.sp_hodlr_from_band(ctx, ab, 0.0, 16, 1e-10)
    try:
        o = sp.sp_qdwh_opts_default()
        o.precision = 7
        with pytest.raises(sp.SpError) as ei:
            sp.sp_qdwh_sign(ctx, A, o)
        assert ei.value.code == sp.SP_EINVAL
    finally:
        sp.sp_hodlr_destroy(A)
