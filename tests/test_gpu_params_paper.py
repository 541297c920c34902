"""The paper's start parameters (Sec. 5, Eq. (param_estimation)) on the GPU
against exact values and against the library's inertia brackets.

normest is a power method: its alpha never exceeds ||A - mu I||_2 and must
come within the method's tolerance of it.  The Hager-Higham 1-norm estimate
of (A - mu I)^{-1} is a lower bound of the exact 1-norm (computed here from
a dense inverse) and in practice within a small factor of it.  The resulting
l0 is compared with sigma_min(X0) (exact, from the oracle's eigenvalues): the
paper's formula is an estimate, which the test records, while the inertia
start is a guaranteed lower bound.
"""
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


def cases():
    yield "uniform tridiagonal n=1024", sp_inputs.uniform_tridiag(1024, 77), 512
    yield "N(0,1) band b=4 n=1024", sp_inputs.normal_band(1024, 4, 78), 512
    yield "prescribed gap 1e-4 b=2 n=512", sp_inputs.prescribed_band(sp_inputs.gap_spectrum(512, 1e-4), 2), 256


@pytest.mark.parametrize("name,ab,nu", list(cases()), ids=[c[0] for c in cases()])
def test_paper_parameters(ctx, name, ab, nu):
    n = ab.shape[0]
    sh = oracle.locate_mu(ab, nu)
    mu = sh.mu
    A = oracle.band_to_dense(ab, mu)
    lam = np.linalg.eigvalsh(A)
    norm2 = float(np.max(np.abs(lam)))
    smin = float(np.min(np.abs(lam)))
    inv1 = float(np.max(np.abs(np.linalg.inv(A)).sum(axis=0)))
    alpha, l0, pit, nsolve = sp.sp_qdwh_params_paper(ctx, ab, mu)
    est = 1.0 / (l0 * np.sqrt(n) * alpha)  # the estimate of ||(A - mu I)^{-1}||_1 inside l0
    a_in, l_in = sp.sp_qdwh_start(ctx, ab, mu)
    print(f"{name}: normest {alpha:.8f} vs ||A||_2 {norm2:.8f} ({pit} iterations); "
          f"1-norm est {est:.4e} vs exact {inv1:.4e} ({nsolve} solves); l0 paper {l0:.3e} vs sigma_min(X0) "
          f"{smin / alpha:.3e} (safe: {l0 <= smin / alpha}); inertia start alpha {a_in:.8f} l0 {l_in:.3e}")
    assert alpha <= norm2 * (1 + 1e-12)
    assert alpha >= norm2 * (1 - 1e-3)
    assert est <= inv1 * (1 + 1e-9)
    assert est >= 0.1 * inv1
    assert a_in >= norm2 and l_in <= smin / a_in
    # QDWH run from the paper's parameters: same projector when l0 is safe
    H = sp.sp_hodlr_from_band(ctx, ab, mu, 64, 1e-10)
    opts = sp.sp_qdwh_opts_default()
    opts.alpha, opts.l0 = alpha, l0
    S, info = sp.sp_qdwh_sign(ctx, H, opts)
    P = sp.sp_projector(ctx, S)
    try:
        Pd = np.zeros((n, n), order="F")
        sp.sp_to_dense(ctx, P, 0, n, Pd, n)
        Pi, nu_ref, _ = oracle.projector(ab, mu)
        err = oracle.sym_norm2(Pd - Pi)
        S2, info2 = sp.sp_qdwh_sign(ctx, H, None)
        sp.sp_hodlr_destroy(S2)
        print(f"   iterations: paper start {info.iters}, inertia start {info2.iters}; "
              f"||P - Pi||_2 from the paper start {err:.2e}")
        assert nu_ref == nu
        if l0 <= smin / alpha:
            assert err <= 1e-8, err
    finally:
        for h in (H, S, P):
            sp.sp_hodlr_destroy(h)
