"""Batched projectors (many independent banded instances of uneven n, b and
mu) against the oracle, instance by instance."""
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


def batch_instances(count, seed0):
    """Small instances of the batched workload's recipe: n log-uniform, b in
    {1,2,4,8}, U[-1,1] entries, nu in {n/3, n/2}."""
    out = []
    for t in range(count):
        s = seed0 + t
        u = sp_inputs.uniform01(s, 3)
        n = int(np.exp(np.log(96) + u[0] * (np.log(700) - np.log(96))))
        b = (1, 2, 4, 8)[min(int(u[1] * 4), 3)]
        nu = n // 3 if u[2] < 0.5 else n // 2
        out.append((sp_inputs.uniform_band(n, b, s), nu))
    return out


@pytest.mark.parametrize("device_bands", [False, True])
def test_batched_projectors_vs_oracle(ctx, device_bands):
    inst = batch_instances(10, 777 + int(device_bands))
    shifts = [oracle.locate_mu(ab, nu) for ab, nu in inst]
    bands = [torch.from_numpy(np.ascontiguousarray(ab)).cuda() if device_bands else np.ascontiguousarray(ab)
             for ab, _ in inst]
    Ps, infos = sp.sp_batched_projector(ctx, bands, [s.mu for s in shifts], leaf=0, tol=1e-10, nstreams=4)
    try:
        for (ab, nu), sh, P, info in zip(inst, shifts, Ps, infos):
            n = ab.shape[0]
            Pref, nu_ref, _ = oracle.projector(ab, sh.mu)
            assert nu_ref == nu
            assert oracle.sym_norm2(dense(ctx, P, n) - Pref) <= 1e-8
            assert round(sp.sp_trace(ctx, P)) == nu
            assert 1 <= info.iters <= 6
    finally:
        for P in Ps:
            sp.sp_hodlr_destroy(P)


def test_batched_matches_single(ctx):
    """A batch computes what the single-instance calls compute, bit for bit
    (same kernels, same fixed-order reductions within an instance)."""
    inst = batch_instances(4, 901)
    shifts = [oracle.locate_mu(ab, nu) for ab, nu in inst]
    Ps, _ = sp.sp_batched_projector(ctx, [np.ascontiguousarray(ab) for ab, _ in inst], [s.mu for s in shifts],
                                    leaf=64, tol=1e-10, nstreams=3)
    try:
        for (ab, nu), sh, P in zip(inst, shifts, Ps):
            n = ab.shape[0]
            A = sp.sp_hodlr_from_band(ctx, ab, sh.mu, 64, 1e-10)
            S, _ = sp.sp_qdwh_sign(ctx, A)
            P1 = sp.sp_projector(ctx, S)
            assert np.array_equal(dense(ctx, P, n), dense(ctx, P1, n))
            for h in (A, S, P1):
                sp.sp_hodlr_destroy(h)
    finally:
        for P in Ps:
            sp.sp_hodlr_destroy(P)


def test_batched_rejects_bad_instance(ctx):
    ab = sp_inputs.uniform_band(50, 2, 5)
    with pytest.raises(sp.SpError) as ei:
        sp.sp_batched_projector(ctx, [ab, ab], [0.0, 0.0], leaf=3)  # leaf < 2b
    assert ei.value.code == sp.SP_EINVAL


def test_batched_concurrent_kernel_limits(ctx):
    """Instances whose leaves (110..128 rows) need different amounts of dynamic
    shared memory above the 48 KB default, run on concurrent streams: the
    per-kernel limit must only ever be raised, never lowered under another
    stream's launch."""
    sizes = [7200, 8000, 7600, 7000, 7800, 7400]
    inst = [(sp_inputs.uniform_band(n, 1, 3100 + i), n // 2) for i, n in enumerate(sizes)]
    mus = [sp.sp_locate_shift(ctx, ab, nu)[0] for ab, nu in inst]
    Ps, infos = sp.sp_batched_projector(ctx, [np.ascontiguousarray(ab) for ab, _ in inst], mus, leaf=128,
                                        tol=1e-10, nstreams=6)
    try:
        for (ab, nu), P in zip(inst, Ps):
            assert round(sp.sp_trace(ctx, P)) == nu
    finally:
        for P in Ps:
            sp.sp_hodlr_destroy(P)


def test_batched_profile_reaches_the_callers_context(ctx):
    """The worker contexts' launch times, counts and flop counters are folded
    into the caller's context, so a profiled batch reports its kernels."""
    inst = batch_instances(3, 911)
    shifts = [oracle.locate_mu(ab, nu) for ab, nu in inst]
    sp.sp_ctx_set_profiling(ctx, True)
    try:
        Ps, _ = sp.sp_batched_projector(ctx, [np.ascontiguousarray(ab) for ab, _ in inst], [s.mu for s in shifts],
                                        leaf=64, tol=1e-10, nstreams=2)
        for P in Ps:
            sp.sp_hodlr_destroy(P)
        prof = sp.sp_ctx_profile(ctx)
    finally:
        sp.sp_ctx_set_profiling(ctx, False)
    la, ms, fl = prof["k_qr"]
    assert la > 0 and ms > 0.0 and fl > 0.0
    gemm = [v for k, v in prof.items() if k.startswith("k_gemm")]
    assert sum(v[0] for v in gemm) > 0 and sum(v[2] for v in gemm) > 0.0
