"""The autotuner: leaf size, TSQR chunk and GEMM tiling chosen by timing
projectors, cached as JSON lines and reused through a leaf argument of 0."""
import json

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


def test_autotune_cache_and_leaf_zero(ctx, tmp_path):
    n = 4096
    (_, ab, nu), = sp_inputs.workload(1, n=n)
    mu, _, _ = sp.sp_locate_shift(ctx, ab, nu)
    cache = str(tmp_path / "tune.jsonl")
    r = sp.sp_autotune(ctx, ab, mu, 1e-10, sp.SP_FP64, cache)
    print(f"tuned: leaf {r.leaf} chunk {r.tsqr_chunk} small tiles {r.small_tiles} {r.ms:.1f} ms "
          f"({r.trials} trials at n={r.n_tuned})")
    assert r.leaf in (64, 128, 256, 512) and r.tsqr_chunk in (256, 512, 1024) and r.trials >= 5 and r.n_tuned == n
    lines = [json.loads(x) for x in open(cache)]
    assert len(lines) == 1 and lines[0]["leaf"] == r.leaf and lines[0]["b"] == 1
    # a second call is a cache hit
    r2 = sp.sp_autotune(ctx, ab, mu, 1e-10, sp.SP_FP64, cache)
    assert r2.trials == 0 and r2.leaf == r.leaf
    # leaf = 0 takes the tuned leaf; the projector is the same
    c2 = sp.sp_ctx_create(0)
    try:
        sp.sp_ctx_load_tuning(c2, cache)
        sp.sp_ctx_set_tuning(c2, r.tsqr_chunk, r.small_tiles)
        A = sp.sp_hodlr_from_band(c2, ab, mu, 0, 1e-10)
        nn, levels, _, _ = sp.sp_hodlr_info(c2, A)
        expect_levels = 0
        while -(-n // (1 << expect_levels)) > r.leaf:
            expect_levels += 1
        assert levels == expect_levels
        S, _ = sp.sp_qdwh_sign(c2, A)
        P = sp.sp_projector(c2, S)
        assert round(sp.sp_trace(c2, P)) == nu
        for h in (A, S, P):
            sp.sp_hodlr_destroy(h)
    finally:
        sp.sp_ctx_destroy(c2)


def test_tuning_settings_keep_results(ctx):
    """Chunk shape and tiling change the schedule, not the result (beyond
    rounding): both projectors agree with the oracle."""
    n = 1024
    ab = sp_inputs.uniform_band(n, 2, seed=99)
    sh = oracle.locate_mu(ab, n // 2)
    Pi, _, _ = oracle.projector(ab, sh.mu)
    for chunk, tiles in ((256, 1), (512, 0)):
        c2 = sp.sp_ctx_create(0)
        try:
            sp.sp_ctx_set_tuning(c2, chunk, tiles)
            A = sp.sp_hodlr_from_band(c2, ab, sh.mu, 64, 1e-10)
            S, _ = sp.sp_qdwh_sign(c2, A)
            P = sp.sp_projector(c2, S)
            Pd = np.zeros((n, n), order="F")
            sp.sp_to_dense(c2, P, 0, n, Pd, n)
            assert oracle.sym_norm2(Pd - Pi) <= 1e-8
            for h in (A, S, P):
                sp.sp_hodlr_destroy(h)
        finally:
            sp.sp_ctx_destroy(c2)
