"""Failure detection, reproducibility and caller-supplied memory, through the C ABI.

Failures are made on the host side (a NaN in the input band, a rank capacity
too small for the truncated ranks, an indefinite matrix handed to the
H-Cholesky); no test faults, traps or hangs the GPU.  Each one checks the
status code, that the message names the failing stage, and that the context
stays usable for the next call.
"""
import ctypes

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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def projector_dense(ctx, ab, mu, leaf, tol=1e-10, rank_cap=0):
    n = ab.shape[0]
    A = sp.sp_hodlr_from_band(ctx, dev(ab), mu, leaf, tol, rank_cap)
    S = P = None
    try:
        S, info = sp.sp_qdwh_sign(ctx, A)
        P = sp.sp_projector(ctx, S)
        out = np.zeros((n, n), order="F")
        sp.sp_to_dense(ctx, P, 0, n, out, n)
        return out, sp.sp_trace(ctx, P), info
    finally:
        for h in (A, S, P):
            sp.sp_hodlr_destroy(h)


def small_case(n=512, b=1):
    ab = sp_inputs.uniform_band(n, b, seed=4711 + b)
    return ab, oracle.locate_mu(ab, n // 2).mu


def test_nan_in_band_is_reported_and_context_recovers(ctx):
    ab, mu = small_case()
    bad = ab.copy()
    bad[100, 0] = np.nan
    A = sp.sp_hodlr_from_band(ctx, dev(bad), mu, 64, 1e-10)
    try:
        with pytest.raises(sp.SpError) as ei:
            sp.sp_qdwh_sign(ctx, A)
        assert ei.value.code == sp.SP_ENONFINITE
        assert "non-finite" in str(ei.value)
    finally:
        sp.sp_hodlr_destroy(A)
    # band entries outside the matrix (lower band storage, i >= n) are ignored
    pad = ab.copy()
    pad[-1, 1] = np.inf
    P, tr, _ = projector_dense(ctx, pad, mu, 64)
    assert round(tr) == ab.shape[0] // 2
    Pref, _, _ = oracle.projector(ab, mu)
    assert oracle.sym_norm2(P - Pref) <= 1e-8


def test_rank_capacity_overflow_is_reported(ctx):
    ab, mu = small_case(1024, 1)
    with pytest.raises(sp.SpError) as ei:
        projector_dense(ctx, ab, mu, 64, rank_cap=2)
    assert ei.value.code == sp.SP_ERANK
    assert "rank capacity" in str(ei.value)
    P, tr, _ = projector_dense(ctx, ab, mu, 64)
    assert round(tr) == 512


def test_indefinite_cholesky_is_reported(ctx):
    """A - mu I with mu inside the spectrum is indefinite: the H-Cholesky meets
    a non-positive leaf pivot."""
    ab, mu = small_case(600, 2)
    A = sp.sp_hodlr_from_band(ctx, dev(ab), mu, 64, 1e-10)
    try:
        with pytest.raises(sp.SpError) as ei:
            sp.sp_hodlr_cholesky(ctx, A)
        assert ei.value.code == sp.SP_EBREAKDOWN
    finally:
        sp.sp_hodlr_destroy(A)
    # the same matrix shifted below its spectrum is SPD and factors
    lo, _ = oracle.gershgorin(ab)
    B = sp.sp_hodlr_from_band(ctx, dev(ab), lo - 1.0, 64, 1e-10)
    L = sp.sp_hodlr_cholesky(ctx, B)
    sp.sp_hodlr_destroy(L)
    sp.sp_hodlr_destroy(B)


@pytest.mark.parametrize("b", [1, 4])
def test_reruns_are_bitwise_identical(ctx, b):
    """No atomics in the arithmetic (split-k GEMMs sum their chunks in order,
    the trace sums in a fixed order): two runs give the same bits."""
    ab, mu = small_case(2048, b)
    P1, t1, _ = projector_dense(ctx, ab, mu, 128)
    P2, t2, _ = projector_dense(ctx, ab, mu, 128)
    assert t1 == t2
    assert np.array_equal(P1, P2)


class CountingAllocator:
    """Caller-side stream-ordered allocator on top of torch's caching
    allocator (a host program's own pool), counting live buffers."""

    def __init__(self):
        self.live = {}
        self.calls = 0
        self.alloc = sp.SP_ALLOC_FN(self._alloc)
        self.free = sp.SP_FREE_FN(self._free)

    def _alloc(self, nbytes, stream, user):
        self.calls += 1
        p = torch.cuda.caching_allocator_alloc(int(nbytes), device=torch.cuda.current_device(),
                                               stream=int(stream or 0))
        self.live[p] = nbytes
        return p

    def _free(self, ptr, nbytes, stream, user):
        assert self.live.pop(ptr) == nbytes
        torch.cuda.caching_allocator_delete(ptr)


def test_caller_allocator_serves_every_buffer(ctx):
    ab, mu = small_case(1024, 2)
    Pref, tref, _ = projector_dense(ctx, ab, mu, 64)
    al = CountingAllocator()
    stream = torch.cuda.current_stream().cuda_stream
    c2 = sp.sp_ctx_create(stream, al.alloc, al.free)
    try:
        P, tr, _ = projector_dense(c2, ab, mu, 64)
        assert tr == tref and np.array_equal(P, Pref)
        assert al.calls > 100
    finally:
        sp.sp_ctx_destroy(c2)
    torch.cuda.synchronize()
    assert not al.live, f"{len(al.live)} buffers not returned"


def test_ctx_create_rejects_half_an_allocator():
    al = CountingAllocator()
    h = ctypes.c_void_p()
    lib = sp.load()
    assert lib.sp_ctx_create(None, al.alloc, sp.SP_FREE_FN(), None, ctypes.byref(h)) == sp.SP_EINVAL


def test_level_ranks_and_nominal_bytes(ctx):
    ab, mu = small_case(2048, 1)
    A = sp.sp_hodlr_from_band(ctx, dev(ab), mu, 128, 1e-10)
    S, info = sp.sp_qdwh_sign(ctx, A)
    try:
        mx, mean, nb = sp.sp_hodlr_level_ranks(ctx, S, 32)
        assert info.levels == 4
        assert list(mx[:4]) == list(info.max_rank_level[:4]) and max(mx) == info.max_rank
        assert np.allclose(mean[:4], list(info.mean_rank_level[:4]))
        assert all(mx[4:] == 0) and all(mean[:4] > 0)
        # storage at the actual ranks is below what the rank capacity allocates
        assert 8 * 2048 * 128 < nb == info.nominal_bytes < info.bytes
    finally:
        sp.sp_hodlr_destroy(A)
        sp.sp_hodlr_destroy(S)
