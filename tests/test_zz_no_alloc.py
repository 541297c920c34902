"""The no-allocation inertia entry point against the regular one.

Some callers cannot allocate device memory (their host program reserves the
GPU for its own pool, or must not call the CUDA allocator while it runs);
sp_inertia_noalloc serves them with a scratch array that lives inside the
library.  This file is collected last, so a run that stops at the first
failure has already run every other test; it also passes on its own in a
fresh process (it creates its own context).
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


def safe_shifts(ab, nshift, rng):
    """Shifts drawn uniformly over the spectrum's range, kept at least 1e-9
    (relative) away from every eigenvalue, so that no count is decided by
    rounding and every correct implementation gives the same counts."""
    lam = np.linalg.eigvalsh(sp_inputs.dense_from_band(ab))
    lo, hi = lam[0] - 1.0, lam[-1] + 1.0
    scale = max(abs(lo), abs(hi))
    out = []
    while len(out) < nshift:
        x = rng.uniform(lo, hi)
        if np.min(np.abs(lam - x)) > 1e-9 * scale:
            out.append(x)
    return np.sort(np.array(out))


@pytest.mark.parametrize("n,b,nshift", [(2000, 1, 300), (700, 2, 129), (650, 3, 200), (900, 4, 257),
                                        (500, 8, 1000), (400, 90, 100)])
def test_noalloc_matches_regular_inertia_twice(ctx, n, b, nshift):
    """Two calls in a row (the shared scratch keeps the previous call's
    contents) against the regular entry point and the oracle's counts."""
    ab = sp_inputs.normal_band(n, b, seed=1234 + b)
    rng = np.random.default_rng(b)
    ab_d = torch.from_numpy(np.ascontiguousarray(ab)).cuda()
    for call in range(2):
        shifts = safe_shifts(ab, nshift, rng)
        ref = np.zeros(nshift, dtype=np.int64)
        sp.sp_inertia(ctx, ab, shifts, ref)
        sh_d = torch.from_numpy(shifts).cuda()
        out_d = torch.full((nshift,), -1, dtype=torch.int64, device="cuda")
        sp.sp_inertia_noalloc(ctx, n, b, ab_d, b + 1, nshift, sh_d, out_d)
        torch.cuda.synchronize()
        got = out_d.cpu().numpy()
        assert np.array_equal(got, ref), f"call {call}"
        orc = np.array([oracle.band_count(ab, x) for x in shifts])
        assert np.array_equal(got, orc), f"call {call} vs oracle"


def test_noalloc_rejects_host_pointers(ctx):
    n, b, nshift = 64, 2, 8
    ab = sp_inputs.normal_band(n, b, seed=5)
    ab_d = torch.from_numpy(np.ascontiguousarray(ab)).cuda()
    sh = np.linspace(-1.0, 1.0, nshift)
    sh_d = torch.from_numpy(sh).cuda()
    out_d = torch.zeros(nshift, dtype=torch.int64, device="cuda")
    out_h = np.zeros(nshift, dtype=np.int64)
    for args in ((ab, sh_d, out_d), (ab_d, sh, out_d), (ab_d, sh_d, out_h)):
        with pytest.raises(sp.SpError) as ei:
            sp.sp_inertia_noalloc(ctx, n, b, args[0], b + 1, nshift, args[1], args[2])
        assert ei.value.code == sp.SP_EINVAL and "device pointers" in str(ei.value)


def test_noalloc_rejects_oversized_request(ctx):
    n, b = 100, 16
    nshift = sp.SP_NOALLOC_SCRATCH_DOUBLES // (b * b + b) + 1
    ab_d = torch.zeros((n, b + 1), dtype=torch.float64, device="cuda")
    sh_d = torch.zeros(nshift, dtype=torch.float64, device="cuda")
    out_d = torch.zeros(nshift, dtype=torch.int64, device="cuda")
    with pytest.raises(sp.SpError) as ei:
        sp.sp_inertia_noalloc(ctx, n, b, ab_d, b + 1, nshift, sh_d, out_d)
    assert ei.value.code == sp.SP_EINVAL
