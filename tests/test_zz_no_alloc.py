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


@pytest.mark.parametrize("n,b,nshift", [(2000, 1, 300), (900, 4, 257), (500, 8, 1000)])
def test_noalloc_matches_regular_inertia_twice(ctx, n, b, nshift):
    ab = sp_inputs.normal_band(n, b, seed=1234 + b)
    rng = np.random.default_rng(b)
    lo, hi = -3.0 * np.sqrt(b + 1), 3.0 * np.sqrt(b + 1)
    ab_d = torch.from_numpy(np.ascontiguousarray(ab)).cuda()
    for call in range(2):
        shifts = np.sort(rng.uniform(lo, hi, nshift))
        ref = np.zeros(nshift, dtype=np.int64)
        sp.sp_inertia(ctx, ab, shifts, ref)
        sh_d = torch.from_numpy(shifts).cuda()
        out_d = torch.full((nshift,), -1, dtype=torch.int64, device="cuda")
        sp.sp_inertia_noalloc(ctx, n, b, ab_d, b + 1, nshift, sh_d, out_d)
        torch.cuda.synchronize()
        assert np.array_equal(out_d.cpu().numpy(), ref), f"call {call}"


def test_noalloc_rejects_oversized_request(ctx):
    n, b = 100, 16
    nshift = sp.SP_NOALLOC_SCRATCH_DOUBLES // (b * b + b) + 1
    ab_d = torch.zeros((n, b + 1), dtype=torch.float64, device="cuda")
    sh_d = torch.zeros(nshift, dtype=torch.float64, device="cuda")
    out_d = torch.zeros(nshift, dtype=torch.int64, device="cuda")
    with pytest.raises(sp.SpError) as ei:
        sp.sp_inertia_noalloc(ctx, n, b, ab_d, b + 1, nshift, sh_d, out_d)
    assert ei.value.code == sp.SP_EINVAL
