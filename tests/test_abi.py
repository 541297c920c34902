"""The C-ABI library builds for sm_103a, loads, and exports every entry
point that include/sp.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_1608_01164_gb300 as sp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "sp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sp_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    sp.build()
    return ctypes.CDLL(sp.LIB_PATH)


def test_header_declares_the_binding_exports():
    assert declared_symbols() == sorted(sp.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_signatures_bind(lib):
    sp.bind(lib)


def test_defaults_without_gpu(lib):
    sp.bind(lib)
    o = sp.sp_qdwh_opts()
    lib.sp_qdwh_opts_default(ctypes.byref(o))
    assert o.max_iter == 10 and o.delta == 1e-15 and o.qr_steps == 1 and o.precision == sp.SP_FP64


def test_invalid_arguments_rejected_without_gpu(lib):
    sp.bind(lib)
    h = ctypes.c_void_p()
    # null context -> SP_EINVAL before any device work
    assert lib.sp_hodlr_from_band(None, 10, 1, None, 2, 0.0, 4, 1e-10, 0, ctypes.byref(h)) == sp.SP_EINVAL
    assert lib.sp_qdwh_sign(None, None, None, None, None) == sp.SP_EINVAL
    # an allocator needs both callbacks
    alloc = sp.SP_ALLOC_FN(lambda nbytes, stream, user: 0)
    assert lib.sp_ctx_create(None, alloc, sp.SP_FREE_FN(), None, ctypes.byref(h)) == sp.SP_EINVAL
    assert lib.sp_ctx_create(None, sp.SP_ALLOC_FN(), sp.SP_FREE_FN(), None, None) == sp.SP_EINVAL


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback: without the built library, loading raises."""
    monkeypatch.setattr(sp, "LIB_PATH", str(tmp_path / "libsp.so"))
    monkeypatch.setattr(sp, "_lib", None)
    with pytest.raises(OSError, match="missing"):
        sp.load()
    with pytest.raises(OSError):
        sp.sp_ctx_create(0)
