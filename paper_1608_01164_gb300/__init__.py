"""Thin Python binding of the sm_103a spectral-projector library (libsp.so).

Argument marshalling only: every function forwards to the C ABI declared in
``include/sp.h`` with the same name; all computation runs in the library's
CUDA kernels.  Buffers may be numpy arrays (host memory) or torch tensors
(device memory, via ``data_ptr()``), as each C entry point allows.

The library is built in-tree by ``build()`` (nvcc, sm_103a) and loaded from
this package directory; if it is missing, loading raises -- there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

_HERE = os.path.dirname(os.path.abspath(__file__))
_CSRC = os.path.join(_HERE, "csrc")
_INCLUDE = os.path.join(os.path.dirname(_HERE), "include")
LIB_PATH = os.path.join(_HERE, "libsp.so")
SOURCES = ["sp_blas.cu", "sp_tc.cu", "sp_lowrank.cu", "sp_hodlr.cu", "sp_qrstep.cu", "sp_param.cu", "sp_api.cu",
           "sp_tune.cu"]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC"]

SP_OK, SP_EINVAL, SP_ENOMEM, SP_ECUDA, SP_EBREAKDOWN, SP_ENONFINITE, SP_ERANK, SP_ETIMEOUT, SP_EINTERNAL = range(9)
SP_FP64, SP_MIXED_FP32, SP_MIXED_NS = 0, 1, 2
SP_NOALLOC_SCRATCH_DOUBLES = 1 << 20

# every entry point declared in include/sp.h
EXPORTS = [
    "sp_qdwh_opts_default", "sp_ctx_create", "sp_ctx_destroy", "sp_last_error", "sp_ctx_sync",
    "sp_hodlr_from_band", "sp_qdwh_sign", "sp_projector", "sp_apply", "sp_to_dense", "sp_trace",
    "sp_hodlr_info", "sp_hodlr_destroy", "sp_hodlr_add", "sp_hodlr_mult", "sp_hodlr_cholesky",
    "sp_hodlr_trsm", "sp_inertia", "sp_locate_shift", "sp_qdwh_start", "sp_givens_generate",
    "sp_fastqr_factors", "sp_ctx_set_profiling", "sp_ctx_profile", "sp_ctx_profile_levels", "sp_kernel_name", "sp_kernel_count",
    "sp_launch_count", "sp_inertia_noalloc", "sp_batched_projector", "sp_hodlr_level_ranks",
    "sp_trace_product_band", "sp_qdwh_params_paper",
    "sp_hodlr_transpose", "sp_autotune", "sp_ctx_load_tuning", "sp_ctx_set_tuning",
]


class SpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sp error {code}: {msg}")
        self.code = code


class sp_qdwh_opts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int), ("delta", ctypes.c_double), ("precision", ctypes.c_int),
                ("polish_steps", ctypes.c_int), ("alpha", ctypes.c_double), ("l0", ctypes.c_double),
                ("qr_steps", ctypes.c_int)]


class sp_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("alpha", ctypes.c_double), ("l0", ctypes.c_double),
                ("l", ctypes.c_double * 16), ("a", ctypes.c_double * 16), ("b", ctypes.c_double * 16),
                ("c", ctypes.c_double * 16), ("kind", ctypes.c_int * 16), ("max_rank", ctypes.c_int),
                ("bytes", ctypes.c_size_t), ("ms_param", ctypes.c_double), ("ms_qr", ctypes.c_double),
                ("ms_chol", ctypes.c_double), ("ms_total", ctypes.c_double), ("flops", ctypes.c_double),
                ("ms_mult", ctypes.c_double), ("ms_factor", ctypes.c_double), ("ms_solve", ctypes.c_double),
                ("ms_combine", ctypes.c_double), ("ms_polish", ctypes.c_double), ("levels", ctypes.c_int),
                ("max_rank_level", ctypes.c_int * 32), ("mean_rank_level", ctypes.c_double * 32),
                ("nominal_bytes", ctypes.c_double)]


class sp_tune_result(ctypes.Structure):
    _fields_ = [("leaf", ctypes.c_int32), ("tsqr_chunk", ctypes.c_int32), ("small_tiles", ctypes.c_int32),
                ("ms", ctypes.c_double), ("trials", ctypes.c_int32), ("n_tuned", ctypes.c_int64)]


# stream-ordered allocator callbacks of sp_ctx_create
SP_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
SP_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


def build(force: bool = False, jobs: int = 6) -> str:
    """Compile the CUDA sources for sm_103a into ``libsp.so`` next to this file."""
    srcs = [os.path.join(_CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(_CSRC, "sp_internal.h"), os.path.join(_INCLUDE, "sp.h")]
    if not force and os.path.exists(LIB_PATH):
        if os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(d) for d in deps):
            return LIB_PATH
    objdir = os.path.join(_HERE, "_build")
    os.makedirs(objdir, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src).replace(".cu", ".o"))
        subprocess.check_call(["nvcc", *NVCC_FLAGS, "-I", _INCLUDE, "-c", src, "-o", obj])
        return obj

    with ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-Xlinker", "--no-undefined", "-o", tmp, *objs])
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


_lib = None


def bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    """Declare the C signatures on a loaded library object."""
    P, I, I32, I64, D, S = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                            ctypes.c_size_t)
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "sp_qdwh_opts_default": (None, [ctypes.POINTER(sp_qdwh_opts)]),
        "sp_ctx_create": (I, [P, SP_ALLOC_FN, SP_FREE_FN, P, PP]),
        "sp_ctx_destroy": (None, [P]),
        "sp_last_error": (ctypes.c_char_p, [P]),
        "sp_ctx_sync": (I, [P]),
        "sp_hodlr_from_band": (I, [P, I64, I32, P, I64, D, I32, D, I32, PP]),
        "sp_qdwh_sign": (I, [P, P, ctypes.POINTER(sp_qdwh_opts), PP, ctypes.POINTER(sp_info)]),
        "sp_projector": (I, [P, P, PP]),
        "sp_apply": (I, [P, P, I64, P, I64, P, I64]),
        "sp_to_dense": (I, [P, P, I64, I64, P, I64]),
        "sp_trace": (I, [P, P, ctypes.POINTER(D)]),
        "sp_hodlr_info": (I, [P, P, ctypes.POINTER(I64), ctypes.POINTER(I32), ctypes.POINTER(I32),
                              ctypes.POINTER(S)]),
        "sp_hodlr_destroy": (None, [P]),
        "sp_hodlr_add": (I, [P, D, P, D, P, D, PP]),
        "sp_hodlr_mult": (I, [P, P, P, PP]),
        "sp_hodlr_transpose": (I, [P, P, PP]),
        "sp_autotune": (I, [P, I64, I32, P, I64, D, D, I32, ctypes.c_char_p, ctypes.POINTER(sp_tune_result)]),
        "sp_ctx_load_tuning": (I, [P, ctypes.c_char_p]),
        "sp_ctx_set_tuning": (I, [P, I32, I32]),
        "sp_hodlr_cholesky": (I, [P, P, PP]),
        "sp_hodlr_trsm": (I, [P, P, I, P, PP]),
        "sp_inertia": (I, [P, I64, I32, P, I64, I32, P, P]),
        "sp_locate_shift": (I, [P, I64, I32, P, I64, I64, ctypes.POINTER(D), ctypes.POINTER(D),
                                ctypes.POINTER(D)]),
        "sp_qdwh_start": (I, [P, I64, I32, P, I64, D, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "sp_givens_generate": (I, [P, I64, I32, P, I64, D, P]),
        "sp_fastqr_factors": (I, [P, P, D, PP, PP]),
        "sp_ctx_set_profiling": (I, [P, I]),
        "sp_ctx_profile": (I, [P, I, ctypes.POINTER(I64), ctypes.POINTER(D), ctypes.POINTER(D)]),
        "sp_ctx_profile_levels": (I, [P, I, ctypes.c_void_p]),
        "sp_kernel_name": (ctypes.c_char_p, [I]),
        "sp_kernel_count": (I, []),
        "sp_launch_count": (I64, []),
        "sp_inertia_noalloc": (I, [P, I64, I32, P, I64, I32, P, P]),
        "sp_batched_projector": (I, [P, I32, P, P, P, P, P, I32, D, I32, ctypes.POINTER(sp_qdwh_opts), I32, P, P]),
        "sp_hodlr_level_ranks": (I, [P, P, I32, P, P, ctypes.POINTER(D)]),
        "sp_trace_product_band": (I, [P, P, I32, P, I64, ctypes.POINTER(D)]),
        "sp_qdwh_params_paper": (I, [P, I64, I32, P, I64, D, ctypes.POINTER(D), ctypes.POINTER(D), P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def load() -> ctypes.CDLL:
    """Load the in-tree libsp.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"{LIB_PATH} is missing: run __graft_entry__.build() (nvcc, sm_103a)")
        _lib = bind(ctypes.CDLL(LIB_PATH))
    return _lib


def use_library(lib: ctypes.CDLL) -> None:
    """Route the wrappers below to an already bound library object."""
    global _lib
    _lib = lib


def _ptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _check(ctx, rc: int):
    if rc != SP_OK:
        msg = _lib.sp_last_error(ctx).decode() if ctx else ""
        raise SpError(rc, msg)


# ---------------------------------------------------------------- wrappers --

def sp_ctx_create(stream: int = 0, alloc=None, free=None, user: int = 0):
    """alloc/free: SP_ALLOC_FN / SP_FREE_FN callbacks (keep references to them
    for the context's lifetime), or None for the device's default pool."""
    lib = load() if _lib is None else _lib
    h = ctypes.c_void_p()
    _check(None, lib.sp_ctx_create(ctypes.c_void_p(stream), alloc if alloc is not None else SP_ALLOC_FN(),
                                   free if free is not None else SP_FREE_FN(), ctypes.c_void_p(user),
                                   ctypes.byref(h)))
    return h


def sp_ctx_destroy(ctx):
    _lib.sp_ctx_destroy(ctx)


def sp_ctx_sync(ctx):
    _check(ctx, _lib.sp_ctx_sync(ctx))


def sp_hodlr_from_band(ctx, ab, mu: float, leaf: int, tol: float, rank_cap: int = 0, n: int | None = None,
                       b: int | None = None, ldab: int | None = None):
    """ab: band storage, shape (n, b+1) C-contiguous (= LAPACK (b+1) x n)."""
    if n is None:
        n, bp1 = ab.shape
        b, ldab = bp1 - 1, bp1
    h = ctypes.c_void_p()
    _check(ctx, _lib.sp_hodlr_from_band(ctx, n, b, _ptr(ab), ldab, float(mu), leaf, float(tol), rank_cap,
                                        ctypes.byref(h)))
    return h


def sp_qdwh_opts_default() -> sp_qdwh_opts:
    o = sp_qdwh_opts()
    _lib.sp_qdwh_opts_default(ctypes.byref(o))
    return o


def sp_qdwh_sign(ctx, A, opts: sp_qdwh_opts | None = None):
    """Returns (sign handle, sp_info)."""
    h = ctypes.c_void_p()
    info = sp_info()
    _check(ctx, _lib.sp_qdwh_sign(ctx, A, ctypes.byref(opts) if opts is not None else None, ctypes.byref(h),
                                  ctypes.byref(info)))
    return h, info


def sp_projector(ctx, S):
    h = ctypes.c_void_p()
    _check(ctx, _lib.sp_projector(ctx, S, ctypes.byref(h)))
    return h


def sp_apply(ctx, M, nrhs: int, X, ldx: int, Y, ldy: int):
    _check(ctx, _lib.sp_apply(ctx, M, nrhs, _ptr(X), ldx, _ptr(Y), ldy))


def sp_to_dense(ctx, M, row0: int, nrows: int, out, ld: int):
    _check(ctx, _lib.sp_to_dense(ctx, M, row0, nrows, _ptr(out), ld))


def sp_trace(ctx, M) -> float:
    t = ctypes.c_double()
    _check(ctx, _lib.sp_trace(ctx, M, ctypes.byref(t)))
    return t.value


def sp_trace_product_band(ctx, M, ab, b=None, ldab=None) -> float:
    """trace(M A) for the symmetric band A given as (n, b+1) band storage."""
    if b is None:
        b = ab.shape[1] - 1
        ldab = ab.shape[1]
    t = ctypes.c_double()
    _check(ctx, _lib.sp_trace_product_band(ctx, M, b, _ptr(ab), ldab, ctypes.byref(t)))
    return t.value


def sp_hodlr_info(ctx, M):
    n, lv, mr, by = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_size_t()
    _check(ctx, _lib.sp_hodlr_info(ctx, M, ctypes.byref(n), ctypes.byref(lv), ctypes.byref(mr), ctypes.byref(by)))
    return n.value, lv.value, mr.value, by.value


def sp_hodlr_level_ranks(ctx, M, nlevels: int = 32):
    """(max rank per level, mean rank per level, nominal bytes) for levels 1..nlevels."""
    import numpy as _np
    mx = _np.zeros(nlevels, dtype=_np.int32)
    mean = _np.zeros(nlevels)
    nb = ctypes.c_double()
    _check(ctx, _lib.sp_hodlr_level_ranks(ctx, M, nlevels, mx.ctypes.data, mean.ctypes.data, ctypes.byref(nb)))
    return mx, mean, nb.value


def sp_hodlr_destroy(M):
    if M:
        _lib.sp_hodlr_destroy(M)


def sp_hodlr_add(ctx, alpha, A, beta, B, gamma):
    h = ctypes.c_void_p()
    _check(ctx, _lib.sp_hodlr_add(ctx, float(alpha), A, float(beta), B, float(gamma), ctypes.byref(h)))
    return h


def sp_autotune(ctx, ab, mu: float, tol: float = 1e-10, precision: int = 0, cache_path: str | None = None):
    """Tuned (leaf, TSQR chunk, small tiles) for this band's size class; see include/sp.h."""
    n, bp1 = ab.shape
    r = sp_tune_result()
    _check(ctx, _lib.sp_autotune(ctx, n, bp1 - 1, _ptr(ab), bp1, float(mu), float(tol), int(precision),
                                 cache_path.encode() if cache_path else None, ctypes.byref(r)))
    return r


def sp_ctx_load_tuning(ctx, cache_path: str):
    _check(ctx, _lib.sp_ctx_load_tuning(ctx, cache_path.encode()))


def sp_ctx_set_tuning(ctx, tsqr_chunk: int = 512, small_tiles: bool = True):
    _check(ctx, _lib.sp_ctx_set_tuning(ctx, int(tsqr_chunk), int(bool(small_tiles))))


def sp_hodlr_transpose(ctx, M):
    h = ctypes.c_void_p()
    _check(ctx, _lib.sp_hodlr_transpose(ctx, M, ctypes.byref(h)))
    return h


def sp_hodlr_mult(ctx, A, B):
    h = ctypes.c_void_p()
    _check(ctx, _lib.sp_hodlr_mult(ctx, A, B, ctypes.byref(h)))
    return h


def sp_hodlr_cholesky(ctx, Z):
    h = ctypes.c_void_p()
    _check(ctx, _lib.sp_hodlr_cholesky(ctx, Z, ctypes.byref(h)))
    return h


def sp_hodlr_trsm(ctx, L, trans: int, B):
    h = ctypes.c_void_p()
    _check(ctx, _lib.sp_hodlr_trsm(ctx, L, int(trans), B, ctypes.byref(h)))
    return h


def sp_inertia(ctx, ab, shifts, counts, n=None, b=None, ldab=None):
    if n is None:
        n, bp1 = ab.shape
        b, ldab = bp1 - 1, bp1
    _check(ctx, _lib.sp_inertia(ctx, n, b, _ptr(ab), ldab, len(shifts), _ptr(shifts), _ptr(counts)))


def sp_locate_shift(ctx, ab, nu: int, n=None, b=None, ldab=None):
    if n is None:
        n, bp1 = ab.shape
        b, ldab = bp1 - 1, bp1
    mu, lo, hi = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(ctx, _lib.sp_locate_shift(ctx, n, b, _ptr(ab), ldab, nu, ctypes.byref(mu), ctypes.byref(lo),
                                     ctypes.byref(hi)))
    return mu.value, lo.value, hi.value


def sp_qdwh_start(ctx, ab, mu: float, n=None, b=None, ldab=None):
    if n is None:
        n, bp1 = ab.shape
        b, ldab = bp1 - 1, bp1
    a, l0 = ctypes.c_double(), ctypes.c_double()
    _check(ctx, _lib.sp_qdwh_start(ctx, n, b, _ptr(ab), ldab, float(mu), ctypes.byref(a), ctypes.byref(l0)))
    return a.value, l0.value


def sp_qdwh_params_paper(ctx, ab, mu: float, n=None, b=None, ldab=None):
    """The paper's normest/condest start: (alpha, l0, power iterations, LU solves)."""
    import numpy as _np
    if n is None:
        n, bp1 = ab.shape
        b, ldab = bp1 - 1, bp1
    a, l0 = ctypes.c_double(), ctypes.c_double()
    it = _np.zeros(2, dtype=_np.int32)
    _check(ctx, _lib.sp_qdwh_params_paper(ctx, n, b, _ptr(ab), ldab, float(mu), ctypes.byref(a), ctypes.byref(l0),
                                          it.ctypes.data))
    return a.value, l0.value, int(it[0]), int(it[1])


def sp_givens_generate(ctx, n: int, b: int, ab, ldab: int, scale: float, cs):
    _check(ctx, _lib.sp_givens_generate(ctx, n, b, _ptr(ab), ldab, float(scale), _ptr(cs)))


def sp_fastqr_factors(ctx, A, scale: float):
    q1, q2 = ctypes.c_void_p(), ctypes.c_void_p()
    _check(ctx, _lib.sp_fastqr_factors(ctx, A, float(scale), ctypes.byref(q1), ctypes.byref(q2)))
    return q1, q2


def sp_ctx_set_profiling(ctx, on: bool):
    _check(ctx, _lib.sp_ctx_set_profiling(ctx, int(bool(on))))


def sp_ctx_profile(ctx):
    """{kernel name: (launches, ms, flops)} for every kernel family."""
    out = {}
    for k in range(_lib.sp_kernel_count()):
        la, ms, fl = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        _check(ctx, _lib.sp_ctx_profile(ctx, k, ctypes.byref(la), ctypes.byref(ms), ctypes.byref(fl)))
        out[_lib.sp_kernel_name(k).decode()] = (la.value, ms.value, fl.value)
    return out


def sp_ctx_profile_levels(ctx, nlevels: int = 32):
    """Per-tree-level self time (ms) of the H-Cholesky nodes while profiling."""
    import numpy as _np
    out = _np.zeros(nlevels)
    _check(ctx, _lib.sp_ctx_profile_levels(ctx, nlevels, out.ctypes.data))
    return out


def sp_launch_count() -> int:
    return int(_lib.sp_launch_count())


def sp_inertia_noalloc(ctx, n: int, b: int, ab, ldab: int, nshift: int, shifts, counts):
    """Device band, shifts and counts; scratch inside the library (no allocation)."""
    _check(ctx, _lib.sp_inertia_noalloc(ctx, n, b, _ptr(ab), ldab, nshift, _ptr(shifts), _ptr(counts)))


def sp_batched_projector(ctx, bands, mus, leaf: int = 0, tol: float = 1e-10, rank_cap: int = 0, opts=None,
                         nstreams: int = 0):
    """bands: list of (n, b+1) band arrays (numpy: host, torch: device); returns
    (list of projector handles, list of sp_info)."""
    import numpy as _np
    nb = len(bands)
    n = _np.array([x.shape[0] for x in bands], dtype=_np.int64)
    b = _np.array([x.shape[1] - 1 for x in bands], dtype=_np.int32)
    ld = _np.array([x.shape[1] for x in bands], dtype=_np.int64)
    ptrs = (ctypes.c_void_p * max(nb, 1))(*[_ptr(x) for x in bands])
    mu = _np.ascontiguousarray(mus, dtype=_np.float64)
    out = (ctypes.c_void_p * max(nb, 1))()
    infos = (sp_info * max(nb, 1))()
    _check(ctx, _lib.sp_batched_projector(ctx, nb, n.ctypes.data, b.ctypes.data, ctypes.cast(ptrs, ctypes.c_void_p),
                                          ld.ctypes.data, mu.ctypes.data, leaf, float(tol), rank_cap,
                                          ctypes.byref(opts) if opts is not None else None, nstreams,
                                          ctypes.cast(out, ctypes.c_void_p), ctypes.cast(infos, ctypes.c_void_p)))
    return [ctypes.c_void_p(out[i]) for i in range(nb)], [infos[i] for i in range(nb)]
