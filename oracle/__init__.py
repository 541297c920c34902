"""CPU oracle for the hQDWH spectral projector (arXiv 1608.01164).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by
the benchmark's CPU-baseline leg, never by the GPU library.  It shares no code
with the CUDA path.

What it computes (plain definitions, FP64 unless stated):
  * ``projector``      Pi_{<mu}(A) = V_nu V_nu^T from a hand-written dense
                       symmetric eigensolver (Sec. 1 and Sec. 2: the spectral
                       projector onto the eigenvalues below mu).
  * ``sturm_count`` / ``band_count``  inertia nu(sigma) = #{lambda < sigma}
                       (Sylvester's law of inertia on an LDL^T factorisation).
  * ``locate_mu``      bisection on the inertia count: mu between lambda_nu and
                       lambda_{nu+1}, with the gap brackets.
  * ``qdwh_dense``     dense QDWH with one QR-based step and then
                       Cholesky-based steps (Sec. 2.1-2.2, Eqs. (reccur),
                       (qdwh_qr_reccur), (qdwh_chol_reccur)).
  * ``fastqr_replay``  dense replay of the Givens sequence of Algorithm 1
                       (tridiagonal) / Algorithm 2 (banded) on [cA; I].
  * ``qdwh_params`` / ``qdwh_schedule``  the scalar recurrence for a_k, b_k,
                       c_k, l_k (Eq. (qdwh_parameters_abc)).
  * error measures e_id, e_trace, e_SP (Eq. (error_measures)).
  * the closed-form projector of tridiag(-1, 2, -1) (Sec. 6.2, 1D Laplace).

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` against a closed form, a brute-force independent
algorithm, a library routine or an invariant.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from typing import NamedTuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/liboracle.so with the host gcc."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        L, D, P = ctypes.c_long, ctypes.c_double, ctypes.c_void_p
        sig = {
            "orc_sturm_count": (L, [L, P, P, D]),
            "orc_band_ldl_count": (L, [L, L, P, L, D]),
            "orc_band_to_dense": (None, [L, L, P, L, D, P, L]),
            "orc_householder_tridiag": (None, [L, P, L, P, P, P, L]),
            "orc_tridiag_qr": (ctypes.c_int, [L, P, P, L, P, L]),
            "orc_eigh": (ctypes.c_int, [L, P, L, P, P, L]),
            "orc_eigh_tridiag": (ctypes.c_int, [L, P, P, P, P, L]),
            "orc_projector": (L, [L, P, L, D, P, L, P]),
            "orc_jacobi_eig_ld": (ctypes.c_int, [L, P, L, P, P, L]),
            "orc_qdwh_h": (D, [D]),
            "orc_qdwh_params": (None, [D, P, P, P, P]),
            "orc_qdwh_dense": (ctypes.c_int, [L, P, L, D, D, D, ctypes.c_int, ctypes.c_int, P, L, P, P, P, P, P, P, L]),
            "orc_fastqr_replay": (L, [L, L, P, L, D, P, L, P, L, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _band_arrays(ab: np.ndarray):
    ab = np.ascontiguousarray(ab, dtype=np.float64)
    n, bp1 = ab.shape
    return ab, n, bp1 - 1


# ---------------------------------------------------------------- inertia ---

def sturm_count(ab: np.ndarray, sigma: float) -> int:
    """#{eigenvalues < sigma} of a symmetric tridiagonal matrix (band storage)."""
    ab, n, b = _band_arrays(ab)
    assert b == 1, "sturm_count needs a tridiagonal band"
    a = np.ascontiguousarray(ab[:, 0])
    e = np.ascontiguousarray(ab[: max(n - 1, 0), 1]) if n > 1 else np.zeros(1)
    return int(_load().orc_sturm_count(n, _p(a), _p(e), float(sigma)))


def band_count(ab: np.ndarray, sigma: float) -> int:
    """#{eigenvalues < sigma} of a symmetric banded matrix (band storage)."""
    ab, n, b = _band_arrays(ab)
    if b == 0:
        return int(np.count_nonzero(ab[:, 0] < sigma))
    if b == 1:
        return sturm_count(ab, sigma)
    return int(_load().orc_band_ldl_count(n, b, _p(ab), b + 1, float(sigma)))


def gershgorin(ab: np.ndarray):
    """Interval [lo, hi] containing the spectrum (Gershgorin discs)."""
    A = None
    n, bp1 = ab.shape
    rad = np.zeros(n)
    for d in range(1, bp1):
        m = n - d
        if m <= 0:
            break
        v = np.abs(ab[:m, d])
        rad[:m] += v
        rad[d:] += v
    lo = float(np.min(ab[:, 0] - rad))
    hi = float(np.max(ab[:, 0] + rad))
    del A
    return lo, hi


class Shift(NamedTuple):
    mu: float           # shift strictly between lambda_nu and lambda_{nu+1}
    nu: int
    lam_nu: tuple       # (lo, hi): lambda_nu in [lo, hi)
    lam_nu1: tuple      # (lo, hi): lambda_{nu+1} in [lo, hi)
    lam_min_lo: float   # lower bound on lambda_1
    lam_max_hi: float   # upper bound on lambda_n


def _bisect_eigenvalue(ab, k, lo, hi, steps=200):
    """Bracket lambda_k (1-based, ascending): returns (x, y) with
    count(x) < k <= count(y), i.e. lambda_k in [x, y)."""
    for _ in range(steps):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if band_count(ab, mid) >= k:
            hi = mid
        else:
            lo = mid
    return lo, hi


def locate_mu(ab: np.ndarray, nu: int) -> Shift:
    """mu = midpoint of the brackets of lambda_nu and lambda_{nu+1}
    (bisection on the inertia count; the reading of Sec. 1's
    lambda_nu < mu < lambda_{nu+1})."""
    n = ab.shape[0]
    glo, ghi = gershgorin(ab)
    pad = 1e-12 * max(1.0, abs(glo), abs(ghi))
    glo -= pad
    ghi += pad
    lam_min = _bisect_eigenvalue(ab, 1, glo, ghi)
    lam_max = _bisect_eigenvalue(ab, n, glo, ghi)
    if nu <= 0:
        return Shift(lam_min[0] - 1.0, 0, (glo, glo), lam_min, glo, lam_max[1])
    if nu >= n:
        return Shift(lam_max[1] + 1.0, n, lam_max, (ghi, ghi), glo, lam_max[1])
    b_nu = _bisect_eigenvalue(ab, nu, glo, ghi)
    b_nu1 = _bisect_eigenvalue(ab, nu + 1, glo, ghi)
    mu = 0.5 * (b_nu[1] + b_nu1[0])
    if not band_count(ab, mu) == nu:
        raise RuntimeError("mu does not separate lambda_nu and lambda_nu+1 (degenerate gap)")
    return Shift(mu, nu, b_nu, b_nu1, lam_min[0], lam_max[1])


def qdwh_start(shift: Shift):
    """alpha >= ||A - mu I||_2 and l0 <= sigma_min((A - mu I)/alpha) from the
    inertia brackets (a guaranteed reading of the paper's normest/condest
    estimates)."""
    mu = shift.mu
    alpha = max(mu - shift.lam_min_lo, shift.lam_max_hi - mu) * (1.0 + 1e-10)
    dist = min(mu - shift.lam_nu[1], shift.lam_nu1[0] - mu)
    return alpha, dist / alpha


# ---------------------------------------------------------- eigensolvers ---

def band_to_dense(ab: np.ndarray, mu: float = 0.0) -> np.ndarray:
    ab, n, b = _band_arrays(ab)
    A = np.zeros((n, n), order="F")
    _load().orc_band_to_dense(n, b, _p(ab), b + 1, float(mu), _p(A), n)
    return A


def eigh(A: np.ndarray):
    """Ascending eigenvalues and eigenvectors of the dense symmetric A."""
    n = A.shape[0]
    B = np.array(A, dtype=np.float64, order="F", copy=True)
    w = np.zeros(n)
    V = np.zeros((n, n), order="F")
    rc = _load().orc_eigh(n, _p(B), n, _p(w), _p(V), n)
    if rc != 0:
        raise RuntimeError("oracle eigh did not converge")
    return w, V


def eigh_tridiag(ab: np.ndarray):
    ab, n, b = _band_arrays(ab)
    assert b == 1
    a = np.ascontiguousarray(ab[:, 0])
    e = np.ascontiguousarray(ab[:, 1])
    w = np.zeros(n)
    V = np.zeros((n, n), order="F")
    rc = _load().orc_eigh_tridiag(n, _p(a), _p(e), _p(w), _p(V), n)
    if rc != 0:
        raise RuntimeError("oracle tridiagonal eigensolver did not converge")
    return w, V


def jacobi_eigh_ld(A: np.ndarray):
    """Independent brute-force eigensolver (cyclic Jacobi, long double)."""
    n = A.shape[0]
    B = np.array(A, dtype=np.float64, order="F", copy=True)
    w = np.zeros(n)
    V = np.zeros((n, n), order="F")
    sweeps = _load().orc_jacobi_eig_ld(n, _p(B), n, _p(w), _p(V), n)
    if sweeps < 0:
        raise RuntimeError("Jacobi did not converge")
    return w, V


def projector_dense(A: np.ndarray, mu: float):
    """Pi_{<mu}(A) = V_nu V_nu^T; returns (Pi, nu, eigenvalues)."""
    n = A.shape[0]
    B = np.array(A, dtype=np.float64, order="F", copy=True)
    P = np.zeros((n, n), order="F")
    w = np.zeros(n)
    nu = _load().orc_projector(n, _p(B), n, float(mu), _p(P), n, _p(w))
    if nu < 0:
        raise RuntimeError("oracle projector failed")
    return P, int(nu), w


def projector(ab: np.ndarray, mu: float):
    """Spectral projector of the banded A onto the eigenvalues below mu."""
    ab, n, b = _band_arrays(ab)
    if b == 1:
        w, V = eigh_tridiag(ab)
        nu = int(np.count_nonzero(w < mu))
        Vn = V[:, :nu]
        return Vn @ Vn.T, nu, w
    return projector_dense(band_to_dense(ab), mu)


def laplace_projector(n: int, nu: int) -> np.ndarray:
    """Closed form of Pi for tridiag(-1, 2, -1): with theta = pi/(n+1),
    Pi_{jl} = (2/(n+1)) sum_{k<=nu} sin(jk theta) sin(lk theta)
            = (D(j-l) - D(j+l)) / (n+1),  D(m) = sum_{k=1}^{nu} cos(k m theta),
    D evaluated by the Dirichlet-kernel identity
      sum_{k=1}^{nu} cos(kx) = sin((nu+1/2)x) / (2 sin(x/2)) - 1/2."""
    theta = math.pi / (n + 1)
    idx = np.arange(1, n + 1, dtype=np.float64)

    def D(m):
        x = m * theta
        out = np.empty_like(x)
        period = np.mod(m, 2 * (n + 1)) == 0
        xs = x[~period]
        out[~period] = np.sin((nu + 0.5) * xs) / (2.0 * np.sin(0.5 * xs)) - 0.5
        out[period] = nu
        return out

    J, L = np.meshgrid(idx, idx, indexing="ij")
    return (D(J - L) - D(J + L)) / (n + 1)


# ---------------------------------------------------------------- QDWH -----

def qdwh_h(l: float) -> float:
    return float(_load().orc_qdwh_h(float(l)))


def qdwh_params(l: float):
    """(a, b, c, l_next) of Eq. (qdwh_parameters_abc) for the bound l."""
    a, b, c, ln = (ctypes.c_double() for _ in range(4))
    _load().orc_qdwh_params(float(l), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(ln))
    return a.value, b.value, c.value, ln.value


def qdwh_schedule(l0: float, delta: float = 1e-15, maxit: int = 20):
    """The scalar recurrence run to the stopping rule |1 - l_k| <= delta:
    a list of (l_k, a_k, b_k, c_k), one per QDWH iteration."""
    out = []
    l = l0
    while abs(1.0 - l) > delta:
        if len(out) >= maxit:
            raise RuntimeError("QDWH schedule did not reach the stopping rule")
        a, b, c, ln = qdwh_params(l)
        out.append((l, a, b, c))
        l = ln
    return out


class QdwhResult(NamedTuple):
    U: np.ndarray
    iters: int
    l: np.ndarray
    a: np.ndarray
    b: np.ndarray
    c: np.ndarray
    kind: np.ndarray   # 1 = QR-based, 2 = Cholesky-based
    X1: np.ndarray


def qdwh_dense(A: np.ndarray, alpha: float, l0: float, delta: float = 1e-15, qr_policy: int = 1,
               maxit: int = 20) -> QdwhResult:
    """Dense QDWH for sign(A) (A symmetric nonsingular, already shifted).
    qr_policy = 1: one QR-based step then Cholesky (the paper's choice);
    qr_policy = -1: QR-based while c_k > 100 (the switching rule compared in
    Table 1)."""
    n = A.shape[0]
    Af = np.array(A, dtype=np.float64, order="F")
    U = np.zeros((n, n), order="F")
    X1 = np.zeros((n, n), order="F")
    lh, ah, bh, ch = (np.zeros(maxit) for _ in range(4))
    kh = np.zeros(maxit, dtype=np.int32)
    it = _load().orc_qdwh_dense(n, _p(Af), n, float(alpha), float(l0), float(delta), int(qr_policy), int(maxit),
                                _p(U), n, _p(lh), _p(ah), _p(bh), _p(ch), _p(kh), _p(X1), n)
    if it < 0:
        raise RuntimeError("dense QDWH failed (Cholesky breakdown or no convergence)")
    return QdwhResult(U, it, lh[:it], ah[:it], bh[:it], ch[:it], kh[:it], X1)


class FastQR(NamedTuple):
    R: np.ndarray        # 2n x n
    Q: np.ndarray        # 2n x 2n (None if not requested)
    p: np.ndarray        # rotation pair, first (kept) row, 0-based
    q: np.ndarray        # rotation pair, second (annihilated) row
    c: np.ndarray
    s: np.ndarray


def fastqr_replay(ab: np.ndarray, scale: float = 1.0, want_q: bool = True) -> FastQR:
    """Dense replay of Algorithm 1/2 on [scale * A; I]."""
    ab, n, b = _band_arrays(ab)
    R = np.zeros((2 * n, n), order="F")
    Q = np.zeros((2 * n, 2 * n), order="F") if want_q else None
    cap = (2 * b + 1) * n + 8
    P = np.zeros(cap, dtype=np.int64)
    Qi = np.zeros(cap, dtype=np.int64)
    C = np.zeros(cap)
    S = np.zeros(cap)
    cnt = _load().orc_fastqr_replay(n, b, _p(ab), b + 1, float(scale), _p(R), 2 * n,
                                    _p(Q) if want_q else None, 2 * n, _p(P), _p(Qi), _p(C), _p(S))
    return FastQR(R, Q, P[:cnt], Qi[:cnt], C[:cnt], S[:cnt])


def fastqr_rotation_count(n: int, b: int) -> int:
    """(2b+1) n - b^2 - b rotations (3n - 2 for b = 1), Sec. 4.1-4.2."""
    return (2 * b + 1) * n - b * b - b


# --------------------------------------------------------- error measures --

def sym_norm2(M: np.ndarray) -> float:
    """2-norm of a symmetric matrix = max |eigenvalue| (oracle eigensolver)."""
    Ms = 0.5 * (M + M.T)
    w, _ = eigh(Ms)
    return float(np.max(np.abs(w))) if w.size else 0.0


def error_measures(U: np.ndarray, A: np.ndarray, Pi: np.ndarray, nu: int):
    """e_id = ||U^2 - I||_2, e_trace = |tr U - tr sign(A)|,
    e_SP = ||(I - U)/2 - Pi||_2  (Eq. (error_measures))."""
    n = U.shape[0]
    e_id = sym_norm2(U @ U - np.eye(n))
    e_trace = abs(float(np.trace(U)) - (n - 2 * nu))
    e_sp = sym_norm2(0.5 * (np.eye(n) - U) - Pi)
    return e_id, e_trace, e_sp
