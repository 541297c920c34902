"""Seeded synthetic inputs for the spectral-projector workloads.

This module only draws random band matrices; it holds none of the method's
arithmetic.  Both the GPU library's tests/benchmark and the CPU oracle take
their inputs from here, so the two sides always see the same bytes.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) evaluated in counter mode -- draw t of a
stream with seed s is mix(s + (t + 1) * 0x9E3779B97F4A7C15) -- mapped to a
53-bit uniform in [0, 1).  Normal deviates use the Box--Muller transform on
consecutive pairs of uniforms.

Band storage (LAPACK lower band, column-major): an array ``ab`` of shape
(n, b + 1), C-contiguous, with ``ab[j, d] = A[j + d, j]`` for
0 <= d <= b and j + d < n; unused tail entries are zero.  Its memory is the
LAPACK (b+1) x n column-major array with ldab = b + 1.

Workloads (the paper's experiments use banded symmetric matrices with
prescribed spectra, Sec. 6.1; these synthetic stand-ins have the same shape,
band structure and an interior shift mu with nu = n/2 or n/3):
  * "uniform_tridiag"  diagonal and off-diagonal i.i.d. U[-1, 1]
  * "laplace"          tridiag(-1, 2, -1) (deterministic)
  * "anderson"         off-diagonal -1, diagonal i.i.d. U[-w, w]
  * "normal_band"      all band entries i.i.d. N(0, 1) * scale
  * "uniform_band"     all band entries i.i.d. U[-1, 1]
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

SEED_BASE = 1608011640


def workload_seed(config_index: int, instance: int = 0) -> int:
    """Seed of instance ``instance`` of workload ``config_index`` (0-based)."""
    return SEED_BASE + 100 * config_index + instance


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` consecutive SplitMix64 outputs (uint64) of stream ``seed``."""
    with np.errstate(over="ignore"):
        t = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + t * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """53-bit uniforms in [0, 1)."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform(seed: int, count: int, lo: float, hi: float, offset: int = 0) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, count, offset)


def normal(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Box--Muller on pairs (u1, u2): sqrt(-2 ln(1 - u1)) cos(2 pi u2)."""
    u = uniform01(seed, 2 * count, 2 * offset)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


def _fill_band(n: int, b: int, values: np.ndarray) -> np.ndarray:
    """Place values into band storage, diagonal first, then sub-diagonal 1, ..."""
    ab = np.zeros((n, b + 1), dtype=np.float64)
    pos = 0
    for d in range(b + 1):
        m = n - d
        if m <= 0:
            break
        ab[:m, d] = values[pos : pos + m]
        pos += m
    return ab


def band_count(n: int, b: int) -> int:
    return sum(max(n - d, 0) for d in range(b + 1))


def uniform_band(n: int, b: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    return _fill_band(n, b, uniform(seed, band_count(n, b), lo, hi))


def normal_band(n: int, b: int, seed: int, scale: float = 1.0) -> np.ndarray:
    return _fill_band(n, b, scale * normal(seed, band_count(n, b)))


def uniform_tridiag(n: int, seed: int) -> np.ndarray:
    return uniform_band(n, 1, seed)


def laplace(n: int) -> np.ndarray:
    ab = np.zeros((n, 2), dtype=np.float64)
    ab[:, 0] = 2.0
    ab[: n - 1, 1] = -1.0
    return ab


def anderson(n: int, seed: int, w: float) -> np.ndarray:
    ab = np.zeros((n, 2), dtype=np.float64)
    ab[:, 0] = uniform(seed, n, -w, w)
    ab[: n - 1, 1] = -1.0
    return ab


def dense_from_band(ab: np.ndarray) -> np.ndarray:
    """Dense symmetric matrix from band storage (input bookkeeping only)."""
    n, bp1 = ab.shape
    A = np.zeros((n, n))
    for d in range(bp1):
        m = n - d
        if m <= 0:
            break
        idx = np.arange(m)
        A[idx + d, idx] = ab[:m, d]
        A[idx, idx + d] = ab[:m, d]
    return A


# --------------------------------------------------------------------------
# Banded matrices with a prescribed spectrum (the paper's synthetic test
# matrices, Sec. 6.1): an orthogonal similarity of diag(lambda) by Givens
# rotations, with the fill-in outside the band chased to the bottom-right
# corner.  Input construction only; nothing of the projector method.
# --------------------------------------------------------------------------

def gap_spectrum(n: int, gap: float) -> np.ndarray:
    """n eigenvalues equispaced in [-1, -gap] (first n/2) and [gap, 1] (the
    rest), endpoints included, so that mu = 0 separates the lower n/2 from the
    upper ones and the spectral gap at mu is exactly 2 gap."""
    k = n // 2
    lo = np.linspace(gap, 1.0, k) if k > 1 else np.full(k, gap)
    hi = np.linspace(gap, 1.0, n - k) if n - k > 1 else np.full(n - k, gap)
    return np.concatenate([-lo[::-1], hi])


def _rotate(A: np.ndarray, p: int, c: float, s: float, lo: int, hi: int) -> None:
    """A <- G^T A G for the rotation G acting on indices p, p+1 as
    [[c, -s], [s, c]] (G^T [x, y] = [c x + s y, -s x + c y]); rows and columns
    are touched only over [lo, hi)."""
    rows = A[p:p + 2, lo:hi]
    x, y = rows[0].copy(), rows[1].copy()
    rows[0] = c * x + s * y
    rows[1] = -s * x + c * y
    cols = A[lo:hi, p:p + 2]
    x, y = cols[:, 0].copy(), cols[:, 1].copy()
    cols[:, 0] = c * x + s * y
    cols[:, 1] = -s * x + c * y


def prescribed_band(lam: np.ndarray, b: int) -> np.ndarray:
    """Symmetric b-banded matrix with eigenvalues lam, in lower band storage.

    For i = n-1, ..., 1 (0-based pair (i-1, i)): the rotation that annihilates
    the second component of [a_ii, 1]^T is applied as a similarity on rows and
    columns i-1, i; the entry it creates b+1 below the diagonal is chased down
    by rotations on (k-1, k) that annihilate it, each moving the bulge b rows
    further, until it leaves the matrix.  Dense O(n^2) storage, O(b) work per
    rotation: meant for n up to a few thousand."""
    lam = np.asarray(lam, dtype=np.float64)
    n = lam.shape[0]
    A = np.diag(lam)
    w = b + 2  # band plus one bulge on each side of the touched indices
    for i in range(n - 1, 0, -1):
        x = A[i, i]
        r = math.hypot(x, 1.0)
        c, s = x / r, 1.0 / r
        p = i - 1
        _rotate(A, p, c, s, max(0, p - w), min(n, p + 2 + w))
        k, m = p + 1 + b, p  # the bulge A[k, m] below the band
        while k < n:
            f, g = A[k - 1, m], A[k, m]
            if g != 0.0:
                r = math.hypot(f, g)
                c, s = f / r, g / r
                _rotate(A, k - 1, c, s, max(0, k - 1 - w), min(n, k + 1 + w))
                A[k, m] = A[m, k] = 0.0
            k, m = k + b, k - 1
    ab = np.zeros((n, b + 1))
    for d in range(b + 1):
        ab[: n - d, d] = np.diagonal(A, -d)
    return ab


# --------------------------------------------------------------------------
# The five workloads.  Each returns a list of (name, ab, nu) instances; the
# shift mu is located separately (by inertia counts) from nu.
# --------------------------------------------------------------------------

def workload(index: int, variant: str = "main", n: int | None = None):
    """Instances of workload ``index`` (0..4).

    0: tridiagonal n=1024, U[-1,1] entries, nu=512, leaf 64, tol 1e-10;
       variant "laplace": tridiag(-1,2,-1), mu = 2.
    1: Anderson tridiagonal n=16384, off-diagonal -1, diagonal U[-0.25,0.25],
       nu = n/2, leaf 128; variant "band8": b=8, N(0,1) entries.
    2: banded n=32768, b=16, N(0,1)/sqrt(16), nu = n/2.
    3: 256 instances, n log-uniform in [512, 8192], b in {1,2,4,8}, U[-1,1],
       nu in {n/3, n/2}.
    4: tridiagonal n=100000, off-diagonal -1, diagonal U[-0.5,0.5], nu=n/2,
       leaf 256; variant "band4": b=4, N(0,1) entries.
    ``n`` overrides the size (for reduced test cases of the same recipe).
    """
    seed = workload_seed(index)
    if index == 0:
        nn = n or 1024
        if variant == "laplace":
            return [("laplace", laplace(nn), nn // 2)]
        return [("uniform_tridiag", uniform_tridiag(nn, seed), nn // 2)]
    if index == 1:
        nn = n or 16384
        if variant == "band8":
            return [("normal_band8", normal_band(nn, 8, seed + 1), nn // 2)]
        return [("anderson", anderson(nn, seed, 0.25), nn // 2)]
    if index == 2:
        nn = n or 32768
        return [("normal_band16", normal_band(nn, 16, seed, 1.0 / math.sqrt(16.0)), nn // 2)]
    if index == 3:
        out = []
        count = 256 if n is None else n
        for t in range(count):
            s = workload_seed(3, t)
            u = uniform01(s, 3, offset=0)
            nn = int(math.floor(math.exp(math.log(512.0) + u[0] * (math.log(8192.0) - math.log(512.0)))))
            b = (1, 2, 4, 8)[min(int(u[1] * 4.0), 3)]
            nu = nn // 3 if u[2] < 0.5 else nn // 2
            ab = _fill_band(nn, b, uniform(s, band_count(nn, b), -1.0, 1.0, offset=3))
            out.append((f"batch{t}_n{nn}_b{b}", ab, nu))
        return out
    if index == 4:
        nn = n or 100000
        if variant == "band4":
            return [("normal_band4", normal_band(nn, 4, seed + 1), nn // 2)]
        return [("anderson_wide", anderson(nn, seed, 0.5), nn // 2)]
    raise ValueError(f"unknown workload {index}")
