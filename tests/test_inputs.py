"""The seeded input generators shared by the oracle tests and the GPU tests:
SplitMix64 pinned to the published test vectors of its reference
implementation, the derived distributions checked by their moments, and the
workload recipes by their shapes and ranges."""
import numpy as np

import sp_inputs


def test_splitmix64_reference_vectors():
    # first outputs of the reference SplitMix64 generator for seeds 0 and 1234567
    assert [int(v) for v in sp_inputs.splitmix64(0, 3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(v) for v in sp_inputs.splitmix64(1234567, 5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
        16408922859458223821]


def test_counter_mode_offsets():
    full = sp_inputs.splitmix64(99, 40)
    assert np.array_equal(sp_inputs.splitmix64(99, 15, offset=25), full[25:])
    u = sp_inputs.uniform01(7, 30)
    assert np.array_equal(sp_inputs.uniform01(7, 10, offset=20), u[20:])


def test_distributions():
    u = sp_inputs.uniform01(2024, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 3e-3 and abs(u.var() - 1.0 / 12.0) < 2e-3
    z = sp_inputs.normal(2025, 200000)
    assert abs(z.mean()) < 1e-2 and abs(z.var() - 1.0) < 1.5e-2
    assert abs(np.mean(z ** 4) - 3.0) < 0.1  # Gaussian kurtosis
    v = sp_inputs.uniform(3, 1000, -0.25, 0.25)
    assert v.min() >= -0.25 and v.max() <= 0.25


def test_workload_recipes():
    (name, ab, nu), = sp_inputs.workload(0)
    assert ab.shape == (1024, 2) and nu == 512
    (_, ab, nu), = sp_inputs.workload(0, variant="laplace")
    assert np.all(ab[:, 0] == 2.0) and np.all(ab[:-1, 1] == -1.0) and ab[-1, 1] == 0.0
    (_, ab, nu), = sp_inputs.workload(1, n=2048)
    assert ab.shape == (2048, 2) and np.all(np.abs(ab[:, 0]) <= 0.25) and np.all(ab[:-1, 1] == -1.0)
    (_, ab, nu), = sp_inputs.workload(4, variant="band4", n=1000)
    assert ab.shape == (1000, 5) and nu == 500
    assert np.all(ab[1000 - 4:, 4] == 0.0)  # entries outside the matrix are zero
    inst = sp_inputs.workload(3, n=64)
    assert len(inst) == 64
    for _, ab, nu in inst:
        n, b = ab.shape[0], ab.shape[1] - 1
        assert 512 <= n <= 8192 and b in (1, 2, 4, 8) and nu in (n // 3, n // 2)
        assert np.all(np.abs(ab) <= 1.0)
    # the same seed gives the same instance; another seed does not
    (_, a1, _), = sp_inputs.workload(1, n=512)
    (_, a2, _), = sp_inputs.workload(1, n=512)
    assert np.array_equal(a1, a2)
    assert not np.array_equal(sp_inputs.uniform_band(300, 2, 1), sp_inputs.uniform_band(300, 2, 2))


def test_prescribed_spectrum_band():
    """Sec. 6.1 construction: the band reproduces the prescribed eigenvalues,
    has exactly b diagonals below the main one, and is populated."""
    for n, b, gap in [(120, 1, 1e-1), (200, 3, 1e-3), (300, 8, 1e-6)]:
        lam = sp_inputs.gap_spectrum(n, gap)
        assert np.sum(lam < 0) == n // 2
        assert np.all(np.abs(lam) >= gap) and np.all(np.abs(lam) <= 1.0)
        assert np.min(np.abs(lam)) == gap and np.max(np.abs(lam)) == 1.0  # the gap is attained
        ab = sp_inputs.prescribed_band(lam, b)
        assert ab.shape == (n, b + 1)
        w = np.linalg.eigvalsh(sp_inputs.dense_from_band(ab))
        assert np.max(np.abs(w - np.sort(lam))) < 1e-12
        assert np.mean(ab[: n - b, b] != 0.0) > 0.7
        assert np.all(ab[: n - 1, 1] != 0.0)
        assert np.all(ab[n - b:, b] == 0.0)  # padding outside the matrix
