"""The seeded generators produce the documented shapes and spectra (CPU only)."""
import numpy as np

from paper_2604_27325_gb300 import workloads as wl


def test_known_spectrum_gap_and_range():
    A, lam = wl.known_spectrum(16, 16)
    assert A.dtype == np.float32 and A.shape == (16, 16, 16)
    assert np.array_equal(A, np.swapaxes(A, 1, 2))
    assert np.all(np.diff(lam, axis=1) >= 1e-3 - 1e-12)
    assert lam.min() >= -1 and lam.max() <= 1
    # the FP32 rounding moves the spectrum by far less than the gap
    w = np.linalg.eigvalsh(A.astype(np.float64))
    assert np.abs(w - lam).max() < 1e-5


def test_covariance_shape_and_spectrum():
    for n in (16, 64):
        A = wl.covariance(32, n)
        assert A.dtype == np.float32 and A.shape == (32, n, n)
        assert np.array_equal(A, np.swapaxes(A, 1, 2))
        w = np.linalg.eigvalsh(A.astype(np.float64))
        assert w.min() > 0 and w.max() < 4.5  # Marchenko-Pastur edge (1 + sqrt(1/2))^2 = 2.91 plus noise


def test_generators_are_seeded():
    assert np.array_equal(wl.covariance(3, 8), wl.covariance(3, 8))
    assert not np.array_equal(wl.covariance(3, 8, seed=1), wl.covariance(3, 8, seed=2))
    m1, n1 = wl.ragged(20)
    m2, n2 = wl.ragged(20)
    assert np.array_equal(n1, n2) and all(np.array_equal(a, b) for a, b in zip(m1, m2))
    assert n1.min() >= 4 and n1.max() <= 64


def test_special_cases_are_symmetric():
    for n in (1, 2, 5, 16):
        for name, M in wl.special_cases(n).items():
            assert M.shape == (n, n) and np.array_equal(M, M.T), name


def test_graded_matrices_are_symmetric_seeded_and_graded():
    A = wl.graded(16, 12, seed=5)
    assert A.shape == (16, 12, 12) and A.dtype == np.float32
    assert np.array_equal(A, np.swapaxes(A, 1, 2))
    assert np.array_equal(A, wl.graded(16, 12, seed=5)) and not np.array_equal(A, wl.graded(16, 12, seed=6))
    # entries spread over several orders of magnitude (the grading reaches up to 10^-6 per side)
    ratios = np.abs(A).max(axis=(1, 2)) / np.abs(A).min(axis=(1, 2))
    assert ratios.max() > 1e4
    assert wl.graded(2, 1).shape == (2, 1, 1)
