"""Seeded synthetic inputs for the batched symmetric eigensolver.

Holds input generation only (no step of the eigensolver itself), so that the CUDA path and the FP64
oracle can be fed the same matrices. Everything is drawn in FP64 with ``numpy.random.default_rng``,
symmetrized as (A + A^T)/2 and rounded to FP32; the oracle upcasts those FP32 values exactly, so both
sides solve the same matrix.

Workloads (the paper uses no public dataset and states no matrix distribution; these stand in):

* ``known_spectrum``: A = Q diag(lam) Q^T, Q from the QR factorization of an N(0,1) n x n matrix with
  column signs fixed by sign(diag R); lam = n sorted draws of U[-1, 1 - (n-1) 1e-3] plus i * 1e-3, so
  every gap is at least 1e-3 and lam stays in [-1, 1].
* ``covariance``: A = X X^T / m + 1e-3 I with X an n x m N(0,1) matrix, m = 2n (Marchenko-Pastur
  ratio 1/2: spectrum about [0.086, 2.91] + 1e-3). The shape follows the paper's batch-512 dimension
  sweep.
* ``ragged``: n drawn uniformly per matrix; even indices known-spectrum, odd indices covariance.
"""
from __future__ import annotations

import numpy as np

SEED_PLAIN = 1001
SEED_UNIFORM_BASE = 2000
SEED_RAGGED = 3001
SEED_DIFF = 4001


def _sym32(A: np.ndarray) -> np.ndarray:
    return (0.5 * (A + np.swapaxes(A, -1, -2))).astype(np.float32)


def known_spectrum(batch: int, n: int, seed: int = SEED_PLAIN, gap: float = 1e-3):
    """A = Q diag(lam) Q^T with min gap ``gap`` and lam in [-1, 1]. Returns (A float32, lam float64)."""
    rng = np.random.default_rng(seed)
    A = np.zeros((batch, n, n))
    lams = np.zeros((batch, n))
    for b in range(batch):
        G = rng.standard_normal((n, n))
        Q, R = np.linalg.qr(G)
        Q = Q * np.where(np.diag(R) < 0, -1.0, 1.0)[None, :]
        lam = np.sort(rng.uniform(-1.0, 1.0 - (n - 1) * gap, size=n)) + gap * np.arange(n)
        A[b] = (Q * lam[None, :]) @ Q.T
        lams[b] = lam
    return _sym32(A), lams


def covariance(batch: int, n: int, seed: int | None = None, ratio: int = 2, ridge: float = 1e-3):
    """A = X X^T / m + ridge I with X ~ N(0,1)^{n x m}, m = ratio * n. Returns float32 [batch, n, n]."""
    if seed is None:
        seed = SEED_UNIFORM_BASE + n
    rng = np.random.default_rng(seed)
    m = ratio * n
    X = rng.standard_normal((batch, n, m))
    A = X @ np.swapaxes(X, 1, 2) / m + ridge * np.eye(n)[None]
    return _sym32(A)


def uniform_sizes(batch: int = 512, sizes=(16, 32, 48, 64)):
    """The uniform-size workload: ``batch`` covariances at each n in ``sizes`` (seed 2000 + n)."""
    return {n: covariance(batch, n) for n in sizes}


def ragged(count: int = 8192, nmin: int = 4, nmax: int = 64, seed: int = SEED_RAGGED):
    """Mixed sizes: n ~ U{nmin..nmax}; even index known-spectrum, odd covariance.

    Returns (list of float32 matrices, ns int32 array)."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(nmin, nmax + 1, size=count).astype(np.int32)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    mats = []
    for i in range(count):
        n = int(ns[i])
        if i % 2 == 0:
            A, _ = known_spectrum(1, n, seed=int(seeds[i]))
        else:
            A = covariance(1, n, seed=int(seeds[i]))
        mats.append(A[0])
    return mats, ns


def differentiation(batch: int = 1024, n: int = 32, seed: int = SEED_DIFF, min_gap: float = 1e-3):
    """Covariances (as ``covariance``) redrawn until the smallest eigen-gap of the FP32 matrix (LAPACK, FP64)
    is at least ``min_gap``, plus the loss weights of L = sum_i w_i lambda_i + <G, V>: w ~ N(0,1)^n and
    G ~ N(0,1)^{n x n} per matrix. Returns (A float32 [b,n,n], w float32 [b,n], G float32 [b,n,n])."""
    rng = np.random.default_rng(seed)
    out = np.zeros((batch, n, n), np.float32)
    k = 0
    while k < batch:
        X = rng.standard_normal((n, 2 * n))
        A = _sym32(X @ X.T / (2 * n) + 1e-3 * np.eye(n))
        if np.diff(np.linalg.eigvalsh(A.astype(np.float64))).min() >= min_gap:
            out[k] = A
            k += 1
    w = rng.standard_normal((batch, n)).astype(np.float32)
    G = rng.standard_normal((batch, n, n)).astype(np.float32)
    return out, w, G


def graded(batch: int, n: int, seed: int = 9, decades: float = 6.0):
    """Symmetric N(0,1) matrices scaled two-sidedly by a geometric grading g_i = 10^(-t i/(n-1)),
    t ~ U[0, decades] per batch entry: entries (and eigenvalues) spread over up to `decades` orders of
    magnitude, the large ones in the leading rows. FP32 [batch, n, n]."""
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((batch, n, n))
    S = (X + np.swapaxes(X, 1, 2)) / 2
    t = rng.uniform(0.0, decades, batch)
    g = 10.0 ** (-t[:, None] * np.linspace(0.0, 1.0, n)[None, :])
    return _sym32(S * g[:, :, None] * g[:, None, :])


def special_cases(n: int, seed: int = 7):
    """Degenerate inputs that force every branch: zero, identity, diagonal, repeated eigenvalues,
    a rank-one matrix, a block-diagonal matrix (exact zero couplings), a tridiagonal Toeplitz matrix.

    Returns a dict name -> float32 [n, n]."""
    rng = np.random.default_rng(seed)
    out = {}
    out["zero"] = np.zeros((n, n), np.float32)
    out["identity"] = np.eye(n, dtype=np.float32)
    out["diagonal"] = np.diag(rng.uniform(-1, 1, n)).astype(np.float32)
    G = rng.standard_normal((n, n))
    Q, _ = np.linalg.qr(G)
    lam = np.repeat(np.array([-0.5, 0.25, 1.0]), (n + 2) // 3)[:n]
    out["repeated"] = _sym32((Q * lam[None, :]) @ Q.T)
    x = rng.standard_normal(n)
    out["rank_one"] = _sym32(np.outer(x, x) / max(n, 1))
    B = np.zeros((n, n))
    h = n // 2
    if h > 0:
        B[:h, :h] = _sym32(rng.standard_normal((h, h)))
    if n - h > 0:
        B[h:, h:] = _sym32(rng.standard_normal((n - h, n - h)))
    out["block_diagonal"] = _sym32(B)
    T = np.diag(np.full(n, 0.5)) + np.diag(np.full(max(n - 1, 0), 0.25), 1) + np.diag(np.full(max(n - 1, 0), 0.25), -1)
    out["toeplitz"] = T.astype(np.float32)
    return out
