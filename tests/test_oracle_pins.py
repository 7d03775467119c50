"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Every stage of the oracle is checked against something other than itself: closed forms, LAPACK
(numpy.linalg), a brute-force cyclic Jacobi written here, and the identities the paper states
(Eq. (2)-(11), (25)). tests/test_oracle_mutations.py plants plausible mistakes in a copy of the oracle
and checks that these pins catch them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2604_27325_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EPS = np.finfo(np.float64).eps


def _tri(d, e):
    return np.diag(d) + np.diag(e, 1) + np.diag(e, -1)


def _rand_sym(rng, n):
    X = rng.standard_normal((n, n))
    return 0.5 * (X + X.T)


# ----------------------------------------------------------------------------- a3: 2x2 leaf


def test_eig2_closed_form():
    """Sec. 2.2: the 2x2 leaf; lam = (a+c)/2 -+ sqrt(((a-c)/2)^2 + b^2)."""
    rng = np.random.default_rng(0)
    for _ in range(200):
        a, b, c = rng.standard_normal(3)
        if rng.random() < 0.1:
            b = 0.0
        lam, Q = oracle.eig2(a, b, c)
        r = math.sqrt(((a - c) / 2) ** 2 + b * b)
        assert sorted(lam) == pytest.approx([(a + c) / 2 - r, (a + c) / 2 + r], abs=1e-14)
        M = np.array([[a, b], [b, c]])
        assert np.allclose(M @ Q, Q * lam[None, :], atol=1e-14)
        assert np.allclose(Q.T @ Q, np.eye(2), atol=1e-15)


# ----------------------------------------------------------------------------- a1


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 16, 33, 64])
def test_householder_reconstructs(n):
    """a1: A = H T H^T with H orthogonal and T tridiagonal (textbook Householder reduction)."""
    rng = np.random.default_rng(n)
    A = _rand_sym(rng, n)
    d, e, H, vk, taus = oracle.tridiagonalize(A)
    T = _tri(d, e) if n > 1 else np.diag(d)
    assert np.linalg.norm(H.T @ H - np.eye(n)) < 1e-14 * n
    assert np.linalg.norm(H @ T @ H.T - A) < 1e-14 * n * np.linalg.norm(A)
    # the product of the stored reflectors is H
    P = np.eye(n)
    for k in range(max(n - 2, 0)):
        v = vk[k]
        assert np.all(v[: k + 1] == 0) and v[k + 1] == 1.0
        P = P @ (np.eye(n) - taus[k] * np.outer(v, v))
    assert np.allclose(P, H, atol=1e-14 * n)
    assert np.allclose(np.linalg.eigvalsh(T), np.linalg.eigvalsh(A), atol=1e-13 * n)


def test_householder_reads_lower_triangle_only():
    rng = np.random.default_rng(3)
    A = _rand_sym(rng, 9)
    B = A.copy()
    B[np.triu_indices(9, 1)] = rng.standard_normal(36) * 100
    d1, e1, *_ = oracle.tridiagonalize(A)
    d2, e2, *_ = oracle.tridiagonalize(B)
    assert np.array_equal(d1, d2) and np.array_equal(e1, e2)


# ----------------------------------------------------------------------------- a2


def test_tearing_golden_4x4():
    """Eq. (1)-(3) on the paper's 4x4 pattern with numbers substituted by hand."""
    g = json.load(open(os.path.join(GOLDEN, "tearing_4x4.json")))
    d1, d2, rho, sig = oracle.tear(g["d"], g["e"], g["cut"])
    e = g["e"]
    T1 = _tri(d1, e[: g["cut"] - 1])
    T2 = _tri(d2, e[g["cut"]:])
    assert np.array_equal(T1, np.array(g["T1_hat"]))
    assert np.array_equal(T2, np.array(g["T2_hat"]))
    assert rho == g["rho"]
    v = np.zeros(4)
    v[g["cut"] - 1], v[g["cut"]] = sig, 1.0
    assert np.array_equal(v, np.array(g["v"]))


@pytest.mark.parametrize("s", [2, 3, 5, 8, 13])
def test_tearing_identity(s):
    """Eq. (2): T = blkdiag(T1^, T2^) + |beta| v v^T for every cut and both signs of beta."""
    rng = np.random.default_rng(s)
    for _ in range(5):
        d, e = rng.standard_normal(s), rng.standard_normal(s - 1)
        T = _tri(d, e)
        for m in range(1, s):
            d1, d2, rho, sig = oracle.tear(d, e, m)
            B = np.zeros((s, s))
            B[:m, :m] = _tri(d1, e[: m - 1])
            B[m:, m:] = _tri(d2, e[m:])
            v = np.zeros(s)
            v[m - 1], v[m] = sig, 1.0
            assert rho == abs(e[m - 1])
            assert np.allclose(B + rho * np.outer(v, v), T, rtol=0, atol=4 * EPS * np.abs(T).max())


# ----------------------------------------------------------------------------- a5: secular equation


def _random_secular(rng, K, spread=1.0):
    d = np.sort(rng.uniform(-spread, spread, K))[::-1].copy()
    z = rng.standard_normal(K)
    z[np.abs(z) < 0.05] = 0.05
    rho = float(rng.uniform(0.1, 2.0))
    return d, z, rho


def _all_roots(d, z, rho, opts=None):
    K = d.shape[0]
    up = d[0] + rho * float(z @ z)
    res = [oracle.secular_root(d, z, rho, up, i, opts) for i in range(K)]
    o = np.array([r[0] for r in res], np.int32)
    t = np.array([r[1] for r in res])
    return o, t, d[o] + t


def test_secular_golden_two_poles():
    """Eq. (8) with two poles: roots of a quadratic derived by hand."""
    g = json.load(open(os.path.join(GOLDEN, "secular_2pole.json")))
    d = np.array(g["D"])[::-1].copy()  # descending, Eq. (9)
    z = np.array(g["z"])[::-1].copy()
    o, t, lam = _all_roots(d, z, g["rho"])
    assert np.allclose(np.sort(lam), g["roots_ascending"], rtol=0, atol=4e-16)


@pytest.mark.parametrize("K", [2, 3, 5, 16, 64])
def test_secular_roots_interlace_and_match_lapack(K):
    """Eq. (9)-(11): d_i < lam_i < d_{i-1}, lam_0 <= d_0 + rho|z|^2; the roots are the eigenvalues of
    D + rho z z^T (LAPACK); trace identity sum lam = sum d + rho |z|^2."""
    rng = np.random.default_rng(100 + K)
    for _ in range(10):
        d, z, rho = _random_secular(rng, K)
        o, t, lam = _all_roots(d, z, rho)
        assert np.all(lam > d)
        assert np.all(lam[1:] < d[:-1])
        assert lam[0] <= d[0] + rho * z @ z
        ref = np.linalg.eigvalsh(np.diag(d) + rho * np.outer(z, z))[::-1]
        assert np.allclose(lam, ref, rtol=0, atol=20 * EPS * K * (np.abs(d).max() + rho * z @ z))
        assert abs(lam.sum() - (d.sum() + rho * z @ z)) < 50 * EPS * K * (np.abs(d).max() + rho * z @ z)
        # each root sits next to the pole it is expressed against
        for i in range(K):
            assert o[i] in (i, i - 1)


def test_secular_characteristic_polynomial():
    """Eq. (6)-(8): det(D + rho z z^T - x I) = det(D - x I) f(x) at arbitrary x."""
    rng = np.random.default_rng(5)
    for K in (2, 4, 7):
        d, z, rho = _random_secular(rng, K)
        _, _, lam = _all_roots(d, z, rho)
        for x in rng.uniform(-2, 2, 5):
            # f(x) at lambda = x: express x against pole 0
            f, *_ = oracle.secular_eval(d, z, rho, 0, x - d[0])
            lhs = np.prod(lam - x)
            rhs = np.prod(d - x) * f
            assert lhs == pytest.approx(rhs, rel=1e-9, abs=1e-12)


def test_secular_derivatives_finite_difference():
    """Eq. (18), (21): f' and f'' against central differences of f."""
    rng = np.random.default_rng(6)
    d, z, rho = _random_secular(rng, 6)
    x = 0.5 * (d[2] + d[3]) - d[0]
    h = 1e-5
    f0, f1, f2, _ = oracle.secular_eval(d, z, rho, 0, x)
    fp = oracle.secular_eval(d, z, rho, 0, x + h)[0]
    fm = oracle.secular_eval(d, z, rho, 0, x - h)[0]
    assert f1 == pytest.approx((fp - fm) / (2 * h), rel=1e-6)
    assert f2 == pytest.approx((fp - 2 * f0 + fm) / h**2, rel=1e-3)


def test_secular_roots_next_to_a_pole():
    """Roots 1e-6 from a pole: each returned root satisfies f = 0 within the rounding bound of Eq. (8),
    lies within that bound of the exact root (extended precision), and the Gu-Eisenstat vectors of the
    merge stay orthogonal (pole-relative coordinates)."""
    import mpmath

    d = np.array([1.0, 0.0])  # descending
    z = np.array([1e-6, 1.0])
    rho = 1.0
    o, t, lam = _all_roots(d, z, rho)
    mp = mpmath.mp
    mp.dps = 50
    a = mp.mpf(z[0]) ** 2
    # f = 1 + a/(1 - lam) - 1/lam = 0  <=>  lam^2 - (2 + a) lam + 1 = 0
    disc = mp.sqrt((2 + a) ** 2 - 4)
    exact = [((2 + a) + disc) / 2, ((2 + a) - disc) / 2]
    for i in range(2):
        f, f1, f2, err = oracle.secular_eval(d, z, rho, int(o[i]), float(t[i]))
        assert abs(f) <= 16 * EPS * err
        # lam - d_o against the exact offset, within the backward-error bound |f|/f'
        off = exact[i] - d[o[i]]
        assert abs(float(t[i] - off)) <= 16 * EPS * err / f1
        assert np.sign(t[i]) == np.sign(float(off))
    lam2, U, _ = oracle.rank_one_eig(d, z, rho)
    assert np.linalg.norm(U.T @ U - np.eye(2)) < 4 * EPS
    M = np.diag(d) + rho * np.outer(z, z)
    assert np.linalg.norm(M @ U - U * lam2[None, :]) < 8 * EPS


@pytest.mark.parametrize("k,eps", [(2, 2.0**-6), (4, 2.0**-3), (8, 2.0**-10)])
def test_section_constants_are_result_neutral(k, eps):
    """k (Eq. (16)) and eps (Eq. (17)) change the work, not the roots."""
    rng = np.random.default_rng(7)
    d, z, rho = _random_secular(rng, 12)
    _, _, ref = _all_roots(d, z, rho)
    _, _, lam = _all_roots(d, z, rho, oracle.default_opts(k_sections=k, section_rel_eps=eps))
    assert np.allclose(lam, ref, rtol=0, atol=1e-14)


# ----------------------------------------------------------------------------- a6: Gu-Eisenstat


@pytest.mark.parametrize("K", [2, 5, 20])
def test_loewner_zhat_with_exact_roots_recovers_z(K):
    """Eq. (25): with the exact eigenvalues of D + rho z z^T, |z^_i| = |z_i| (Loewner's identity)."""
    rng = np.random.default_rng(200 + K)
    d, z, rho = _random_secular(rng, K)
    lam = np.linalg.eigvalsh(np.diag(d) + rho * np.outer(z, z))[::-1]  # LAPACK, descending
    # express each root against the nearer of its two bracketing poles
    o = np.empty(K, np.int32)
    for i in range(K):
        cands = [i] + ([i - 1] if i > 0 else [])
        o[i] = min(cands, key=lambda j: abs(lam[i] - d[j]))
    t = lam - d[o]
    zh = oracle.loewner_zhat(d, z, rho, o, t)
    assert np.allclose(zh, z, rtol=1e-8, atol=0)


def test_loewner_zhat_clustered_poles():
    """Eq. (25) when 56 poles cluster at the 1e-9 scale: the two plain products of Eq. (25) underflow
    binary64 (56 factors of ~1e-9), the quotient does not; |z^| must still equal |z| with exact roots."""
    rng = np.random.default_rng(210)
    K = 56
    d = np.sort(rng.uniform(-1e-9, 5e-9, K))[::-1].copy()
    z = rng.standard_normal(K)
    z /= np.linalg.norm(z) / np.sqrt(2.0)
    rho = 1e-9
    lam = np.linalg.eigvalsh(np.diag(d) + rho * np.outer(z, z))[::-1]
    o = np.empty(K, np.int32)
    for i in range(K):
        cands = [i] + ([i - 1] if i > 0 else [])
        o[i] = min(cands, key=lambda j: abs(lam[i] - d[j]))
    zh = oracle.loewner_zhat(d, z, rho, o, lam - d[o])
    assert np.all(np.isfinite(zh))
    assert np.allclose(zh, z, rtol=1e-6, atol=0)


# ----------------------------------------------------------------------------- a4-a6: one merge


def _check_eigpairs(M, lam, U, tol):
    """tol is absolute for M-sized quantities; orthogonality is checked against tol / max(1, |M|)."""
    n = M.shape[0]
    scale = max(1.0, np.abs(M).max())
    assert np.linalg.norm(U.T @ U - np.eye(n)) < tol / scale * max(1.0, n / 4)
    assert np.linalg.norm(M @ U - U * lam[None, :]) < tol
    assert np.allclose(lam, np.linalg.eigvalsh(M), rtol=0, atol=tol)


@pytest.mark.parametrize("case", ["generic", "zero_z", "equal_poles", "near_poles", "rho_zero", "all_equal",
                                  "rotation_small_coupling"])
def test_rank_one_eig_with_deflation(case):
    """Eq. (4) middle factor D + rho z z^T, including both kinds of deflation."""
    rng = np.random.default_rng(11)
    s = 12
    D = rng.uniform(-1, 1, s)
    z = rng.standard_normal(s)
    rho = 0.7
    if case == "zero_z":
        z[[1, 4, 5]] = 0.0
    elif case == "equal_poles":
        D[3] = D[7] = D[9]
    elif case == "near_poles":
        D[2] = D[6] + 1e-17
    elif case == "rho_zero":
        rho = 0.0
    elif case == "all_equal":
        D[:] = 0.25
    elif case == "rotation_small_coupling":
        # large rho: a coupling of 1e-12 escapes deflation (i) but its pole pair is rotated by (ii)
        # although the two poles are far apart
        rho = 1e3
        z[5] = 1e-12
    lam, U, st = oracle.rank_one_eig(D, z, rho)
    M = np.diag(D) + rho * np.outer(z, z)
    _check_eigpairs(M, lam, U, 1e-13 * s * max(1.0, np.abs(M).max()))
    assert np.all(np.diff(lam) >= 0)
    if case in ("zero_z",):
        assert st.deflated >= 3
    if case in ("equal_poles", "all_equal"):
        assert st.rotations >= 2
    if case == "rotation_small_coupling":
        assert st.rotations >= 1
    if case == "rho_zero":
        assert st.deflated == s


# ----------------------------------------------------------------------------- a2-a7 on T alone


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 15, 16, 31, 64])
def test_tridiagonal_toeplitz_closed_form(n):
    """T = tridiag(b, a, b): lam_k = a + 2b cos(k pi/(n+1)), v_k[j] ~ sin(j k pi/(n+1))."""
    a, b = 0.3, -0.45
    lam, Q, st = oracle.tridiag_eig(np.full(n, a), np.full(n - 1, b))
    k = np.arange(1, n + 1)
    ref = np.sort(a + 2 * b * np.cos(k * np.pi / (n + 1)))
    assert np.allclose(lam, ref, rtol=0, atol=1e-14 * n)
    j = np.arange(1, n + 1)
    for col in range(n):
        # eigenvalue lam[col] = a + 2b cos(kk pi/(n+1)) for the matching kk
        kk = int(np.argmin(np.abs(a + 2 * b * np.cos(k * np.pi / (n + 1)) - lam[col]))) + 1
        v = np.sin(j * kk * np.pi / (n + 1))
        v /= np.linalg.norm(v)
        assert min(np.linalg.norm(Q[:, col] - v), np.linalg.norm(Q[:, col] + v)) < 1e-12 * n


@pytest.mark.parametrize("leaf", [1, 2, 3, 4, 5, 8])
def test_tridiag_eig_leaf_size(leaf):
    """Sec. 2.2: dividing down to blocks of 1..8 rows (QL leaves from 3 rows) gives the same
    eigendecomposition."""
    rng = np.random.default_rng(12)
    for n in (21, 37, 64):
        d, e = rng.standard_normal(n), rng.standard_normal(n - 1)
        lam, Q, st = oracle.tridiag_eig(d, e, oracle.default_opts(leaf_size=leaf))
        _check_eigpairs(_tri(d, e), lam, Q, 1e-13 * n)
        assert st.not_conv == 0


# ----------------------------------------------------------------------------- a3: QL leaves


@pytest.mark.parametrize("s", [1, 2, 3, 4, 5, 6, 7, 8])
def test_tridiag_ql_against_lapack(s):
    """Implicit QL leaf: eigenpairs of random tridiagonals against LAPACK, orthogonality, ascending."""
    rng = np.random.default_rng(100 + s)
    for trial in range(20):
        d = rng.standard_normal(s) * (10.0 ** rng.integers(-3, 4))
        e = rng.standard_normal(max(s - 1, 0)) * (10.0 ** rng.integers(-3, 4))
        lam, Q, bad = oracle.tridiag_ql(d, e)
        assert bad == 0
        T = _tri(d, e)
        nrm = max(np.abs(np.linalg.eigvalsh(T)).max(), 1e-300)
        assert np.all(np.diff(lam) >= 0)
        assert np.allclose(lam, np.linalg.eigvalsh(T), rtol=0, atol=1e-14 * nrm * s)
        assert np.linalg.norm(Q.T @ Q - np.eye(s)) < 1e-14 * s
        assert np.linalg.norm(T @ Q - Q * lam[None, :]) < 1e-14 * nrm * s


def test_tridiag_ql_special_cases():
    """Split tridiagonals (zero couplings), repeated eigenvalues and the Toeplitz closed form."""
    # zero off-diagonals: diagonal entries are the eigenvalues, Q a permutation
    d = np.array([3.0, -1.0, 2.0, 0.5, 2.0])
    lam, Q, bad = oracle.tridiag_ql(d, np.zeros(4))
    assert bad == 0 and np.array_equal(lam, np.sort(d))
    assert np.allclose(np.abs(Q) @ np.ones(5), np.ones(5))
    # one interior zero coupling: two independent blocks
    d, e = np.array([1.0, 2.0, 3.0, 4.0, 5.0, 6.0]), np.array([0.5, 0.25, 0.0, 0.75, 1.0])
    lam, Q, bad = oracle.tridiag_ql(d, e)
    assert bad == 0
    _check_eigpairs(_tri(d, e), lam, Q, 1e-14 * 6 * 6)
    # Toeplitz: eigenvalues a + 2b cos(k pi/(s+1)), a double root free family
    for s in (3, 5, 8):
        a, b = 0.3, -0.7
        lam, Q, bad = oracle.tridiag_ql(np.full(s, a), np.full(s - 1, b))
        ref = np.sort(a + 2 * b * np.cos(np.arange(1, s + 1) * np.pi / (s + 1)))
        assert bad == 0 and np.allclose(lam, ref, rtol=0, atol=1e-14 * s)
    # a matrix with a repeated eigenvalue (glued identical blocks with zero coupling)
    d, e = np.array([2.0, 1.0, 2.0, 1.0]), np.array([0.5, 0.0, 0.5])
    lam, Q, bad = oracle.tridiag_ql(d, e)
    assert bad == 0
    _check_eigpairs(_tri(d, e), lam, Q, 1e-14 * 16)


@pytest.mark.parametrize("leaf", [4, 8])
def test_eigh_with_ql_leaves(leaf):
    """The whole path with QL leaves against LAPACK on covariances and gapped spectra."""
    from paper_2604_27325_gb300 import workloads as wl
    for n in (9, 16, 40, 64):
        A = wl.covariance(2, n, seed=70 + n).astype(np.float64)
        for b in range(2):
            W, V, st = oracle.eigh(A[b], oracle.default_opts(leaf_size=leaf))
            assert st.not_conv == 0
            _check_eigpairs(A[b], W, V, 1e-12 * n)


# ----------------------------------------------------------------------------- a1-a9: whole path


def _jacobi_eig(A, sweeps=60):
    """Brute-force cyclic Jacobi (textbook), independent of every oracle routine."""
    A = A.copy()
    n = A.shape[0]
    V = np.eye(n)
    for _ in range(sweeps):
        off = np.sqrt(np.sum(np.triu(A, 1) ** 2))
        if off < 1e-300:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                if A[p, q] == 0.0:
                    continue
                th = (A[q, q] - A[p, p]) / (2 * A[p, q])
                t = (1.0 if th >= 0 else -1.0) / (abs(th) + math.sqrt(th * th + 1))
                c = 1 / math.sqrt(t * t + 1)
                s = t * c
                J = np.eye(n)
                J[p, p] = J[q, q] = c
                J[p, q], J[q, p] = s, -s
                A = J.T @ A @ J
                V = V @ J
    lam = np.diag(A)
    o = np.argsort(lam, kind="stable")
    return lam[o], V[:, o]


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 8])
def test_whole_path_vs_bruteforce_jacobi(n):
    rng = np.random.default_rng(300 + n)
    for _ in range(4):
        A = _rand_sym(rng, n)
        W, V, _ = oracle.eigh(A)
        lj, Vj = _jacobi_eig(A)
        assert np.allclose(W, lj, rtol=0, atol=1e-13)
        for c in range(n):
            assert min(np.linalg.norm(V[:, c] - Vj[:, c]), np.linalg.norm(V[:, c] + Vj[:, c])) < 1e-10


@pytest.mark.parametrize("n", [1, 2, 3, 4, 7, 16, 17, 32, 48, 63, 64])
def test_whole_path_vs_lapack(n):
    """Plain definition A = V diag(W) V^T against numpy.linalg.eigh on covariance and gapped inputs."""
    A = np.concatenate([wl.covariance(4, n, seed=n), wl.known_spectrum(4, n, seed=n)[0]]).astype(np.float64)
    for M in A:
        W, V, st = oracle.eigh(M)
        nrm = max(np.abs(np.linalg.eigvalsh(M)).max(), 1e-300)
        assert np.allclose(W, np.linalg.eigvalsh(M), rtol=0, atol=1e-13 * nrm * max(n, 4))
        assert np.linalg.norm(M @ V - V * W[None, :]) <= 1e-13 * n * nrm
        assert np.linalg.norm(V.T @ V - np.eye(n)) <= 1e-13 * n
        assert st.not_conv == 0


@pytest.mark.parametrize("n", [4, 16, 64])
def test_whole_path_known_spectrum(n):
    """A = Q diag(lam) Q^T built in FP64: recovered eigenvalues equal lam."""
    rng = np.random.default_rng(400 + n)
    Q, R = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.sort(rng.uniform(-1, 1, n))
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    W, V, _ = oracle.eigh(A)
    assert np.allclose(W, lam, rtol=0, atol=1e-14 * n)


def test_whole_path_diagonal_and_sign_convention():
    """Diagonal A: W = sorted diagonal, V = permutation; every column's largest entry is positive."""
    rng = np.random.default_rng(13)
    dg = rng.uniform(-1, 1, 10)
    W, V, _ = oracle.eigh(np.diag(dg))
    assert np.array_equal(W, np.sort(dg))
    assert np.array_equal(np.abs(V), np.eye(10)[:, np.argsort(dg)])
    A = _rand_sym(rng, 12)
    W, V, _ = oracle.eigh(A)
    idx = np.argmax(np.abs(V), axis=0)
    assert np.all(V[idx, np.arange(12)] > 0)


@pytest.mark.parametrize("n", [16, 64])
@pytest.mark.parametrize("name", ["zero", "identity", "diagonal", "repeated", "rank_one", "block_diagonal", "toeplitz"])
def test_whole_path_special_cases(name, n):
    M = wl.special_cases(n)[name].astype(np.float64)
    W, V, st = oracle.eigh(M)
    _check_eigpairs(M, W, V, 1e-13 * n)
    assert st.not_conv == 0


def test_batch_driver_matches_single_and_is_thread_independent():
    A = wl.covariance(9, 12, seed=5)
    W1, V1, st1, u1 = oracle.eigh_batch_f32(A, nthreads=1)
    W4, V4, st4, u4 = oracle.eigh_batch_f32(A, nthreads=4)
    assert u1 == 1 and u4 == 4
    assert np.array_equal(W1, W4) and np.array_equal(V1, V4)
    assert st1.as_dict() == st4.as_dict()
    for b in range(9):
        W, V, _ = oracle.eigh(A[b].astype(np.float64))
        assert np.array_equal(W, W1[b]) and np.array_equal(V, V1[b])


# ----------------------------------------------------------------------------- gradient of the layer


def _gapped(rng, n, gap):
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.sort(rng.uniform(-1, 1 - (n - 1) * gap, n)) + gap * np.arange(n)
    A = (Q * lam) @ Q.T
    return 0.5 * (A + A.T)


@pytest.mark.parametrize("n", [4, 9, 32])
def test_backward_against_central_differences(n):
    """dL/dA for L = sum w_i lambda_i + <G, V> against FP64 central differences (h = 1e-6) along
    random symmetric directions (the sign convention keeps V differentiable away from ties)."""
    rng = np.random.default_rng(600 + n)
    A = _gapped(rng, n, 2e-2)
    w, G = rng.standard_normal(n), rng.standard_normal((n, n))

    def loss(M):
        W, V, _ = oracle.eigh(M)
        return w @ W + np.sum(G * V)

    W, V, _ = oracle.eigh(A)
    gA = oracle.eigh_backward(W, V, w, G)
    assert np.allclose(gA, gA.T, atol=0)
    h = 1e-6
    for _ in range(4):
        E = rng.standard_normal((n, n))
        E = 0.5 * (E + E.T)
        fd = (loss(A + h * E) - loss(A - h * E)) / (2 * h)
        assert abs(fd - np.sum(gA * E)) <= 1e-6 * max(1.0, abs(fd)) * n


def test_backward_closed_forms():
    """Only eigenvalues in the loss: gA = V diag(w) V^T; w = 1 gives d trace(A)/dA = I."""
    rng = np.random.default_rng(610)
    A = _gapped(rng, 7, 1e-2)
    W, V, _ = oracle.eigh(A)
    assert np.allclose(oracle.eigh_backward(W, V, np.ones(7), None), np.eye(7), atol=1e-13)
    w = rng.standard_normal(7)
    assert np.allclose(oracle.eigh_backward(W, V, w, None), (V * w) @ V.T, atol=1e-13)


def test_backward_masks_degenerate_pairs():
    """A repeated eigenvalue: the pair's F entry is masked (finite result), and with an eigenvalue-only
    loss the gradient is unaffected by the mask."""
    rng = np.random.default_rng(620)
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    lam = np.array([-1.0, -0.2, 0.3, 0.3, 0.8, 1.1])
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    W, V, _ = oracle.eigh(A)
    G = rng.standard_normal((6, 6))
    gA = oracle.eigh_backward(W, V, None, G, gap_eps=1e-6)
    assert np.all(np.isfinite(gA))
    w = rng.standard_normal(6)
    assert np.allclose(oracle.eigh_backward(W, V, w, None, gap_eps=1e-6), (V * w) @ V.T, atol=1e-13)
