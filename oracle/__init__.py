"""FP64 CPU oracle of the batched divide-and-conquer eigendecomposition (test infrastructure).

This package is the checker, not the product: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import it. It wraps ``bed_oracle.c`` (plain C, FP64) through
ctypes and shares no code with the CUDA library.

Each wrapper cites the stage of Song, "A Short Note on Batch-efficient Divide-and-Conquer Algorithm
for EigenDecomposition" that the C function follows; the C file lists the stages and readings.
Parity unpinned: iteration counts and the section constants (k of Eq. (16), eps of Eq. (17)).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bed_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


class Opts(C.Structure):
    """Constants the paper leaves unnamed (mirror of ``orc_opts``)."""

    _fields_ = [
        ("k_sections", C.c_int),
        ("section_rel_eps", C.c_double),
        ("max_section_iters", C.c_int),
        ("max_halley_iters", C.c_int),
        ("stop_c", C.c_double),
        ("deflate_c", C.c_double),
        ("leaf_size", C.c_int),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("roots", C.c_int64),
        ("iters", C.c_int64),
        ("deflated", C.c_int64),
        ("rotations", C.c_int64),
        ("not_conv", C.c_int64),
    ]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile ``bed_oracle.c`` with gcc into ``oracle/_build/liboracle.so``."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm", "-lpthread"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # BED_ORACLE_LIB points the wrappers at another build of the oracle (the mutation tests
            # load copies with planted mistakes this way).
            L = C.CDLL(os.environ.get("BED_ORACLE_LIB") or build())
            dp = C.POINTER(C.c_double)
            ip = C.POINTER(C.c_int)
            L.orc_default_opts.argtypes = [C.POINTER(Opts)]
            L.orc_tridiagonalize.argtypes = [C.c_int, dp, dp, dp, dp, dp, dp]
            L.orc_tear.argtypes = [C.c_int, dp, dp, C.c_int, dp, dp, dp, dp]
            L.orc_eig2.argtypes = [C.c_double, C.c_double, C.c_double, dp, dp]
            L.orc_secular_eval.argtypes = [C.c_int, dp, dp, C.c_double, C.c_int, C.c_double, dp, dp, dp, dp]
            L.orc_secular_root.argtypes = [C.c_int, dp, dp, C.c_double, C.c_double, C.c_int,
                                           C.POINTER(Opts), ip, dp, C.POINTER(Stats)]
            L.orc_loewner_zhat.argtypes = [C.c_int, dp, dp, C.c_double, ip, dp, dp]
            L.orc_rank_one_eig.argtypes = [C.c_int, dp, dp, C.c_double, C.POINTER(Opts), dp, dp,
                                           C.POINTER(Stats)]
            L.orc_tridiag_eig.argtypes = [C.c_int, dp, dp, C.POINTER(Opts), dp, dp, C.POINTER(Stats)]
            L.orc_tridiag_ql.argtypes = [C.c_int, dp, dp, dp, dp]
            L.orc_tridiag_ql.restype = C.c_int
            L.orc_eigh.argtypes = [C.c_int, dp, C.POINTER(Opts), dp, dp, C.POINTER(Stats)]
            L.orc_eigh_batch_f32.argtypes = [C.c_int64, C.c_int, C.POINTER(C.c_float), C.POINTER(Opts),
                                             dp, dp, C.c_int, C.POINTER(Stats)]
            L.orc_eigh_batch_f32.restype = C.c_int
            L.orc_eigh_backward.argtypes = [C.c_int, dp, dp, dp, dp, C.c_double, dp]
            L.orc_eigh_backward.restype = None
            _lib = L
        return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def default_opts(**over) -> Opts:
    o = Opts()
    lib().orc_default_opts(C.byref(o))
    for k, v in over.items():
        setattr(o, k, v)
    return o


def tridiagonalize(A):
    """a1: A = H T H^T (Householder; textbook reduction). Returns d, e, H, reflectors (rows), taus."""
    A = _f64(A)
    n = A.shape[0]
    d, e = np.zeros(n), np.zeros(max(n - 1, 1))
    vk, taus, H = np.zeros((n, n)), np.zeros(max(n - 1, 1)), np.zeros((n, n))
    lib().orc_tridiagonalize(n, _dp(A), _dp(d), _dp(e), _dp(vk), _dp(taus), _dp(H))
    return d, e[: max(n - 1, 0)], H, vk, taus[: max(n - 1, 0)]


def tear(d, e, m):
    """a2: Eq. (2)-(3); returns (d1, d2, rho, sigma)."""
    d, e = _f64(d), _f64(e)
    s = d.shape[0]
    d1, d2 = np.zeros(m), np.zeros(s - m)
    rho, sig = C.c_double(), C.c_double()
    lib().orc_tear(s, _dp(d), _dp(e), m, _dp(d1), _dp(d2), C.byref(rho), C.byref(sig))
    return d1, d2, rho.value, sig.value


def eig2(a, b, c):
    """a3: 2x2 leaf by one Jacobi rotation (Sec. 2.2)."""
    lam, Q = np.zeros(2), np.zeros(4)
    lib().orc_eig2(a, b, c, _dp(lam), _dp(Q))
    return lam, Q.reshape(2, 2)


def tridiag_ql(d, e):
    """a3 for larger leaves: implicit QL with Wilkinson shifts. Returns (lam ascending, Q, capped)."""
    d, e = _f64(d), _f64(e)
    s = d.shape[0]
    e = np.concatenate([e, [0.0]])
    lam, Q = np.zeros(s), np.zeros((s, s))
    bad = lib().orc_tridiag_ql(s, _dp(d), _dp(e), _dp(lam), _dp(Q))
    return lam, Q, bad


def secular_eval(d, z, rho, o, tau):
    """Eq. (8), (18), (21) at lambda = d[o] + tau; returns f, f', f'', error scale."""
    d, z = _f64(d), _f64(z)
    out = [C.c_double() for _ in range(4)]
    lib().orc_secular_eval(d.shape[0], _dp(d), _dp(z), rho, o, tau, *[C.byref(x) for x in out])
    return tuple(x.value for x in out)


def secular_root(d_desc, z, rho, upper0, i, opts=None):
    """a5: root i of Eq. (8), poles DESCENDING (Eq. (9)); returns (origin, tau, stats)."""
    d, z = _f64(d_desc), _f64(z)
    o, t, st = C.c_int(), C.c_double(), Stats()
    lib().orc_secular_root(d.shape[0], _dp(d), _dp(z), rho, upper0, i,
                           C.byref(opts) if opts is not None else None, C.byref(o), C.byref(t), C.byref(st))
    return o.value, t.value, st


def loewner_zhat(d_desc, z, rho, origin, tau):
    """a6: Eq. (25) from roots given as (origin pole, offset) pairs."""
    d, z, tau = _f64(d_desc), _f64(z), _f64(tau)
    origin = np.ascontiguousarray(origin, dtype=np.int32)
    zh = np.zeros_like(d)
    lib().orc_loewner_zhat(d.shape[0], _dp(d), _dp(z), rho, origin.ctypes.data_as(C.POINTER(C.c_int)),
                           _dp(tau), _dp(zh))
    return zh


def rank_one_eig(D, z, rho, opts=None):
    """a4-a6: eigendecomposition of D + rho z z^T (Eq. (4) middle factor) with deflation."""
    D, z = _f64(D), _f64(z)
    s = D.shape[0]
    lam, U, st = np.zeros(s), np.zeros((s, s)), Stats()
    lib().orc_rank_one_eig(s, _dp(D), _dp(z), rho, C.byref(opts) if opts is not None else None,
                           _dp(lam), _dp(U), C.byref(st))
    return lam, U, st


def tridiag_eig(d, e, opts=None):
    """a2-a7: divide and conquer on the tridiagonal (d, e)."""
    d, e = _f64(d), _f64(e)
    s = d.shape[0]
    e = np.concatenate([e, [0.0]])
    lam, Q, st = np.zeros(s), np.zeros((s, s)), Stats()
    lib().orc_tridiag_eig(s, _dp(d), _dp(e), C.byref(opts) if opts is not None else None,
                          _dp(lam), _dp(Q), C.byref(st))
    return lam, Q, st


def eigh(A, opts=None):
    """a1-a9 for one FP64 matrix (lower triangle read): (W ascending, V columns, stats)."""
    A = _f64(A)
    n = A.shape[0]
    W, V, st = np.zeros(n), np.zeros((n, n)), Stats()
    lib().orc_eigh(n, _dp(A), C.byref(opts) if opts is not None else None, _dp(W), _dp(V), C.byref(st))
    return W, V, st


def eigh_batch_f32(A, nthreads: int | None = None, opts=None):
    """Batched a1-a9: A float32 [b, n, n] upcast exactly to FP64; returns (W, V, stats, threads)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    b, n, _ = A.shape
    W, V, st = np.zeros((b, n)), np.zeros((b, n, n)), Stats()
    if b == 0:
        return W, V, st, 0
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    used = lib().orc_eigh_batch_f32(b, n, A.ctypes.data_as(C.POINTER(C.c_float)),
                                    C.byref(opts) if opts is not None else None,
                                    _dp(W), _dp(V), int(nthreads), C.byref(st))
    return W, V, st, used


def eigh_backward(W, V, gW, gV, gap_eps: float = 0.0):
    """Gradient dL/dA (symmetric) from the eigendecomposition's W, V and the loss gradients gW, gV
    (either may be None). FP64; one matrix."""
    W, V = _f64(W), _f64(V)
    n = W.shape[0]
    gA = np.zeros((n, n))
    gW = _f64(gW) if gW is not None else None
    gV = _f64(gV) if gV is not None else None
    lib().orc_eigh_backward(n, _dp(W), _dp(V), _dp(gW) if gW is not None else None,
                            _dp(gV) if gV is not None else None, gap_eps, _dp(gA))
    return gA
