"""Thin ctypes binding of the C ABI in ``include/bed.h`` (argument marshalling only).

Every function named ``bed_*`` here calls the C function of the same name in ``libbed.so``; the
convenience wrapper :func:`batched_eigh` allocates outputs with PyTorch (device memory and streams
only) and calls :func:`bed_eigh_f32`. There is no CPU fallback: without a GPU or without the built
library the calls raise.
"""
from __future__ import annotations

import ctypes as C
import threading

import torch

from . import build as _build

BED_OK = 0
BED_ERR_INVALID_ARG = 1
BED_ERR_UNSUPPORTED_N = 2
BED_ERR_CUDA = 3

BED_INFO_OK = 0
BED_INFO_NOT_CONVERGED = 1
BED_INFO_NONFINITE = 2
BED_INFO_TIMEOUT = 4


class bed_params(C.Structure):
    _fields_ = [
        ("leaf_size", C.c_int),
        ("k_multisection", C.c_int),
        ("max_section_iters", C.c_int),
        ("max_halley_iters", C.c_int),
        ("section_rel_eps", C.c_float),
        ("stop_c", C.c_float),
        ("deflation_tol_scale", C.c_float),
        ("threads_per_matrix", C.c_int),
        ("retire_by_vote", C.c_int),
    ]


class bed_counters(C.Structure):
    _fields_ = [
        ("matrices", C.c_ulonglong),
        ("roots", C.c_ulonglong),
        ("evals", C.c_ulonglong),
        ("deflated", C.c_ulonglong),
    ]


EXPORTED = [
    "bed_default_params",
    "bed_eigh_f32",
    "bed_eigh_f32_counted",
    "bed_max_n",
    "bed_status_string",
    "bed_last_cuda_error",
    "bed_plan_describe",
]

_lock = threading.Lock()
_lib = None


def lib() -> C.CDLL:
    """Load ``libbed.so`` (building it with nvcc first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(_build.build())
            vp = C.c_void_p
            L.bed_default_params.argtypes = [C.POINTER(bed_params)]
            L.bed_default_params.restype = None
            L.bed_eigh_f32.argtypes = [vp, vp, vp, vp, C.c_int64, C.c_int, C.POINTER(bed_params), vp]
            L.bed_eigh_f32.restype = C.c_int
            L.bed_eigh_f32_counted.argtypes = [vp, vp, vp, vp, C.c_int64, C.c_int, C.POINTER(bed_params), vp, vp]
            L.bed_eigh_f32_counted.restype = C.c_int
            L.bed_max_n.argtypes = []
            L.bed_max_n.restype = C.c_int
            L.bed_status_string.argtypes = [C.c_int]
            L.bed_status_string.restype = C.c_char_p
            L.bed_last_cuda_error.argtypes = []
            L.bed_last_cuda_error.restype = C.c_char_p
            L.bed_plan_describe.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
            L.bed_plan_describe.restype = C.c_int
            _lib = L
        return _lib


# ------------------------------------------------------------------ same-name wrappers of the C ABI


def bed_default_params() -> bed_params:
    p = bed_params()
    lib().bed_default_params(C.byref(p))
    return p


def bed_eigh_f32(A_ptr: int, W_ptr: int, V_ptr: int, info_ptr: int | None, batch: int, n: int,
                 params: bed_params | None = None, stream: int = 0) -> int:
    """Raw call: device pointers as integers; returns the bed_status code."""
    return lib().bed_eigh_f32(A_ptr, W_ptr, V_ptr, info_ptr, batch, n,
                              C.byref(params) if params is not None else None, stream)


def bed_eigh_f32_counted(A_ptr: int, W_ptr: int, V_ptr: int, info_ptr: int | None, batch: int, n: int,
                         params: bed_params | None, counters_ptr: int, stream: int = 0) -> int:
    return lib().bed_eigh_f32_counted(A_ptr, W_ptr, V_ptr, info_ptr, batch, n,
                                      C.byref(params) if params is not None else None, counters_ptr, stream)


def bed_max_n() -> int:
    return lib().bed_max_n()


def bed_status_string(s: int) -> str:
    return lib().bed_status_string(s).decode()


def bed_last_cuda_error() -> str:
    return lib().bed_last_cuda_error().decode()


def bed_plan_describe(n: int, leaf_size: int = 2):
    """Host-side divide tree: list of (lo, mid, hi, level) merges, deepest level first."""
    merges = (C.c_int * (3 * 64))()
    levels = (C.c_int * 64)()
    k = lib().bed_plan_describe(n, leaf_size, merges, levels)
    if k < 0:
        raise ValueError(f"unsupported n={n} / leaf_size={leaf_size}")
    return [(merges[3 * i], merges[3 * i + 1], merges[3 * i + 2], levels[i]) for i in range(k)]


# ------------------------------------------------------------------ convenience wrapper


class BedError(RuntimeError):
    pass


def _check(status: int):
    if status != BED_OK:
        msg = bed_status_string(status)
        if status == BED_ERR_CUDA:
            msg += ": " + bed_last_cuda_error()
        raise BedError(msg)


def make_params(**kw) -> bed_params:
    p = bed_default_params()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def batched_eigh(A: torch.Tensor, params: bed_params | None = None, check: bool = False,
                 return_info: bool = False, counters: torch.Tensor | None = None):
    """Eigendecomposition of a batch of symmetric FP32 matrices ``A[..., n, n]`` (lower triangle read).

    Returns ``(W, V)`` with W ascending and the eigenvectors in the columns of V (torch.linalg.eigh
    conventions); with ``return_info`` also the int32 per-matrix status flags. A CUDA tensor is solved
    in place on the current stream; a CPU tensor is copied to the current CUDA device through pinned
    memory, solved, and the results are copied back (the end-to-end path). ``check=True`` synchronizes
    and raises if any matrix reports a non-zero info.
    """
    if A.dtype != torch.float32:
        raise TypeError("batched_eigh expects float32 matrices")
    if A.dim() < 2 or A.shape[-1] != A.shape[-2]:
        raise ValueError("batched_eigh expects [..., n, n]")
    if not torch.cuda.is_available():
        raise BedError("batched_eigh needs a CUDA device; there is no CPU path")
    host = not A.is_cuda
    lead = A.shape[:-2]
    n = A.shape[-1]
    Ad = A.reshape(-1, n, n)
    if host:
        Ad = Ad.contiguous().pin_memory().to("cuda", non_blocking=True)
    else:
        Ad = Ad.contiguous()
    b = Ad.shape[0]
    dev = Ad.device
    W = torch.empty((b, n), dtype=torch.float32, device=dev)
    V = torch.empty((b, n, n), dtype=torch.float32, device=dev)
    info = torch.empty((b,), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    if counters is not None:
        st = bed_eigh_f32_counted(Ad.data_ptr(), W.data_ptr(), V.data_ptr(), info.data_ptr(), b, n, params,
                                  counters.data_ptr(), stream)
    else:
        st = bed_eigh_f32(Ad.data_ptr(), W.data_ptr(), V.data_ptr(), info.data_ptr(), b, n, params, stream)
    _check(st)
    if host:
        Wh = torch.empty((b, n), dtype=torch.float32, pin_memory=True)
        Vh = torch.empty((b, n, n), dtype=torch.float32, pin_memory=True)
        Ih = torch.empty((b,), dtype=torch.int32, pin_memory=True)
        Wh.copy_(W, non_blocking=True)
        Vh.copy_(V, non_blocking=True)
        Ih.copy_(info, non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()
        W, V, info = Wh, Vh, Ih
    if check:
        bad = int((info != 0).sum().item())
        if bad:
            raise BedError(f"{bad} matrices reported a non-zero info")
    W = W.reshape(*lead, n)
    V = V.reshape(*lead, n, n)
    info = info.reshape(lead)
    return (W, V, info) if return_info else (W, V)
