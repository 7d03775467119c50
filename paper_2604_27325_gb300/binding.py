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
BED_ERR_TOO_LARGE = 4
BED_ERR_TIMEOUT = 5
BED_NOALLOC_MAX_COUNT = 65536

BED_INFO_OK = 0
BED_INFO_NOT_CONVERGED = 1
BED_INFO_NONFINITE = 2
BED_INFO_TIMEOUT = 4
BED_INFO_BAD_N = 8


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
        ("merge_tensor_cores", C.c_int),
        ("stage_wait_us", C.c_int),
        ("matrices_per_cta", C.c_int),
        ("n_bisect_first", C.c_int),
    ]


class bed_counters(C.Structure):
    _fields_ = [
        ("matrices", C.c_ulonglong),
        ("roots", C.c_ulonglong),
        ("evals", C.c_ulonglong),
        ("deflated", C.c_ulonglong),
    ]


class bed_ragged_tuning(C.Structure):
    _fields_ = [("team", C.c_ubyte * 65), ("leaf", C.c_ubyte * 65)]


class bed_server_config(C.Structure):
    _fields_ = [("device_budget_bytes", C.c_size_t), ("host_result_bytes", C.c_size_t), ("streams", C.c_int),
                ("max_launch_matrices", C.c_int), ("mode", C.c_int), ("zero_copy", C.c_int)]


class bed_server_stats(C.Structure):
    _fields_ = [("requests", C.c_int64), ("matrices", C.c_int64), ("launches", C.c_int64),
                ("peak_device_bytes", C.c_int64), ("p50_s", C.c_double), ("p99_s", C.c_double),
                ("mean_s", C.c_double), ("max_s", C.c_double), ("span_s", C.c_double),
                ("max_admit_wait_s", C.c_double), ("max_enqueue_s", C.c_double), ("max_inflight_s", C.c_double)]


EXPORTED = [
    "bed_default_params",
    "bed_eigh_f32",
    "bed_eigh_f32_counted",
    "bed_eigh_f32_host",
    "bed_eigh_f32_pinned",
    "bed_eigh_many_f32_pinned",
    "bed_eigh_backward_f32",
    "bed_eigh_ragged_f32",
    "bed_eigh_ragged_f32_noalloc",
    "bed_eigh_ragged_workspace_size",
    "bed_ragged_default_tuning",
    "bed_server_default_config",
    "bed_server_create",
    "bed_server_submit",
    "bed_server_wait",
    "bed_server_release",
    "bed_server_get_stats",
    "bed_server_reset_stats",
    "bed_server_destroy",
    "bed_fma_peak_chains",
    "bed_fma_peak_launch",
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
            L.bed_eigh_f32_host.argtypes = [vp, vp, vp, vp, C.c_int64, C.c_int, C.POINTER(bed_params), vp, vp, vp,
                                            vp, C.c_int, vp, vp]
            L.bed_eigh_f32_host.restype = C.c_int
            L.bed_eigh_f32_pinned.argtypes = [vp, vp, vp, vp, C.c_int64, C.c_int, C.POINTER(bed_params), vp]
            L.bed_eigh_f32_pinned.restype = C.c_int
            L.bed_eigh_many_f32_pinned.argtypes = [C.c_int, vp, vp, vp, vp, vp, vp, C.POINTER(bed_params), vp, vp,
                                                   C.c_int]
            L.bed_eigh_many_f32_pinned.restype = C.c_int
            L.bed_fma_peak_chains.argtypes = []
            L.bed_fma_peak_chains.restype = C.c_int
            L.bed_fma_peak_launch.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp]
            L.bed_fma_peak_launch.restype = C.c_int
            L.bed_max_n.argtypes = []
            L.bed_max_n.restype = C.c_int
            L.bed_status_string.argtypes = [C.c_int]
            L.bed_status_string.restype = C.c_char_p
            L.bed_last_cuda_error.argtypes = []
            L.bed_last_cuda_error.restype = C.c_char_p
            L.bed_plan_describe.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
            L.bed_plan_describe.restype = C.c_int
            L.bed_eigh_backward_f32.argtypes = [vp, vp, vp, vp, vp, C.c_int64, C.c_int, C.c_float, vp]
            L.bed_eigh_backward_f32.restype = C.c_int
            L.bed_server_default_config.argtypes = [C.POINTER(bed_server_config)]
            L.bed_server_default_config.restype = None
            L.bed_server_create.argtypes = [C.POINTER(bed_server_config), C.POINTER(bed_params),
                                            C.POINTER(bed_ragged_tuning), C.POINTER(vp)]
            L.bed_server_create.restype = C.c_int
            L.bed_server_submit.argtypes = [vp, vp, C.c_int32, C.c_int32, C.POINTER(C.c_int64)]
            L.bed_server_submit.restype = C.c_int
            L.bed_server_wait.argtypes = [vp, C.c_int64, C.c_double, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp)]
            L.bed_server_wait.restype = C.c_int
            L.bed_server_release.argtypes = [vp, C.c_int64]
            L.bed_server_release.restype = C.c_int
            L.bed_server_get_stats.argtypes = [vp, C.POINTER(bed_server_stats)]
            L.bed_server_get_stats.restype = C.c_int
            L.bed_server_reset_stats.argtypes = [vp]
            L.bed_server_reset_stats.restype = C.c_int
            L.bed_server_destroy.argtypes = [vp]
            L.bed_server_destroy.restype = None
            L.bed_ragged_default_tuning.argtypes = [C.POINTER(bed_ragged_tuning)]
            L.bed_ragged_default_tuning.restype = None
            L.bed_eigh_ragged_workspace_size.argtypes = [C.c_int64]
            L.bed_eigh_ragged_workspace_size.restype = C.c_size_t
            L.bed_eigh_ragged_f32.argtypes = [vp, vp, vp, C.c_int64, vp, vp, vp, vp, C.POINTER(bed_params),
                                              C.POINTER(bed_ragged_tuning), vp, C.c_size_t, vp, vp]
            L.bed_eigh_ragged_f32.restype = C.c_int
            L.bed_eigh_ragged_f32_noalloc.argtypes = [vp, vp, vp, C.c_int64, vp, vp, vp, vp, C.POINTER(bed_params),
                                                      C.POINTER(bed_ragged_tuning), vp, vp]
            L.bed_eigh_ragged_f32_noalloc.restype = C.c_int
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


def bed_eigh_f32_pinned(A_host: int, W_host: int, V_host: int, info_host: int | None, batch: int, n: int,
                        params: bed_params | None = None, stream: int = 0) -> int:
    return lib().bed_eigh_f32_pinned(A_host, W_host, V_host, info_host, batch, n,
                                     C.byref(params) if params is not None else None, stream)


def bed_eigh_many_f32_pinned(ns, batches, A_host, W_host, V_host, info_host, params: bed_params | None,
                             origin: int, side) -> int:
    """Sequences of sizes, counts and host pointers (ints; info_host None or a sequence with None entries)."""
    k = len(ns)
    P = C.c_void_p * k
    infos = None if info_host is None else P(*[p or None for p in info_host])
    return lib().bed_eigh_many_f32_pinned(k, (C.c_int * k)(*ns), (C.c_int64 * k)(*batches), P(*A_host), P(*W_host),
                                          P(*V_host), infos, C.byref(params) if params is not None else None, origin,
                                          (C.c_void_p * len(side))(*side), len(side))


def bed_eigh_f32_host(A_host: int, W_host: int, V_host: int, info_host: int | None, batch: int, n: int,
                      params: bed_params | None, A_dev: int, W_dev: int, V_dev: int, info_dev: int | None,
                      chunks: int = 0, s0: int = 0, s1: int = 0) -> int:
    return lib().bed_eigh_f32_host(A_host, W_host, V_host, info_host, batch, n,
                                   C.byref(params) if params is not None else None, A_dev, W_dev, V_dev, info_dev,
                                   chunks, s0, s1)


def bed_eigh_f32_counted(A_ptr: int, W_ptr: int, V_ptr: int, info_ptr: int | None, batch: int, n: int,
                         params: bed_params | None, counters_ptr: int, stream: int = 0) -> int:
    return lib().bed_eigh_f32_counted(A_ptr, W_ptr, V_ptr, info_ptr, batch, n,
                                      C.byref(params) if params is not None else None, counters_ptr, stream)


def bed_eigh_backward_f32(W_ptr: int, V_ptr: int, gW_ptr: int | None, gV_ptr: int | None, gA_ptr: int, batch: int,
                          n: int, gap_eps: float = 0.0, stream: int = 0) -> int:
    """Raw call of the backward kernel: device pointers as integers; returns the bed_status code."""
    return lib().bed_eigh_backward_f32(W_ptr, V_ptr, gW_ptr, gV_ptr, gA_ptr, batch, n, gap_eps, stream)


def bed_ragged_default_tuning() -> bed_ragged_tuning:
    t = bed_ragged_tuning()
    lib().bed_ragged_default_tuning(C.byref(t))
    return t


def bed_eigh_ragged_workspace_size(count: int) -> int:
    return int(lib().bed_eigh_ragged_workspace_size(count))


def bed_eigh_ragged_f32(A_ptr: int, offsets_ptr: int, ns_ptr: int, count: int, W_ptr: int, w_offsets_ptr: int,
                        V_ptr: int, info_ptr: int | None, params: bed_params | None, tuning: bed_ragged_tuning | None,
                        workspace_ptr: int, workspace_bytes: int, counters_ptr: int | None = None,
                        stream: int = 0) -> int:
    """Raw call: device pointers as integers; returns the bed_status code."""
    return lib().bed_eigh_ragged_f32(A_ptr, offsets_ptr, ns_ptr, count, W_ptr, w_offsets_ptr, V_ptr, info_ptr,
                                     C.byref(params) if params is not None else None,
                                     C.byref(tuning) if tuning is not None else None,
                                     workspace_ptr, workspace_bytes, counters_ptr, stream)


def bed_eigh_ragged_f32_noalloc(A_ptr: int, offsets_ptr: int, ns_ptr: int, count: int, W_ptr: int,
                                w_offsets_ptr: int, V_ptr: int, info_ptr: int | None, params: bed_params | None,
                                tuning: bed_ragged_tuning | None, counters_ptr: int | None = None,
                                stream: int = 0) -> int:
    """Raw call of the workspace-free ragged entry point (for callers that cannot allocate device
    memory): at most BED_NOALLOC_MAX_COUNT matrices; returns the bed_status code."""
    return lib().bed_eigh_ragged_f32_noalloc(A_ptr, offsets_ptr, ns_ptr, count, W_ptr, w_offsets_ptr, V_ptr,
                                             info_ptr, C.byref(params) if params is not None else None,
                                             C.byref(tuning) if tuning is not None else None, counters_ptr, stream)


def bed_server_default_config() -> bed_server_config:
    c = bed_server_config()
    lib().bed_server_default_config(C.byref(c))
    return c


def bed_server_create(cfg: bed_server_config | None = None, params: bed_params | None = None,
                      tuning: bed_ragged_tuning | None = None):
    h = C.c_void_p()
    st = lib().bed_server_create(C.byref(cfg) if cfg is not None else None,
                                 C.byref(params) if params is not None else None,
                                 C.byref(tuning) if tuning is not None else None, C.byref(h))
    return st, h


def bed_server_submit(h, A_ptr: int, b: int, n: int):
    rid = C.c_int64()
    st = lib().bed_server_submit(h, A_ptr, b, n, C.byref(rid))
    return st, rid.value


def bed_server_wait(h, rid: int, timeout_s: float = -1.0):
    W, V, I = C.c_void_p(), C.c_void_p(), C.c_void_p()
    st = lib().bed_server_wait(h, rid, timeout_s, C.byref(W), C.byref(V), C.byref(I))
    return st, W.value, V.value, I.value


def bed_server_release(h, rid: int) -> int:
    return lib().bed_server_release(h, rid)


def bed_server_get_stats(h) -> bed_server_stats:
    out = bed_server_stats()
    _check(lib().bed_server_get_stats(h, C.byref(out)))
    return out


def bed_server_reset_stats(h) -> int:
    return lib().bed_server_reset_stats(h)


def bed_server_destroy(h) -> None:
    lib().bed_server_destroy(h)


def bed_max_n() -> int:
    return lib().bed_max_n()


def bed_fma_peak_chains() -> int:
    return lib().bed_fma_peak_chains()


def bed_fma_peak_launch(out, blocks: int, threads: int, iters: int, stream=None) -> int:
    return lib().bed_fma_peak_launch(out, blocks, threads, iters, stream)


def fp32_fma_peak(device=None, reps: int = 5, iters: int = 200000) -> dict:
    """Measured FP32 FMA throughput of the device (TFLOP/s, best of ``reps`` CUDA-event-timed launches
    of the FMA-chain probe at full occupancy: 8 blocks of 256 threads per SM)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads = 8 * sms, 256
    out = torch.empty(blocks * threads, dtype=torch.float32, device=dev)
    s = torch.cuda.current_stream(dev)
    _check(bed_fma_peak_launch(out.data_ptr(), blocks, threads, 1000, s.cuda_stream))
    best = 0.0
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        _check(bed_fma_peak_launch(out.data_ptr(), blocks, threads, iters, s.cuda_stream))
        e1.record(s)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        flops = 2.0 * bed_fma_peak_chains() * iters * blocks * threads
        best = max(best, flops / (ms / 1e3) / 1e12)
    return {"tflops": best, "blocks": blocks, "threads": threads, "iters": iters, "chains": bed_fma_peak_chains()}


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


def concurrent_params(params: bed_params | None, n: int, count: int) -> bed_params | None:
    """The parameters a batch of size n gets when ``count`` batches run side by side (the rule of
    bed_eigh_many_f32_pinned): with the team shape left automatic and count > 1, sizes 17..32 run
    64-thread teams, half the registers of the automatic 128-thread team, so that more of them fit beside
    the larger sizes' blocks."""
    if count > 1 and 16 < n <= 32 and (params is None or params.threads_per_matrix == 0):
        q = bed_params.from_buffer_copy(params if params is not None else bed_default_params())
        q.threads_per_matrix = 64
        return q
    return params


def team_threads(n: int, params: bed_params | None = None) -> int:
    """Threads per matrix of a uniform launch of size n with these parameters (the rule bed.h states for
    threads_per_matrix: automatic 4 nmax threads, 128 for nmax = 64 without the tensor-core merges)."""
    p = params if params is not None else bed_default_params()
    if p.threads_per_matrix:
        return int(p.threads_per_matrix)
    nmax = next(m for m in (16, 32, 48, 64) if m >= n)
    return 128 if (nmax == 64 and not p.merge_tensor_cores) else 4 * nmax


def batched_eigh(A: torch.Tensor, params: bed_params | None = None, check: bool = False,
                 return_info: bool = False, counters: torch.Tensor | None = None):
    """Eigendecomposition of a batch of symmetric FP32 matrices ``A[..., n, n]`` (lower triangle read).

    Returns ``(W, V)`` with W ascending and the eigenvectors in the columns of V (torch.linalg.eigh
    conventions); with ``return_info`` also the int32 per-matrix status flags. A CUDA tensor is solved
    in place on the current stream; a CPU tensor is solved from page-locked host memory by the
    zero-copy entry point (the kernel reads it and writes the results to host memory; with
    ``counters``, which live on the device, it is copied to the device and back instead).
    ``check=True`` synchronizes and raises if any matrix reports a non-zero info.
    """
    if not A.is_cuda and counters is None and A.dtype == torch.float32:
        return batched_eigh_many([A], params, check, return_info)[0]
    out = _eigh_enqueue(A, params, counters)
    if out[3]:
        torch.cuda.current_stream(out[0].device if out[0].is_cuda else None).synchronize()
    return _eigh_finish(out, check, return_info)


def _eigh_enqueue(A: torch.Tensor, params, counters):
    """Enqueues the solve of one uniform batch on the current stream; for a CPU tensor also the copies to
    and from the device (results land in pinned host tensors once the stream reaches them).
    Returns (W, V, info, host, lead, n)."""
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
        W, V, info = Wh, Vh, Ih
    return W, V, info, host, lead, n


def _eigh_finish(out, check: bool, return_info: bool):
    W, V, info, host, lead, n = out
    if check:
        bad = int((info != 0).sum().item())
        if bad:
            raise BedError(f"{bad} matrices reported a non-zero info")
    W = W.reshape(*lead, n)
    V = V.reshape(*lead, n, n)
    info = info.reshape(lead)
    return (W, V, info) if return_info else (W, V)


class RaggedBatch:
    """Device-resident packed batch of matrices of mixed size (the ragged entry point's layout).

    Matrices are packed back to back (each starting on a 16-byte boundary, so that even sizes can be
    staged by bulk copy); outputs and the workspace are allocated once with PyTorch and reused by every
    :meth:`solve`, which makes the call capturable into a CUDA graph (:meth:`capture`, :meth:`replay`).
    """

    def __init__(self, ns, device="cuda", params: bed_params | None = None, tuning: bed_ragged_tuning | None = None):
        self.ns = [int(n) for n in ns]
        self.count = len(self.ns)
        off, woff = [], []
        a = w = 0
        for n in self.ns:
            off.append(a)
            woff.append(w)
            a += (n * n + 3) // 4 * 4
            w += n
        self.offsets_list, self.woffsets_list = off, woff
        self.device = torch.device(device)
        self.A = torch.zeros(max(a, 4), dtype=torch.float32, device=self.device)
        self.V = torch.zeros(max(a, 4), dtype=torch.float32, device=self.device)
        self.W = torch.zeros(max(w, 1), dtype=torch.float32, device=self.device)
        self.info = torch.zeros(max(self.count, 1), dtype=torch.int32, device=self.device)
        self.offsets = torch.tensor(off or [0], dtype=torch.int64, device=self.device)
        self.w_offsets = torch.tensor(woff or [0], dtype=torch.int64, device=self.device)
        self.ns_dev = torch.tensor(self.ns or [1], dtype=torch.int32, device=self.device)
        self.ws_bytes = bed_eigh_ragged_workspace_size(self.count)
        self.workspace = torch.zeros(max(self.ws_bytes // 4, 4), dtype=torch.int32, device=self.device)
        self.params = params
        self.tuning = tuning
        self.graph = None

    def load(self, mats):
        """Copy a list of n x n matrices (numpy or torch, any device) into the packed input."""
        for k, M in enumerate(mats):
            n = self.ns[k]
            t = torch.as_tensor(M, dtype=torch.float32).reshape(-1)
            self.A[self.offsets_list[k]: self.offsets_list[k] + n * n].copy_(t, non_blocking=True)
        return self

    def solve(self, counters: torch.Tensor | None = None, stream=None):
        s = (stream or torch.cuda.current_stream(self.device)).cuda_stream
        st = bed_eigh_ragged_f32(self.A.data_ptr(), self.offsets.data_ptr(), self.ns_dev.data_ptr(), self.count,
                                 self.W.data_ptr(), self.w_offsets.data_ptr(), self.V.data_ptr(),
                                 self.info.data_ptr(), self.params, self.tuning, self.workspace.data_ptr(),
                                 self.ws_bytes, counters.data_ptr() if counters is not None else None, s)
        _check(st)
        return self

    def capture(self):
        """Record one solve into a CUDA graph (the first, setup-performing call is made beforehand)."""
        self.solve()
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            g.capture_begin()
            self.solve(stream=s)
            g.capture_end()
        torch.cuda.current_stream(self.device).wait_stream(s)
        self.graph = g
        return self

    def replay(self):
        self.graph.replay()
        return self

    def results(self):
        """List of (W, V) views, V with eigenvectors in columns."""
        out = []
        for k, n in enumerate(self.ns):
            o, w = self.offsets_list[k], self.woffsets_list[k]
            out.append((self.W[w: w + n], self.V[o: o + n * n].view(n, n)))
        return out


_side_streams: dict = {}


def _streams(dev: torch.device, k: int):
    lst = _side_streams.setdefault(dev.index, [])
    while len(lst) < k:
        lst.append(torch.cuda.Stream(dev))
    return lst[:k]


def batched_eigh_many(mats, params: bed_params | None = None, check: bool = False,
                      return_info: bool = False, host_chunks: int = 0):
    """Eigendecompositions of several uniform batches: a list of FP32 tensors ``[..., n_i, n_i]``, all on
    the CPU or all on one CUDA device.

    Each batch gets one launch on its own stream, forked from the current stream and joined back to it,
    so that batches of different n run side by side on the GPU instead of one after another; with the
    team shape left automatic, batches of 17..32 rows then run 64-thread teams (:func:`concurrent_params`). CPU tensors
    are solved in place in page-locked host memory (``bed_eigh_many_f32_pinned``: the kernels read the
    matrices and write the results across the host-device link, no device buffers, one call for all
    batches); with ``host_chunks > 0`` they go through ``bed_eigh_f32_host`` instead (copy in, solve and
    copy out in that many pieces over two streams). Host results are returned once they are in
    (page-locked) host memory.
    Returns a list of ``(W, V)`` (``(W, V, info)`` with ``return_info``), in the order of ``mats``."""
    mats = list(mats)
    if not mats:
        return []
    if not torch.cuda.is_available():
        raise BedError("batched_eigh_many needs a CUDA device; there is no CPU path")
    host = not mats[0].is_cuda
    if any((not M.is_cuda) != host for M in mats):
        raise ValueError("batched_eigh_many expects all batches on the CPU or all on one CUDA device")
    dev = torch.device("cuda", torch.cuda.current_device()) if host else mats[0].device
    if not host and any(M.device != dev for M in mats):
        raise ValueError("batched_eigh_many expects all batches on one CUDA device")
    cur = torch.cuda.current_stream(dev)
    if host and host_chunks <= 0:
        return _many_pinned(mats, params, check, return_info, dev, cur)
    live = sum(1 for M in mats if M.numel() > 0)  # batches that launch (the count the team rule sees)
    fork = torch.cuda.Event()
    fork.record(cur)
    # largest n first: its launch is the longest and should start first
    order = sorted(range(len(mats)), key=lambda i: -mats[i].shape[-1])
    outs = [None] * len(mats)
    side = _streams(dev, 2 * len(mats) if host else len(mats))
    keep = []  # host inputs and device scratch of the copy path, alive until the final synchronize
    for k, i in enumerate(order):
        if host:
            Ah, lead, n = _host_batch(mats[i])
            b = Ah.shape[0]
            Wh = torch.empty((b, n), dtype=torch.float32, pin_memory=True)
            Vh = torch.empty((b, n, n), dtype=torch.float32, pin_memory=True)
            Ih = torch.empty((b,), dtype=torch.int32, pin_memory=True)
            outs[i] = (Wh, Vh, Ih, True, lead, n)
            # copy-in / solve / copy-out pipelined in pieces over two streams (bed_eigh_f32_host)
            s0, s1 = side[2 * k], side[2 * k + 1]
            s0.wait_event(fork)
            s1.wait_event(fork)
            with torch.cuda.stream(s0):
                Ad = torch.empty((b, n, n), dtype=torch.float32, device=dev)
                Wd = torch.empty((b, n), dtype=torch.float32, device=dev)
                Vd = torch.empty((b, n, n), dtype=torch.float32, device=dev)
                Id = torch.empty((b,), dtype=torch.int32, device=dev)
            for t in (Ad, Wd, Vd, Id):
                t.record_stream(s1)
            keep.append((Ah, Ad, Wd, Vd, Id))
            _check(bed_eigh_f32_host(Ah.data_ptr(), Wh.data_ptr(), Vh.data_ptr(), Ih.data_ptr(), b, n,
                                     concurrent_params(params, n, live),
                                     Ad.data_ptr(), Wd.data_ptr(), Vd.data_ptr(), Id.data_ptr(), host_chunks,
                                     s0.cuda_stream, s1.cuda_stream))
            for s in (s0, s1):
                join = torch.cuda.Event()
                join.record(s)
                cur.wait_event(join)
        else:
            s = side[k]
            s.wait_event(fork)
            with torch.cuda.stream(s):
                outs[i] = _eigh_enqueue(mats[i], concurrent_params(params, mats[i].shape[-1], live), None)
            join = torch.cuda.Event()
            join.record(s)
            cur.wait_event(join)
            for t in outs[i][:3]:
                t.record_stream(cur)
    if host:
        cur.synchronize()
        del keep
    return [_eigh_finish(o, check, return_info) for o in outs]


def _host_batch(A: torch.Tensor):
    """A CPU batch as a page-locked [b, n, n] tensor, with its leading shape and n."""
    if A.dtype != torch.float32 or A.dim() < 2 or A.shape[-1] != A.shape[-2]:
        raise ValueError("batched_eigh_many expects float32 [..., n, n] batches")
    lead, n = A.shape[:-2], A.shape[-1]
    Ah = A.reshape(-1, n, n).contiguous()
    if not Ah.is_pinned():
        Ah = Ah.pin_memory()
    return Ah, lead, n


def _many_pinned(mats, params, check, return_info, dev, cur):
    """Host batches through one bed_eigh_many_f32_pinned call on the current stream, then wait."""
    pend = _enqueue_pinned(mats, params, dev, cur, _streams(dev, len(mats)))
    return pend.wait(check, return_info)


class PendingEigh:
    """Results of an enqueued host-memory solve: :meth:`wait` blocks until they are in (page-locked)
    host memory and returns them like :func:`batched_eigh_many`. Dropping an unfinished one waits."""

    def __init__(self, outs, stream, keep):
        self._outs, self._stream, self._keep = outs, stream, keep

    def done(self) -> bool:
        return self._stream.query()

    def wait(self, check: bool = False, return_info: bool = False):
        self._stream.synchronize()
        self._keep = None
        return [_eigh_finish(o, check, return_info) for o in self._outs]

    def __del__(self):
        if getattr(self, "_keep", None) is not None:
            try:
                self._stream.synchronize()
            except Exception:
                pass


def _enqueue_pinned(mats, params, dev, origin, side):
    ins = [_host_batch(M) for M in mats]
    outs = []
    for Ah, lead, n in ins:
        b = Ah.shape[0]
        W = torch.empty((b, n), dtype=torch.float32, pin_memory=True)
        V = torch.empty((b, n, n), dtype=torch.float32, pin_memory=True)
        I = torch.empty((b,), dtype=torch.int32, pin_memory=True)
        outs.append((W, V, I, True, lead, n))
    live = [k for k, (Ah, _, _) in enumerate(ins) if Ah.shape[0] > 0]
    if live:
        _check(bed_eigh_many_f32_pinned([ins[k][2] for k in live], [ins[k][0].shape[0] for k in live],
                                        [ins[k][0].data_ptr() for k in live], [outs[k][0].data_ptr() for k in live],
                                        [outs[k][1].data_ptr() for k in live], [outs[k][2].data_ptr() for k in live],
                                        params, origin.cuda_stream, [s.cuda_stream for s in side[: len(live)]]))
    return PendingEigh(outs, origin, [x[0] for x in ins])


_async_slots: dict = {}


def batched_eigh_many_async(mats, params: bed_params | None = None, slots: int = 2) -> PendingEigh:
    """Enqueues the zero-copy solve of several uniform batches held in CPU tensors and returns at once.

    Calls rotate over ``slots`` sets of streams (a completion stream and one stream per batch), so that
    up to ``slots`` calls are in flight and one call's reads and writes across the host-device link
    overlap another's solve. The work does not wait for anything on the caller's current stream (the
    inputs are host tensors). Returns a :class:`PendingEigh`; its ``wait()`` gives the results."""
    mats = list(mats)
    if not torch.cuda.is_available():
        raise BedError("batched_eigh_many_async needs a CUDA device; there is no CPU path")
    if any(M.is_cuda for M in mats):
        raise ValueError("batched_eigh_many_async expects CPU tensors")
    if slots < 1:
        raise ValueError("slots must be >= 1")
    dev = torch.device("cuda", torch.cuda.current_device())
    st = _async_slots.setdefault(dev.index, {"next": 0, "sets": []})
    sets = st["sets"]
    k = st["next"] % slots
    st["next"] = k + 1
    while len(sets) <= k:
        sets.append([torch.cuda.Stream(dev)])
    streams = sets[k]
    while len(streams) < 1 + len(mats):
        streams.append(torch.cuda.Stream(dev))
    return _enqueue_pinned(mats, params, dev, streams[0], streams[1:])


def batched_eigh_ragged(mats, params: bed_params | None = None, tuning: bed_ragged_tuning | None = None,
                        return_info: bool = False):
    """Eigendecompositions of a list of square FP32 matrices of mixed size (one persistent launch)."""
    if not torch.cuda.is_available():
        raise BedError("batched_eigh_ragged needs a CUDA device; there is no CPU path")
    ns = [int(torch.as_tensor(M).shape[-1]) for M in mats]
    rb = RaggedBatch(ns, params=params, tuning=tuning).load(mats).solve()
    res = rb.results()
    return (res, rb.info[: rb.count]) if return_info else res


class EighFunction(torch.autograd.Function):
    """Differentiable batched eigendecomposition: forward by bed_eigh_f32, backward by
    bed_eigh_backward_f32 (both CUDA kernels of this library)."""

    @staticmethod
    def forward(ctx, A, params, gap_eps):
        W, V = batched_eigh(A, params)
        ctx.save_for_backward(W, V)
        ctx.gap_eps = float(gap_eps)
        return W, V

    @staticmethod
    def backward(ctx, gW, gV):
        W, V = ctx.saved_tensors
        n = V.shape[-1]
        Wc = W.reshape(-1, n).contiguous()
        Vc = V.reshape(-1, n, n).contiguous()
        b = Vc.shape[0]
        gWc = gW.reshape(-1, n).contiguous().float() if gW is not None else None
        gVc = gV.reshape(-1, n, n).contiguous().float() if gV is not None else None
        gA = torch.empty_like(Vc)
        st = bed_eigh_backward_f32(Wc.data_ptr(), Vc.data_ptr(), gWc.data_ptr() if gWc is not None else None,
                                   gVc.data_ptr() if gVc is not None else None, gA.data_ptr(), b, n, ctx.gap_eps,
                                   torch.cuda.current_stream(V.device).cuda_stream)
        _check(st)
        return gA.reshape(V.shape), None, None


def eigh(A: torch.Tensor, params: bed_params | None = None, gap_eps: float = 0.0):
    """Differentiable ``(W, V) = eigh(A)`` for a CUDA FP32 batch ``A[..., n, n]`` (lower triangle read).
    The gradient returned for A is symmetric (gradient over symmetric perturbations); eigenvalue pairs
    closer than ``gap_eps`` do not couple their eigenvectors in the backward pass. The default 0 masks
    exact ties only: for inputs that may have nearly repeated eigenvalues (closer than about
    n * 2^-24 * max|lambda|, which FP32 cannot resolve) pass e.g. ``gap_eps = 1e-6 * max|lambda|``, or
    the 1/gap factors of such pairs turn rounding noise into large gradients."""
    if not A.is_cuda:
        raise BedError("eigh (differentiable) expects a CUDA tensor")
    return EighFunction.apply(A, params, gap_eps)
