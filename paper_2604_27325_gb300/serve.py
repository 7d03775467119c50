"""Continuous-batching request loop for batched eigendecompositions on one GPU.

A request is a batch of b symmetric FP32 matrices of one size n (host memory). The server

* admits requests in arrival order while their device memory fits a fixed budget (a pre-allocated arena:
  no device allocation happens per request); a request larger than the whole budget is refused;
* keeps each admitted request's inputs and outputs resident in the arena until it completes;
* coalesces everything admitted since the last launch into ONE ragged launch (matrices of all sizes
  together, `bed_eigh_ragged_f32`), on one of several streams, so that work of requests that arrived
  while others were running overlaps on the device;
* completes requests from a second thread that polls the launches' events, copies results to host
  memory and frees their arena space, which admits the requests waiting behind them.

`QueueServer` is the plain alternative: one request at a time, one uniform-size launch each, FIFO.
Both record per-request latency (submit to result on the host) and completed matrices.
"""
from __future__ import annotations

import bisect
import collections
import concurrent.futures as cf
import ctypes as C
import threading
import time

import numpy as np
import torch

from . import binding as B

ALIGN = 4  # floats: every request starts on a 16-byte boundary


def _pad(x: int) -> int:
    return (x + ALIGN - 1) // ALIGN * ALIGN


class Arena:
    """First-fit allocator over [0, capacity) (in floats) with coalescing free blocks. Host-side
    bookkeeping for one pre-allocated device buffer."""

    def __init__(self, capacity: int):
        self.capacity = capacity
        self.free_off = [0]
        self.free_len = [capacity]
        self.used = 0

    def alloc(self, size: int):
        size = _pad(max(size, 1))
        for k, (o, ln) in enumerate(zip(self.free_off, self.free_len)):
            if ln >= size:
                if ln == size:
                    del self.free_off[k]
                    del self.free_len[k]
                else:
                    self.free_off[k] = o + size
                    self.free_len[k] = ln - size
                self.used += size
                return o
        return None

    def free(self, off: int, size: int):
        size = _pad(max(size, 1))
        k = bisect.bisect_left(self.free_off, off)
        self.free_off.insert(k, off)
        self.free_len.insert(k, size)
        self.used -= size
        # coalesce with the right neighbour, then the left one
        if k + 1 < len(self.free_off) and self.free_off[k] + self.free_len[k] == self.free_off[k + 1]:
            self.free_len[k] += self.free_len.pop(k + 1)
            self.free_off.pop(k + 1)
        if k > 0 and self.free_off[k - 1] + self.free_len[k - 1] == self.free_off[k]:
            self.free_len[k - 1] += self.free_len.pop(k)
            self.free_off.pop(k)


class Request:
    __slots__ = ("rid", "A", "n", "b", "t_submit", "t_done", "future", "a_off", "w_off", "Wh", "Vh")

    def __init__(self, rid, A):
        self.rid = rid
        self.A = A
        self.b, self.n = int(A.shape[0]), int(A.shape[-1])
        self.t_submit = time.perf_counter()
        self.t_done = None
        self.future = cf.Future()
        self.a_off = self.w_off = None
        self.Wh = self.Vh = None

    @property
    def a_size(self):
        return self.b * self.n * self.n

    @property
    def w_size(self):
        return self.b * self.n


class _Stats:
    def __init__(self):
        self.lock = threading.Lock()
        self.latencies = []
        self.matrices = 0
        self.requests = 0
        self.launches = 0
        self.peak_bytes = 0

    def summary(self, seconds: float | None = None):
        with self.lock:
            lat = np.array(self.latencies) * 1e3
            out = {"requests": self.requests, "matrices": self.matrices, "launches": self.launches,
                   "peak_device_bytes": self.peak_bytes}
        if lat.size:
            out.update(p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                       mean_ms=float(lat.mean()), max_ms=float(lat.max()))
        if seconds:
            out["matrices_per_s"] = out["matrices"] / seconds
        return out


class _Launch:
    __slots__ = ("slot", "event", "batch", "info")

    def __init__(self, slot, event, batch, info):
        self.slot, self.event, self.batch, self.info = slot, event, batch, info


class Server:
    """Continuous batching over the ragged persistent kernel (see the module docstring)."""

    def __init__(self, budget_bytes: int = 4 << 30, streams: int = 3, max_launch_matrices: int = 16384,
                 tuning: B.bed_ragged_tuning | None = None, params: B.bed_params | None = None, device=None):
        self.dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.budget = int(budget_bytes)
        # A and V share one layout (the ragged entry point uses the same offsets for both); W needs at
        # most 1/16 of A + V for n >= 8, generously 1/8 here.
        unit = self.budget // 4
        cap_av = max(unit * 15 // 16 // 2, 64)
        cap_w = max(unit - 2 * cap_av, 64)
        self.A = torch.empty(cap_av, dtype=torch.float32, device=self.dev)
        self.V = torch.empty(cap_av, dtype=torch.float32, device=self.dev)
        self.W = torch.empty(cap_w, dtype=torch.float32, device=self.dev)
        self.av_arena, self.w_arena = Arena(cap_av), Arena(cap_w)
        self.max_launch = int(max_launch_matrices)
        self.tuning, self.params = tuning, params
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(streams)]
        ws = B.bed_eigh_ragged_workspace_size(self.max_launch)
        self.workspaces = [torch.empty(ws // 4, dtype=torch.int32, device=self.dev) for _ in range(streams)]
        self.ws_bytes = ws
        m = self.max_launch
        self.idx_host = [(torch.empty(m, dtype=torch.int64, pin_memory=True), torch.empty(m, dtype=torch.int32, pin_memory=True),
                          torch.empty(m, dtype=torch.int64, pin_memory=True)) for _ in range(streams)]
        self.idx_dev = [(torch.empty(m, dtype=torch.int64, device=self.dev), torch.empty(m, dtype=torch.int32, device=self.dev),
                         torch.empty(m, dtype=torch.int64, device=self.dev)) for _ in range(streams)]
        self.idx_np = [(a.numpy(), b.numpy(), c.numpy()) for a, b, c in self.idx_host]
        self._ramp = np.arange(self.max_launch, dtype=np.int64)
        self.info_dev = [torch.empty(m, dtype=torch.int32, device=self.dev) for _ in range(streams)]
        self.slot_busy = [False] * streams
        self.pending = collections.deque()
        self.inflight = collections.deque()  # _Launch records, oldest first
        self.cv = threading.Condition()
        self.stats = _Stats()
        self.running = True
        self._rid = 0
        torch.cuda.synchronize(self.dev)
        self.t_sched = threading.Thread(target=self._schedule, daemon=True)
        self.t_done = threading.Thread(target=self._complete, daemon=True)
        self.t_sched.start()
        self.t_done.start()

    # ------------------------------------------------------------------ public
    def submit(self, A) -> cf.Future:
        """Queue b x n x n FP32 matrices (host); the future resolves to host tensors (W [b,n], V [b,n,n],
        info [b]), or raises MemoryError if the request alone exceeds the device-memory budget."""
        A = torch.as_tensor(A)
        if A.dtype != torch.float32 or A.dim() != 3 or A.shape[1] != A.shape[2] or not 1 <= A.shape[-1] <= 64:
            raise ValueError("a request is a float32 [b, n, n] batch with 1 <= n <= 64")
        if not A.is_pinned():
            A = A.contiguous().pin_memory()
        with self.cv:
            self._rid += 1
            r = Request(self._rid, A)
            if r.a_size > self.av_arena.capacity or r.w_size > self.w_arena.capacity or r.b > self.max_launch:
                r.future.set_exception(MemoryError("request exceeds the device-memory budget"))
                return r.future
            self.pending.append(r)
            self.cv.notify_all()
        return r.future

    def close(self):
        with self.cv:
            self.running = False
            self.cv.notify_all()
        self.t_sched.join()
        self.t_done.join()

    def device_bytes_in_use(self):
        return 4 * (2 * self.av_arena.used + self.w_arena.used)

    # ------------------------------------------------------------------ scheduler thread
    def _admit(self):
        """Requests at the head of the queue that fit the arenas (FIFO, no overtaking)."""
        batch, count = [], 0
        while self.pending:
            r = self.pending[0]
            if count + r.b > self.max_launch:
                break
            a = self.av_arena.alloc(r.a_size)
            if a is None:
                break
            w = self.w_arena.alloc(r.w_size)
            if w is None:
                self.av_arena.free(a, r.a_size)
                break
            r.a_off, r.w_off = a, w
            self.pending.popleft()
            batch.append(r)
            count += r.b
        if batch:
            with self.stats.lock:
                self.stats.peak_bytes = max(self.stats.peak_bytes, self.device_bytes_in_use())
        return batch

    def _schedule(self):
        torch.cuda.set_device(self.dev)
        while True:
            with self.cv:
                while self.running and (not self.pending or all(self.slot_busy)):
                    self.cv.wait()
                if not self.running and not self.pending:
                    return
                slot = self.slot_busy.index(False)
                batch = self._admit()
                if not batch:  # the head does not fit yet: wait for memory to be freed
                    self.cv.wait(0.001)
                    continue
                self.slot_busy[slot] = True
            self._launch(slot, batch)

    def _launch(self, slot, batch):
        s = self.streams[slot]
        off_h, ns_h, woff_h = self.idx_host[slot]
        off_d, ns_d, woff_d = self.idx_dev[slot]
        # index arrays of the launch: matrix j of request r sits at a_off + j n^2 (A and V), w_off + j n (W)
        off_np, ns_np, woff_np = self.idx_np[slot]
        k = 0
        for r in batch:
            j = self._ramp[: r.b]
            off_np[k: k + r.b] = j * (r.n * r.n) + r.a_off
            woff_np[k: k + r.b] = j * r.n + r.w_off
            ns_np[k: k + r.b] = r.n
            k += r.b
        with torch.cuda.stream(s):
            off_d[:k].copy_(off_h[:k], non_blocking=True)
            ns_d[:k].copy_(ns_h[:k], non_blocking=True)
            woff_d[:k].copy_(woff_h[:k], non_blocking=True)
            for r in batch:
                self.A[r.a_off: r.a_off + r.a_size].copy_(r.A.view(-1), non_blocking=True)
            info = self.info_dev[slot]
            st = B.bed_eigh_ragged_f32(self.A.data_ptr(), off_d.data_ptr(), ns_d.data_ptr(), k, self.W.data_ptr(),
                                       woff_d.data_ptr(), self.V.data_ptr(), info.data_ptr(), self.params, self.tuning,
                                       self.workspaces[slot].data_ptr(), self.ws_bytes, None, s.cuda_stream)
            if st != B.BED_OK:
                err = B.BedError(B.bed_status_string(st))
                for r in batch:
                    r.future.set_exception(err)
            for r in batch:
                r.Wh = torch.empty(r.b, r.n, dtype=torch.float32, pin_memory=True)
                r.Vh = torch.empty(r.b, r.n, r.n, dtype=torch.float32, pin_memory=True)
                r.Wh.view(-1).copy_(self.W[r.w_off: r.w_off + r.w_size], non_blocking=True)
                r.Vh.view(-1).copy_(self.V[r.a_off: r.a_off + r.a_size], non_blocking=True)
            info_h = torch.empty(k, dtype=torch.int32, pin_memory=True)
            info_h.copy_(info[:k], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        with self.cv:
            self.inflight.append(_Launch(slot, ev, batch, info_h))
            self.cv.notify_all()
        with self.stats.lock:
            self.stats.launches += 1

    # ------------------------------------------------------------------ completion thread
    def _complete(self):
        torch.cuda.set_device(self.dev)
        while True:
            with self.cv:
                while self.running and not self.inflight:
                    self.cv.wait()
                if not self.running and not self.inflight and not self.pending:
                    return
                oldest = self.inflight[0] if self.inflight else None
            if oldest is None:  # closing while the scheduler still drains the queue
                with self.cv:
                    self.cv.wait(0.001)
                continue
            oldest.event.synchronize()  # blocks without holding the interpreter lock
            with self.cv:
                done = [it for it in self.inflight if it.event.query()]
            now = time.perf_counter()
            with self.cv:
                ids = {id(it) for it in done}
                self.inflight = collections.deque(it for it in self.inflight if id(it) not in ids)
                for it in done:
                    for r in it.batch:
                        self.av_arena.free(r.a_off, r.a_size)
                        self.w_arena.free(r.w_off, r.w_size)
                    self.slot_busy[it.slot] = False
                self.cv.notify_all()
            for it in done:
                k = 0
                info_h = it.info
                for r in it.batch:
                    r.t_done = now
                    inf = info_h[k: k + r.b]
                    k += r.b
                    if not r.future.done():
                        r.future.set_result((r.Wh, r.Vh, inf.clone()))
                    r.A = None
                    with self.stats.lock:
                        self.stats.latencies.append(r.t_done - r.t_submit)
                        self.stats.matrices += r.b
                        self.stats.requests += 1


class QueueServer:
    """Plain FIFO queue: one request at a time, one uniform-size launch each, on one stream."""

    def __init__(self, params: B.bed_params | None = None, device=None):
        self.dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.params = params
        self.q = collections.deque()
        self.cv = threading.Condition()
        self.running = True
        self.stats = _Stats()
        self.stream = torch.cuda.Stream(self.dev)
        self.t = threading.Thread(target=self._run, daemon=True)
        self.t.start()

    def submit(self, A) -> cf.Future:
        A = torch.as_tensor(A)
        if not A.is_pinned():
            A = A.contiguous().pin_memory()
        r = Request(0, A)
        with self.cv:
            self.q.append(r)
            self.cv.notify_all()
        return r.future

    def close(self):
        with self.cv:
            self.running = False
            self.cv.notify_all()
        self.t.join()

    def _run(self):
        torch.cuda.set_device(self.dev)
        while True:
            with self.cv:
                while self.running and not self.q:
                    self.cv.wait()
                if not self.q:
                    return
                r = self.q.popleft()
            with torch.cuda.stream(self.stream):
                Ad = r.A.to(self.dev, non_blocking=True)
                W = torch.empty(r.b, r.n, device=self.dev)
                V = torch.empty(r.b, r.n, r.n, device=self.dev)
                info = torch.empty(r.b, dtype=torch.int32, device=self.dev)
                st = B.bed_eigh_f32(Ad.data_ptr(), W.data_ptr(), V.data_ptr(), info.data_ptr(), r.b, r.n,
                                    self.params, self.stream.cuda_stream)
                Wh = W.to("cpu", non_blocking=True)
                Vh = V.to("cpu", non_blocking=True)
                ih = info.to("cpu", non_blocking=True)
            self.stream.synchronize()
            r.t_done = time.perf_counter()
            if st != B.BED_OK:
                r.future.set_exception(B.BedError(B.bed_status_string(st)))
            else:
                r.future.set_result((Wh, Vh, ih))
            with self.stats.lock:
                self.stats.latencies.append(r.t_done - r.t_submit)
                self.stats.matrices += r.b
                self.stats.requests += 1


def request_pool(seed: int = 5001, nmin: int = 8, nmax: int = 64, bmax: int = 256, per_n: int = 256):
    """Seeded matrices per size (half gapped known spectra, half covariances) from which requests draw."""
    from . import workloads

    pool = {}
    for n in range(nmin, nmax + 1):
        a = workloads.known_spectrum(per_n // 2, n, seed=seed + 2 * n)[0]
        c = workloads.covariance(per_n - per_n // 2, n, seed=seed + 2 * n + 1)
        m = np.empty((per_n, n, n), np.float32)
        m[0::2], m[1::2] = a, c
        pool[n] = torch.from_numpy(m).pin_memory()
    return pool


def run_load(server, rate: float = 2000.0, seconds: float = 60.0, seed: int = 5001, pool=None,
             nmin: int = 8, nmax: int = 64, bmax: int = 256, warmup_s: float = 1.0):
    """Poisson arrivals at `rate` requests/s for `seconds`; each request b ~ U{1..bmax} matrices of one size
    n ~ U{nmin..nmax} drawn from the pool. A warm-up of `warmup_s` at the same rate runs first and is not
    counted. Returns the server's statistics over the measured run."""
    pool = pool or request_pool(seed, nmin, nmax, bmax)
    if warmup_s > 0:
        run_load(server, rate, warmup_s, seed + 1, pool, nmin, nmax, bmax, warmup_s=0.0)
        server.stats = _Stats()
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    t = 0.0
    futs = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > seconds:
            break
        n = int(rng.integers(nmin, nmax + 1))
        b = int(rng.integers(1, bmax + 1))
        start = int(rng.integers(0, pool[n].shape[0] - b + 1))
        delay = t0 + t - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        futs.append(server.submit(pool[n][start: start + b]))
    for f in futs:
        f.result()
    wall = time.perf_counter() - t0
    out = server.stats.summary(wall)
    out["offered_requests"] = len(futs)
    out["wall_s"] = wall
    return out


class NativeServer:
    """The library's native request loop (C++ threads; include/bed.h, bed_server_*), mode "batch" for
    continuous batching over the ragged kernel or "fifo" for one uniform-size launch per request."""

    def __init__(self, budget_bytes: int = 4 << 30, host_result_bytes: int = 2 << 30, streams: int = 3,
                 max_launch_matrices: int = 16384, mode: str = "batch", tuning: B.bed_ragged_tuning | None = None,
                 params: B.bed_params | None = None, zero_copy: bool = True):
        cfg = B.bed_server_default_config()
        cfg.device_budget_bytes, cfg.host_result_bytes = int(budget_bytes), int(host_result_bytes)
        cfg.streams, cfg.max_launch_matrices = int(streams), int(max_launch_matrices)
        cfg.mode = 0 if mode == "batch" else 1
        cfg.zero_copy = 1 if zero_copy else 0
        st, self.h = B.bed_server_create(cfg, params, tuning)
        B._check(st)
        self.keep = {}  # request id -> input tensor, alive until the request completes

    def submit(self, A: torch.Tensor, pin: bool = True) -> int:
        """Queue a float32 [b, n, n] CPU tensor (copied to page-locked memory first unless ``pin`` is
        False, in which case the server stages it through its device arena); returns the request id
        (BedError if refused)."""
        A = A.contiguous()
        if pin and not A.is_pinned():
            A = A.pin_memory()
        st, rid = B.bed_server_submit(self.h, A.data_ptr(), int(A.shape[0]), int(A.shape[-1]))
        self.keep[rid] = A
        if st != B.BED_OK:
            B.bed_server_release(self.h, rid)
            self.keep.pop(rid, None)
            raise B.BedError(B.bed_status_string(st))
        return rid

    def result(self, rid: int, b: int, n: int, copy: bool = True, timeout_s: float = -1.0):
        """Waits for a request; returns (W [b,n], V [b,n,n], info [b]) (copied out unless copy=False, in
        which case the views are valid only until release) and releases it when copying."""
        st, W, V, I = B.bed_server_wait(self.h, rid, timeout_s)
        B._check(st)
        self.keep.pop(rid, None)
        if not copy:
            return W, V, I
        wv = torch.from_numpy(np.ctypeslib.as_array((C.c_float * (b * n)).from_address(W)).copy()).view(b, n)
        vv = torch.from_numpy(np.ctypeslib.as_array((C.c_float * (b * n * n)).from_address(V)).copy()).view(b, n, n)
        iv = torch.from_numpy(np.ctypeslib.as_array((C.c_int32 * b).from_address(I)).copy())
        B.bed_server_release(self.h, rid)
        return wv, vv, iv

    def release(self, rid: int):
        B.bed_server_release(self.h, rid)

    def stats(self) -> dict:
        s = B.bed_server_get_stats(self.h)
        out = {"requests": s.requests, "matrices": s.matrices, "launches": s.launches,
               "peak_device_bytes": s.peak_device_bytes}
        if s.requests:
            out.update(p50_ms=s.p50_s * 1e3, p99_ms=s.p99_s * 1e3, mean_ms=s.mean_s * 1e3, max_ms=s.max_s * 1e3,
                       max_admit_wait_ms=s.max_admit_wait_s * 1e3, max_enqueue_ms=s.max_enqueue_s * 1e3,
                       max_inflight_ms=s.max_inflight_s * 1e3)
        if s.span_s > 0:
            out["matrices_per_s"] = s.matrices / s.span_s
        return out

    def reset_stats(self):
        B.bed_server_reset_stats(self.h)

    def close(self):
        if self.h:
            B.bed_server_destroy(self.h)
            self.h = None


def run_load_native(server: NativeServer, rate: float = 2000.0, seconds: float = 60.0, seed: int = 5001,
                    pool=None, nmin: int = 8, nmax: int = 64, bmax: int = 256, warmup_s: float = 1.0):
    """Poisson load on a NativeServer: arrivals at `rate` requests/s for `seconds`, each request
    b ~ U{1..bmax} matrices of one size n ~ U{nmin..nmax} drawn from the pinned pool (the pool's memory
    is submitted in place, by address). One thread submits on schedule and, between arrivals, releases
    completed requests in submission order (a zero-timeout wait on the oldest), so no second Python
    thread competes for the interpreter. A warm-up of `warmup_s` at the same rate runs first and is not
    counted. Returns the server's statistics of the measured run plus the offered and achieved rates."""
    import collections

    pool = pool or request_pool(seed, nmin, nmax, bmax)
    if warmup_s > 0:
        run_load_native(server, rate, warmup_s, seed + 1, pool, nmin, nmax, bmax, warmup_s=0.0)
        server.reset_stats()
    rng = np.random.default_rng(seed)
    count = max(1, int(rate * seconds * 1.2) + 16)
    t_arr = np.cumsum(rng.exponential(1.0 / rate, size=count))
    t_arr = t_arr[t_arr <= seconds]
    ns = rng.integers(nmin, nmax + 1, size=len(t_arr))
    bs = rng.integers(1, bmax + 1, size=len(t_arr))
    u = rng.random(len(t_arr))
    base = {n: (pool[n].data_ptr(), pool[n].shape[0]) for n in range(nmin, nmax + 1)}
    h = server.h
    lib = B.lib()
    wait_c, rel_c = lib.bed_server_wait, lib.bed_server_release
    outstanding = collections.deque()

    def drain(block: bool):
        while outstanding:
            rid = outstanding[0]
            st = wait_c(h, rid, -1.0 if block else 0.0, None, None, None)
            if st == B.BED_ERR_TIMEOUT:
                return
            rel_c(h, rid)
            outstanding.popleft()

    rid = C.c_int64()
    submit_c = lib.bed_server_submit
    t0 = time.perf_counter()
    for k in range(len(t_arr)):
        n, b = int(ns[k]), int(bs[k])
        ptr, rows = base[n]
        start = int(u[k] * (rows - b + 1))
        last = -1.0
        while True:
            now = time.perf_counter() - t0
            if now >= t_arr[k]:
                break
            if outstanding and now - last > 20e-6:  # poll completions at most every 20 us
                drain(False)
                last = now
        st = submit_c(h, C.c_void_p(ptr + 4 * start * n * n), b, n, C.byref(rid))
        if st != B.BED_OK:
            raise B.BedError(B.bed_status_string(st))
        outstanding.append(rid.value)
    t_sub = time.perf_counter() - t0
    drain(True)
    out = server.stats()
    out["offered_requests"] = len(t_arr)
    out["offered_rate"] = rate
    out["achieved_submit_rate"] = len(t_arr) / max(t_sub, 1e-9)
    out["wall_s"] = time.perf_counter() - t0
    if out.get("launches"):
        out["requests_per_launch"] = out["requests"] / out["launches"]
    return out
