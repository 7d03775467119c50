"""Continuous batching: results are the same alone and in the mix, memory stays within budget (GPU)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_27325_gb300 import binding as B
from paper_2604_27325_gb300 import serve
from parity import assert_parity

pytestmark = pytest.mark.gpu


def _requests(seed, count):
    pool = serve.request_pool(seed, per_n=64)
    rng = np.random.default_rng(seed)
    reqs = []
    for _ in range(count):
        n = int(rng.integers(8, 65))
        b = int(rng.integers(1, 65))
        s = int(rng.integers(0, 64 - b + 1))
        reqs.append(pool[n][s: s + b])
    return reqs


def test_each_result_is_the_same_alone_and_in_the_mix():
    reqs = _requests(11, 60)
    srv = serve.Server(budget_bytes=256 << 20, streams=3)
    mixed = [f.result() for f in [srv.submit(r) for r in reqs]]  # all submitted at once: coalesced launches
    alone = [srv.submit(r).result() for r in reqs]               # one at a time: one launch each
    stats = srv.stats.summary()
    srv.close()
    assert stats["launches"] < len(reqs) + len(reqs)  # the mixed phase shared launches
    for (W1, V1, i1), (W2, V2, i2), A in zip(mixed, alone, reqs):
        assert torch.equal(W1, W2) and torch.equal(V1, V2)
        assert int(i1.abs().sum()) == 0
    for A, (W, V, info) in list(zip(reqs, mixed))[:12]:
        Wo, Vo, _, _ = oracle.eigh_batch_f32(A.numpy(), nthreads=4)
        assert_parity(A.numpy(), W.numpy(), V.numpy(), info.numpy(), Wo, Vo, "served request")


def test_budget_admission_and_refusal():
    reqs = _requests(12, 40)
    budget = 3 << 20  # smaller than the sum of the requests: they must wait for memory to free up
    srv = serve.Server(budget_bytes=budget, streams=2)
    too_big = torch.zeros(256, 64, 64)
    f_big = srv.submit(too_big)
    futs = [srv.submit(r) for r in reqs]
    res = [f.result() for f in futs]
    stats = srv.stats.summary()
    srv.close()
    with pytest.raises(MemoryError):
        f_big.result()
    assert stats["requests"] == len(reqs)
    assert stats["peak_device_bytes"] <= budget
    assert all(W.shape[0] == A.shape[0] for (W, _, _), A in zip(res, reqs))


def test_queue_server_gives_the_same_results():
    reqs = _requests(13, 10)
    q = serve.QueueServer()
    a = [q.submit(r).result() for r in reqs]
    q.close()
    srv = serve.Server(budget_bytes=64 << 20)
    b = [srv.submit(r).result() for r in reqs]
    srv.close()
    for (W1, V1, _), (W2, V2, _), A in zip(a, b, reqs):
        Wo, Vo, _, _ = oracle.eigh_batch_f32(A.numpy(), nthreads=4)
        assert_parity(A.numpy(), W1.numpy(), V1.numpy(), np.zeros(A.shape[0]), Wo, Vo, "queue server")
        assert_parity(A.numpy(), W2.numpy(), V2.numpy(), np.zeros(A.shape[0]), Wo, Vo, "batching server")


def test_short_poisson_run():
    srv = serve.Server(budget_bytes=1 << 30)
    out = serve.run_load(srv, rate=500.0, seconds=1.0, seed=14)
    srv.close()
    assert out["requests"] == out["offered_requests"] and out["p99_ms"] > 0


def test_native_server_same_results_alone_and_in_the_mix():
    reqs = _requests(21, 50)
    srv = serve.NativeServer(budget_bytes=256 << 20, host_result_bytes=256 << 20, streams=3)
    ids = [srv.submit(r) for r in reqs]                      # together: coalesced into shared launches
    mixed = [srv.result(i, r.shape[0], r.shape[-1]) for i, r in zip(ids, reqs)]
    mixed_launches = srv.stats()["launches"]
    alone = []
    for r in reqs:                                           # one at a time: one launch each
        i = srv.submit(r)
        alone.append(srv.result(i, r.shape[0], r.shape[-1]))
    srv.close()
    assert mixed_launches < len(reqs)
    for (W1, V1, i1), (W2, V2, i2) in zip(mixed, alone):
        assert torch.equal(W1, W2) and torch.equal(V1, V2) and int(i1.abs().sum()) == 0
    for A, (W, V, info) in list(zip(reqs, mixed))[:10]:
        Wo, Vo, _, _ = oracle.eigh_batch_f32(A.numpy(), nthreads=4)
        assert_parity(A.numpy(), W.numpy(), V.numpy(), info.numpy(), Wo, Vo, "native server")


def test_native_server_budget_and_fifo_mode():
    reqs = _requests(22, 30)
    budget = 3 << 20
    # inputs and results through the device arena: admission is held to the device budget
    srv = serve.NativeServer(budget_bytes=budget, host_result_bytes=64 << 20, streams=2, zero_copy=False)
    with pytest.raises(B.BedError):
        srv.submit(torch.zeros(256, 64, 64).pin_memory())
    ids = [srv.submit(r) for r in reqs]
    res = [srv.result(i, r.shape[0], r.shape[-1]) for i, r in zip(ids, reqs)]
    st = srv.stats()
    srv.close()
    assert st["requests"] == len(reqs) and 0 < st["peak_device_bytes"] <= budget
    fifo = serve.NativeServer(budget_bytes=64 << 20, host_result_bytes=64 << 20, mode="fifo")
    ids = [fifo.submit(r) for r in reqs]
    res2 = [fifo.result(i, r.shape[0], r.shape[-1]) for i, r in zip(ids, reqs)]
    st2 = fifo.stats()
    fifo.close()
    assert st2["launches"] == len(reqs)
    for (W1, V1, _), (W2, V2, _), A in zip(res, res2, reqs):
        Wo, Vo, _, _ = oracle.eigh_batch_f32(A.numpy(), nthreads=4)
        assert_parity(A.numpy(), W1.numpy(), V1.numpy(), np.zeros(A.shape[0]), Wo, Vo, "batch mode")
        assert_parity(A.numpy(), W2.numpy(), V2.numpy(), np.zeros(A.shape[0]), Wo, Vo, "fifo mode")


def test_native_short_poisson_run():
    srv = serve.NativeServer(budget_bytes=1 << 30, host_result_bytes=512 << 20)
    out = serve.run_load_native(srv, rate=1000.0, seconds=1.0, seed=23)
    srv.close()
    assert out["requests"] == out["offered_requests"] and out["p99_ms"] > 0
    # each part of a request's time is bounded by the slowest request's whole latency
    for part in ("max_admit_wait_ms", "max_enqueue_ms", "max_inflight_ms"):
        assert 0.0 <= out[part] <= out["max_ms"] + 1e-6, (part, out[part], out["max_ms"])
    assert out["max_inflight_ms"] > 0


def test_native_server_zero_copy_equals_staged_and_unpinned_inputs_are_staged():
    """Zero-copy (inputs read in place, results written in place) and the staged data path run the same
    kernels on the same matrices: bitwise equal results. An input that is not page-locked is staged
    through the device arena even in zero-copy mode, with the same results."""
    reqs = _requests(31, 24)
    out = {}
    for zc in (True, False):
        srv = serve.NativeServer(budget_bytes=256 << 20, host_result_bytes=256 << 20, zero_copy=zc)
        ids = [srv.submit(r) for r in reqs]
        out[zc] = [srv.result(i, r.shape[0], r.shape[-1]) for i, r in zip(ids, reqs)]
        if zc:
            assert srv.stats()["peak_device_bytes"] == 0  # nothing staged
            ids = [srv.submit(r.clone(), pin=False) for r in reqs[:6]]
            out["unpinned"] = [srv.result(i, r.shape[0], r.shape[-1]) for i, r in zip(ids, reqs[:6])]
            assert srv.stats()["peak_device_bytes"] > 0
        srv.close()
    for (W1, V1, i1), (W2, V2, i2) in zip(out[True], out[False]):
        assert torch.equal(W1, W2) and torch.equal(V1, V2) and torch.equal(i1, i2)
    for (W1, V1, _), (W3, V3, _) in zip(out[True][:6], out["unpinned"]):
        assert torch.equal(W1, W3) and torch.equal(V1, V3)


@pytest.mark.parametrize("mode", ["batch", "fifo"])
def test_native_server_refuses_requests_beyond_the_launch_cap(mode):
    """A request larger than max_launch_matrices is refused before admission in both modes (its
    descriptors would not fit the per-launch arrays)."""
    srv = serve.NativeServer(budget_bytes=64 << 20, host_result_bytes=64 << 20, max_launch_matrices=8, mode=mode)
    with pytest.raises(B.BedError, match="TOO_LARGE"):
        srv.submit(torch.zeros(9, 8, 8))
    rid = srv.submit(_requests(5, 1)[0][:8])
    st, _, _, _ = B.bed_server_wait(srv.h, rid, 10.0)
    assert st == B.BED_OK
    srv.release(rid)
    srv.close()


def test_native_server_shutdown_completes_every_admitted_request():
    """Requests queued right before destroy are launched and completed (the completion thread waits for
    batches still being launched)."""
    reqs = _requests(41, 40)
    srv = serve.NativeServer(budget_bytes=256 << 20, host_result_bytes=256 << 20)
    for r in reqs:
        srv.submit(r)
    srv.close()  # must return: every admitted launch is retired
