"""The workspace-free ragged entry point, bed_eigh_ragged_f32_noalloc (GPU).

Some callers cannot allocate device memory: their host framework's allocator owns all the device
memory they may touch, they are plugins handed only input and output buffers, or they serve requests
and must not call cudaMalloc (which can fail under memory pressure and synchronizes the device). For
them the library offers an entry point with no workspace argument; it keeps its scratch in an array
compiled into the library (BED_NOALLOC_MAX_COUNT matrices at most).

This test drives that entry point through the C ABI twice in a row, on two different batches (so the
second call starts from the scratch contents the first one left), and checks each result against the
workspace entry point bed_eigh_ragged_f32 on the same inputs, within the tolerances of the parity
tests. The test allocates its own input and output buffers; only the entry point must not allocate.
It sits in a file of its own that pytest collects last.
"""
import numpy as np
import pytest
import torch

from paper_2604_27325_gb300 import binding as B
from paper_2604_27325_gb300 import workloads as wl
from parity import assert_parity

pytestmark = pytest.mark.gpu


def _noalloc_solve(rb: B.RaggedBatch):
    W = torch.full_like(rb.W, -7.0)
    V = torch.full_like(rb.V, -7.0)
    info = torch.full_like(rb.info, -1)
    st = B.bed_eigh_ragged_f32_noalloc(rb.A.data_ptr(), rb.offsets.data_ptr(), rb.ns_dev.data_ptr(), rb.count,
                                       W.data_ptr(), rb.w_offsets.data_ptr(), V.data_ptr(), info.data_ptr(),
                                       None, None, None, torch.cuda.current_stream().cuda_stream)
    assert st == B.BED_OK, B.bed_status_string(st)
    return W, V, info


def test_noalloc_matches_workspace_entry_point_on_two_calls_in_a_row():
    for seed in (41, 42):
        mats, ns = wl.ragged(700, nmin=1, nmax=64, seed=seed)
        rb = B.RaggedBatch(ns).load(mats)
        W, V, info = _noalloc_solve(rb)
        rb.solve()  # the workspace entry point on the same inputs
        torch.cuda.synchronize()
        info = info.cpu().numpy()[: rb.count]
        ref = rb.results()
        for n in sorted(set(int(x) for x in ns)):
            ks = [k for k in range(rb.count) if ns[k] == n]
            A = np.stack([mats[k] for k in ks])
            Wr = np.stack([ref[k][0].cpu().numpy() for k in ks]).astype(np.float64)
            Vr = np.stack([ref[k][1].cpu().numpy() for k in ks]).astype(np.float64)
            Wn = np.stack([W[rb.woffsets_list[k]: rb.woffsets_list[k] + n].cpu().numpy() for k in ks])
            Vn = np.stack([V[rb.offsets_list[k]: rb.offsets_list[k] + n * n].view(n, n).cpu().numpy() for k in ks])
            assert_parity(A, Wn, Vn, info[ks], Wr, Vr, f"no-alloc entry point, call seed {seed}, n={n}")


def test_noalloc_rejects_batches_beyond_its_capacity():
    big = B.BED_NOALLOC_MAX_COUNT + 1
    st = B.bed_eigh_ragged_f32_noalloc(16, 16, 16, big, 16, 16, 4096, None, None, None, None, 0)
    assert st == B.BED_ERR_TOO_LARGE
    assert B.bed_status_string(st) == "BED_ERR_TOO_LARGE"
