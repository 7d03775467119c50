"""Ragged batches (mixed n in one persistent launch) against the oracle and the uniform path (GPU)."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2604_27325_gb300 import binding as B
from paper_2604_27325_gb300 import workloads as wl
from parity import assert_parity, compare, record

pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 1
TEAM_THREADS = {0: 256, 1: 128, 2: 64, 3: 32, 4: 192}


def oracle_one(M):
    W, V, st, _ = oracle.eigh_batch_f32(M[None], nthreads=1)
    assert st.not_conv == 0
    return W[0], V[0]


def check_against_oracle(mats, res, info, what):
    by_n = {}
    for k, M in enumerate(mats):
        by_n.setdefault(M.shape[0], []).append(k)
    for n, ks in by_n.items():
        A = np.stack([mats[k] for k in ks])
        Wo, Vo, st, _ = oracle.eigh_batch_f32(A, nthreads=NTHREADS)
        W = np.stack([res[k][0].cpu().numpy() for k in ks])
        V = np.stack([res[k][1].cpu().numpy() for k in ks])
        assert_parity(A, W, V, info[ks], Wo, Vo, f"{what} n={n}")


def test_ragged_mixed_sizes_against_oracle():
    mats, ns = wl.ragged(600, nmin=1, nmax=64, seed=123)
    rb = B.RaggedBatch(ns).load(mats).solve()
    torch.cuda.synchronize()
    check_against_oracle(mats, rb.results(), rb.info.cpu().numpy()[: rb.count], "ragged")


def test_ragged_gapped_half_raw_eigenvectors():
    """The even indices of the ragged workload have known spectra with every gap >= 1e-3: there each
    eigenvector is pinned by its raw distance to the oracle's (up to sign), not only the gap-scaled bound."""
    mats, ns = wl.ragged(400, nmin=2, nmax=64, seed=321)
    rb = B.RaggedBatch(ns).load(mats).solve()
    torch.cuda.synchronize()
    res = rb.results()
    worst = 0.0
    for k in range(0, len(ns), 2):
        Wo, Vo = oracle_one(mats[k])
        r = compare(mats[k][None], res[k][0].cpu().numpy()[None], res[k][1].cpu().numpy()[None], Wo[None],
                    Vo[None])
        assert max(r[key] for key in ("eig", "res", "orth", "vec", "proj")) <= 1.0, (k, r)
        record(r, ns[k])
        worst = max(worst, r["vec_raw"])
    assert worst <= 1e-3, worst


@pytest.mark.parametrize("team,n", [(0, 64), (0, 41), (0, 33), (1, 32), (1, 19), (2, 16), (2, 5), (3, 16), (3, 3),
                                    (4, 48), (4, 40), (4, 33), (4, 20)])
@pytest.mark.parametrize("leaf", [1, 2, 8])
def test_ragged_equals_uniform_path_bitwise(team, n, leaf):
    """A ragged team runs the same per-matrix code as the uniform launch of the same shape."""
    A = wl.covariance(37, n, seed=500 + n)
    t = B.bed_ragged_default_tuning()
    t.team[n], t.leaf[n] = team, leaf
    rb = B.RaggedBatch([n] * 37, tuning=t).load(list(A)).solve()
    nmax = {0: 64, 1: 32, 2: 16, 3: 16, 4: 48}[team]
    Ad = torch.from_numpy(A).cuda()
    W = torch.empty(37, n, device="cuda")
    V = torch.empty(37, n, n, device="cuda")
    p = B.make_params(threads_per_matrix=TEAM_THREADS[team], leaf_size=leaf)
    assert TEAM_THREADS[team] in (2 * nmax, 4 * nmax)
    assert B.bed_eigh_f32(Ad.data_ptr(), W.data_ptr(), V.data_ptr(), None, 37, n, p,
                          torch.cuda.current_stream().cuda_stream) == B.BED_OK
    torch.cuda.synchronize()
    res = rb.results()
    for k in range(37):
        assert torch.equal(res[k][0], W[k]) and torch.equal(res[k][1], V[k])


@pytest.mark.parametrize("n48,n16,count48,count16", [(40, 12, 20, 30), (48, 16, 25, 9), (33, 5, 7, 7)])
def test_mixed_team_classes_equal_uniform_path_bitwise(n48, n16, count48, count16):
    """48-row-class and 16-row-class matrices in one ragged launch give bitwise the results of the
    uniform launches of the same team shapes (192 and 64 threads)."""
    A48 = wl.covariance(count48, n48, seed=700 + n48)
    A16 = wl.known_spectrum(count16, n16, seed=800 + n16)[0]
    ns = [n48] * count48 + [n16] * count16
    rb = B.RaggedBatch(ns).load(list(A48) + list(A16)).solve()
    torch.cuda.synchronize()
    res = rb.results()
    assert int((rb.info[: rb.count] != 0).sum()) == 0
    for A, n, tpm, off in ((A48, n48, 192, 0), (A16, n16, 64, count48)):
        Ad = torch.from_numpy(A).cuda()
        W = torch.empty(A.shape[0], n, device="cuda")
        V = torch.empty(A.shape[0], n, n, device="cuda")
        assert B.bed_eigh_f32(Ad.data_ptr(), W.data_ptr(), V.data_ptr(), None, A.shape[0], n,
                              B.make_params(threads_per_matrix=tpm), torch.cuda.current_stream().cuda_stream) == B.BED_OK
        torch.cuda.synchronize()
        for k in range(A.shape[0]):
            assert torch.equal(res[off + k][0], W[k]) and torch.equal(res[off + k][1], V[k])


def test_ragged_bad_sizes_are_flagged_and_skipped():
    ns = [8, 0, 12, 65, 3]
    rb = B.RaggedBatch(ns)
    for k, n in enumerate(ns):
        if 1 <= n <= 64:
            o = rb.offsets_list[k]
            rb.A[o: o + n * n].copy_(torch.from_numpy(wl.covariance(1, n, seed=n)[0].reshape(-1)))
    rb.solve()
    torch.cuda.synchronize()
    info = rb.info.cpu().numpy()[:5]
    assert info[1] == B.BED_INFO_BAD_N and info[3] == B.BED_INFO_BAD_N
    assert info[0] == info[2] == info[4] == 0


def test_ragged_graph_replay_matches_direct_call():
    mats, ns = wl.ragged(300, nmin=4, nmax=64, seed=7)
    rb = B.RaggedBatch(ns).load(mats).solve()
    torch.cuda.synchronize()
    W0, V0 = rb.W.clone(), rb.V.clone()
    rb.W.zero_()
    rb.V.zero_()
    rb.capture()
    rb.W.zero_()
    rb.V.zero_()
    for _ in range(2):
        rb.replay()
    torch.cuda.synchronize()
    assert torch.equal(rb.W, W0) and torch.equal(rb.V, V0)
    # new inputs in the same buffers are picked up by the replay
    mats2 = [wl.covariance(1, n, seed=900 + k)[0] for k, n in enumerate(ns)]
    rb.load(mats2).replay()
    torch.cuda.synchronize()
    check_against_oracle(mats2, rb.results(), rb.info.cpu().numpy()[: rb.count], "graph replay")


def test_ragged_counters_and_empty():
    mats, ns = wl.ragged(64, nmin=4, nmax=64, seed=9)
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    rb = B.RaggedBatch(ns).load(mats).solve(counters=cnt)
    torch.cuda.synchronize()
    matrices, roots, evals, deflated = cnt.tolist()
    assert matrices == 64 and roots > 0 and evals > roots
    rb0 = B.RaggedBatch([])
    rb0.solve()
    torch.cuda.synchronize()


def test_ragged_workload_full_size_graph_replay_against_oracle():
    """The ragged workload at its full size (8192 matrices, n ~ U{4..64}) in the configuration the
    benchmark times (tuned table, CUDA-graph replay), every matrix against the oracle."""
    from paper_2604_27325_gb300 import autotune

    mats, ns = wl.ragged(8192)
    rb = B.RaggedBatch(ns, tuning=autotune.load()).load(mats)
    rb.capture()
    rb.replay()
    torch.cuda.synchronize()
    check_against_oracle(mats, rb.results(), rb.info.cpu().numpy()[: rb.count], "ragged 8192")
