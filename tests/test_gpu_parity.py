"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on seeded inputs (GPU)."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2604_27325_gb300 import binding as B
from paper_2604_27325_gb300 import workloads as wl
from parity import assert_parity

pytestmark = pytest.mark.gpu

NTHREADS = os.cpu_count() or 1


def run_gpu(A, params=None, offset=0):
    """A float32 numpy [b, n, n] -> (W, V, info) numpy, through bed_eigh_f32 on the current stream.
    offset > 0 places A at a non-16-byte-aligned address (exercises the plain-load staging path)."""
    b, n, _ = A.shape
    flat = torch.zeros(A.size + 8, dtype=torch.float32, device="cuda")
    Ad = flat[offset: offset + A.size].view(b, n, n)
    Ad.copy_(torch.from_numpy(np.ascontiguousarray(A)))
    W = torch.full((b, n), -7.0, device="cuda")
    V = torch.full((b, n, n), -7.0, device="cuda")
    info = torch.full((b,), -1, dtype=torch.int32, device="cuda")
    st = B.bed_eigh_f32(Ad.data_ptr(), W.data_ptr(), V.data_ptr(), info.data_ptr(), b, n, params,
                        torch.cuda.current_stream().cuda_stream)
    assert st == B.BED_OK, B.bed_status_string(st)
    torch.cuda.synchronize()
    return W.cpu().numpy(), V.cpu().numpy(), info.cpu().numpy()


def run_oracle(A):
    Wo, Vo, st, _ = oracle.eigh_batch_f32(A, nthreads=NTHREADS)
    assert st.not_conv == 0
    return Wo, Vo


# ----------------------------------------------------------------------------- the workloads


def test_plain_known_spectrum_batch64_n16():
    A, lam = wl.known_spectrum(64, 16, seed=wl.SEED_PLAIN)
    W, V, info = run_gpu(A)
    Wo, Vo = run_oracle(A)
    r = assert_parity(A, W, V, info, Wo, Vo, "known spectrum 64 x 16")
    # every gap of these spectra is >= 1e-3, so each eigenvector is pinned on its own, not only through
    # the gap-scaled bound: the raw distance to the oracle's vector (up to sign) stays small
    assert r["vec_raw"] <= 2.5e-4, r


@pytest.mark.parametrize("n", [16, 32, 48, 64])
def test_uniform_covariance_batch512(n):
    A = wl.covariance(512, n)
    W, V, info = run_gpu(A)
    Wo, Vo = run_oracle(A)
    assert_parity(A, W, V, info, Wo, Vo, f"covariance 512 x {n}")


@pytest.mark.parametrize("n", list(range(1, 65)))
def test_every_n_ragged_batch(n):
    """Every supported size, both input families, a batch that is not a multiple of anything."""
    A = np.concatenate([wl.covariance(5, n, seed=9000 + n), wl.known_spectrum(6, n, seed=9100 + n)[0]])
    W, V, info = run_gpu(A)
    Wo, Vo = run_oracle(A)
    assert_parity(A, W, V, info, Wo, Vo, f"n={n}")


# ----------------------------------------------------------------------------- edge cases


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 16, 17, 33, 64])
@pytest.mark.parametrize("name", ["zero", "identity", "diagonal", "repeated", "rank_one", "block_diagonal", "toeplitz"])
def test_degenerate_inputs(n, name):
    A = wl.special_cases(n)[name][None].repeat(3, axis=0)
    W, V, info = run_gpu(A)
    Wo, Vo = run_oracle(A)
    assert_parity(A, W, V, info, Wo, Vo, f"{name} n={n}")
    if name == "diagonal":
        assert np.array_equal(W[0], np.sort(np.diag(A[0])))


def test_empty_batch():
    W = torch.empty(0, 8, device="cuda")
    assert B.bed_eigh_f32(0, W.data_ptr(), W.data_ptr() + 4, None, 0, 8) == B.BED_OK


@pytest.mark.parametrize("n", [7, 16, 64])
def test_upper_triangle_is_ignored(n):
    A = wl.covariance(4, n, seed=77)
    G = A.copy()
    iu = np.triu_indices(n, 1)
    G[:, iu[0], iu[1]] = np.float32(123.0)
    W1, V1, _ = run_gpu(A)
    W2, V2, _ = run_gpu(G)
    assert np.array_equal(W1, W2) and np.array_equal(V1, V2)


@pytest.mark.parametrize("scale", [1e-30, 1e-12, 1e12, 1e30])
def test_extreme_scales(scale):
    A = (wl.covariance(8, 32, seed=5).astype(np.float64) * scale).astype(np.float32)
    W, V, info = run_gpu(A)
    Wo, Vo = run_oracle(A)
    assert_parity(A, W, V, info, Wo, Vo, f"scale {scale}")


def test_nonfinite_input_flags_only_that_matrix():
    A = wl.covariance(6, 12, seed=3)
    A[2, 5, 1] = np.nan
    A[4, 0, 0] = np.inf
    W, V, info = run_gpu(A)
    assert info[2] == B.BED_INFO_NONFINITE and info[4] == B.BED_INFO_NONFINITE
    assert np.all(np.isnan(W[[2, 4]])) and np.all(np.isnan(V[[2, 4]]))
    ok = [0, 1, 3, 5]
    Wo, Vo = run_oracle(A[ok])
    assert_parity(A[ok], W[ok], V[ok], info[ok], Wo, Vo, "finite matrices of a mixed batch")


@pytest.mark.parametrize("n", [15, 16, 48])
def test_unaligned_input_takes_the_plain_load_path_with_identical_results(n):
    A = wl.covariance(9, n, seed=11)
    W1, V1, i1 = run_gpu(A, offset=0)
    W2, V2, i2 = run_gpu(A, offset=1)
    assert np.array_equal(W1, W2) and np.array_equal(V1, V2) and np.array_equal(i1, i2)


# ----------------------------------------------------------------------------- parameters


@pytest.mark.parametrize("n", [16, 48, 64])
def test_vote_retirement_is_result_neutral(n):
    """Progressive shrinkage (Eq. (22)) recast as warp-vote retirement changes work, not results."""
    A = wl.covariance(64, n, seed=21)
    W1, V1, _ = run_gpu(A, B.make_params(retire_by_vote=1))
    W0, V0, _ = run_gpu(A, B.make_params(retire_by_vote=0))
    assert np.array_equal(W1, W0) and np.array_equal(V1, V0)


@pytest.mark.parametrize(
    "kw",
    [dict(leaf_size=1), dict(k_multisection=2), dict(k_multisection=8, section_rel_eps=2.0**-10),
     dict(section_rel_eps=0.5, max_section_iters=0), dict(threads_per_matrix=128), dict(n_bisect_first=3),
     dict(n_bisect_first=8, section_rel_eps=2.0**-10)],
)
def test_parameter_variants_hold_tolerance(kw):
    A = wl.covariance(32, 64 if kw.get("threads_per_matrix") == 128 else 40, seed=31)
    W, V, info = run_gpu(A, B.make_params(**kw))
    Wo, Vo = run_oracle(A)
    assert_parity(A, W, V, info, Wo, Vo, str(kw))


def test_counters():
    A = wl.covariance(16, 32, seed=41)
    cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
    Ad = torch.from_numpy(A).cuda()
    W = torch.empty(16, 32, device="cuda")
    V = torch.empty(16, 32, 32, device="cuda")
    st = B.bed_eigh_f32_counted(Ad.data_ptr(), W.data_ptr(), V.data_ptr(), None, 16, 32, None, cnt.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    assert st == B.BED_OK
    torch.cuda.synchronize()
    matrices, roots, evals, deflated = cnt.tolist()
    assert matrices == 16
    # each merge of size s yields s eigenpairs: roots + deflated = sum of merge sizes
    total = 16 * sum(hi - lo for lo, _, hi, _ in B.bed_plan_describe(32, B.make_params().leaf_size))
    assert roots + deflated == total
    assert roots > 0 and evals > roots


def test_bisection_steps_reach_the_secular_solver():
    """n_bisect_first changes the sectioning points (bisection instead of Eq. (16)'s multi-section), so
    with a small switch threshold the f evaluations the roots take change, while the results stay within
    tolerance (checked in test_parameter_variants_hold_tolerance)."""
    A = wl.covariance(16, 32, seed=43)
    Ad = torch.from_numpy(A).cuda()
    W = torch.empty(16, 32, device="cuda")
    V = torch.empty(16, 32, 32, device="cuda")
    evals = {}
    for nb in (1, 6):
        cnt = torch.zeros(4, dtype=torch.int64, device="cuda")
        p = B.make_params(n_bisect_first=nb, section_rel_eps=2.0**-10)
        st = B.bed_eigh_f32_counted(Ad.data_ptr(), W.data_ptr(), V.data_ptr(), None, 16, 32, p, cnt.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
        assert st == B.BED_OK
        torch.cuda.synchronize()
        matrices, roots, ev, _ = cnt.tolist()
        assert matrices == 16 and roots > 0
        evals[nb] = ev
    assert evals[1] != evals[6]


def test_host_buffers_end_to_end():
    A = wl.covariance(8, 24, seed=51)
    W, V, info = B.batched_eigh(torch.from_numpy(A), return_info=True)
    assert not W.is_cuda
    Wo, Vo = run_oracle(A)
    assert_parity(A, W.numpy(), V.numpy(), info.numpy(), Wo, Vo, "host path")


def test_large_batch_sampled():
    """A batch much larger than the GPU's resident blocks; sampled matrices against the oracle."""
    b, n = 4096, 64
    A = wl.covariance(b, n, seed=61)
    W, V, info = run_gpu(A)
    assert np.all(info == 0)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(b, 48, replace=False))
    Wo, Vo = run_oracle(A[idx])
    assert_parity(A[idx], W[idx], V[idx], info[idx], Wo, Vo, "sampled large batch")


@pytest.mark.parametrize("n", [7, 20, 48, 64])
def test_matrices_per_block_gives_the_same_results(n):
    """matrices_per_cta = k: ceil(batch / k) blocks each solving several matrices in turn (the staging
    copy and its mbarrier reused from one matrix to the next) give bitwise the one-block-per-matrix
    results, on the bulk-copy path (even n) and the plain-load path (odd n)."""
    A = np.concatenate([wl.covariance(45, n, seed=1200 + n), wl.known_spectrum(12, n, seed=1300 + n)[0]])
    W0, V0, i0 = run_gpu(A)
    for k in (1, 3, 8, 1000):
        W, V, info = run_gpu(A, B.make_params(matrices_per_cta=k))
        assert np.array_equal(W, W0) and np.array_equal(V, V0) and np.array_equal(info, i0), k
    Wo, Vo = run_oracle(A)
    assert_parity(A, W0, V0, i0, Wo, Vo, f"n={n}")


@pytest.mark.parametrize("seed", [1, 2])
def test_every_n_random_families_both_team_shapes(seed):
    """Every n, three input families (covariances, gapped known spectra, graded matrices whose entries
    span up to six orders of magnitude), on the automatic team shape and on the other one of its size
    class, against the oracle."""
    for n in range(1, 65):
        nmax = next(m for m in (16, 32, 48, 64) if m >= n)
        other = 256 if nmax == 64 else 2 * nmax
        A = np.concatenate([wl.covariance(4, n, seed=10000 * seed + n),
                            wl.known_spectrum(4, n, seed=20000 * seed + n)[0],
                            wl.graded(4, n, seed=30000 * seed + n)])
        Wo, Vo = run_oracle(A)
        for tpm in (0, other):
            W, V, info = run_gpu(A, B.make_params(threads_per_matrix=tpm))
            assert_parity(A, W, V, info, Wo, Vo, f"seed={seed} n={n} threads={tpm}")


@pytest.mark.parametrize("nmax,tpm", [(16, 32), (32, 64), (48, 96), (64, 256)])
def test_every_n_on_the_other_team_shape(nmax, tpm):
    """Every n of a size class on the team shape that the automatic choice does not give it alone (two
    lanes per row for 16, 32 and 48 rows -- the 64-thread teams are what sizes 17..32 run beside other
    sizes -- and four lanes per row for 64), covariances and gapped known spectra, against the oracle."""
    p = B.make_params(threads_per_matrix=tpm)
    for n in range(nmax - 15, nmax + 1):
        A = np.concatenate([wl.covariance(6, n, seed=9600 + n), wl.known_spectrum(4, n, seed=9700 + n)[0]])
        W, V, info = run_gpu(A, p)
        Wo, Vo = run_oracle(A)
        assert_parity(A, W, V, info, Wo, Vo, f"n={n} threads={tpm}")


@pytest.mark.parametrize("tpm", [96, 192, 128, 256])
def test_thread_count_selects_team_shape_n40(tpm):
    """n = 40 runs on the 48-row team (96 or 192 threads) or, when asked, the 64-row team (128, 256):
    every shape holds the tolerance."""
    A = wl.covariance(48, 40, seed=33)
    W, V, info = run_gpu(A, B.make_params(threads_per_matrix=tpm))
    Wo, Vo = run_oracle(A)
    assert_parity(A, W, V, info, Wo, Vo, f"n=40 threads={tpm}")


def test_thread_count_rejects_shapes_below_n():
    A = torch.from_numpy(wl.covariance(2, 40, seed=34)).cuda()
    W = torch.empty(2, 40, device="cuda")
    V = torch.empty(2, 40, 40, device="cuda")
    for tpm in (64, 100, 2 * 32):  # 64 = 4 x 16 or 2 x 32: both below n = 40
        st = B.bed_eigh_f32(A.data_ptr(), W.data_ptr(), V.data_ptr(), None, 2, 40,
                            B.make_params(threads_per_matrix=tpm), torch.cuda.current_stream().cuda_stream)
        assert st == B.BED_ERR_INVALID_ARG


@pytest.mark.parametrize("where", ["host", "device"])
def test_many_batches_on_streams_match_single_calls(where):
    """batched_eigh_many runs each batch on its own stream; results are those of one call per batch with
    the parameters a batch gets beside others (64-thread teams for 17..32 rows)."""
    mats = [torch.from_numpy(wl.covariance(40, n, seed=60 + n)) for n in (64, 17, 48, 5, 32)]
    if where == "device":
        mats = [M.cuda() for M in mats]
    many = B.batched_eigh_many(mats, return_info=True)
    torch.cuda.synchronize()
    for M, (W, V, info) in zip(mats, many):
        p1 = B.concurrent_params(None, M.shape[-1], len(mats))
        assert (p1 is not None) == (16 < M.shape[-1] <= 32)
        W1, V1, info1 = B.batched_eigh(M, params=p1, return_info=True)
        torch.cuda.synchronize()
        assert W.is_cuda == (where == "device")
        assert torch.equal(W.cpu(), W1.cpu()) and torch.equal(V.cpu(), V1.cpu())
        assert int((info != 0).sum()) == 0


# ----------------------------------------------------------------------------- QL leaves (Sec. 2.2)


@pytest.mark.parametrize("leaf", [3, 4, 5, 8])
def test_every_n_with_ql_leaves(leaf):
    """Leaves of up to `leaf` rows solved by the in-kernel implicit QL iteration, every n."""
    p = B.make_params(leaf_size=leaf)
    for n in range(1, 65):
        A = np.concatenate([wl.covariance(3, n, seed=9200 + n), wl.known_spectrum(3, n, seed=9300 + n)[0]])
        W, V, info = run_gpu(A, p)
        Wo, Vo = run_oracle(A)
        assert_parity(A, W, V, info, Wo, Vo, f"leaf={leaf} n={n}")


@pytest.mark.parametrize("leaf", [4, 8])
@pytest.mark.parametrize("name", ["zero", "identity", "diagonal", "repeated", "rank_one", "block_diagonal", "toeplitz"])
def test_degenerate_inputs_with_ql_leaves(leaf, name):
    for n in (3, 5, 8, 9, 16, 37, 64):
        A = wl.special_cases(n)[name][None].repeat(2, axis=0)
        W, V, info = run_gpu(A, B.make_params(leaf_size=leaf))
        Wo, Vo = run_oracle(A)
        assert_parity(A, W, V, info, Wo, Vo, f"{name} leaf={leaf} n={n}")


@pytest.mark.parametrize("n", [16, 32, 48, 64])
def test_uniform_covariance_with_ql_leaves(n):
    A = wl.covariance(512, n)
    W, V, info = run_gpu(A, B.make_params(leaf_size=8))
    Wo, Vo = run_oracle(A)
    assert_parity(A, W, V, info, Wo, Vo, f"covariance 512 x {n}, leaf 8")


@pytest.mark.parametrize("chunks", [0, 1, 3, 7])
def test_host_entry_point_pipelined(chunks):
    """bed_eigh_f32_host (copy-in, solve, copy-out in pieces over two streams) gives the results of
    bed_eigh_f32 on the same matrices, bitwise, for any cut of the batch."""
    A = wl.covariance(300, 37, seed=77)
    b, n = A.shape[0], A.shape[-1]
    Ah = torch.from_numpy(A).pin_memory()
    Wh = torch.full((b, n), -7.0).pin_memory()
    Vh = torch.full((b, n, n), -7.0).pin_memory()
    Ih = torch.full((b,), -1, dtype=torch.int32).pin_memory()
    Ad = torch.empty(b, n, n, device="cuda")
    Wd = torch.empty(b, n, device="cuda")
    Vd = torch.empty(b, n, n, device="cuda")
    Id = torch.empty(b, dtype=torch.int32, device="cuda")
    s0, s1 = torch.cuda.Stream(), torch.cuda.Stream()
    st = B.bed_eigh_f32_host(Ah.data_ptr(), Wh.data_ptr(), Vh.data_ptr(), Ih.data_ptr(), b, n, None, Ad.data_ptr(),
                             Wd.data_ptr(), Vd.data_ptr(), Id.data_ptr(), chunks, s0.cuda_stream, s1.cuda_stream)
    assert st == B.BED_OK
    torch.cuda.synchronize()
    W, V, info = run_gpu(A)
    assert np.array_equal(Wh.numpy(), W) and np.array_equal(Vh.numpy(), V) and np.array_equal(Ih.numpy(), info)
    # argument errors come back before anything is enqueued
    assert B.bed_eigh_f32_host(Ah.data_ptr(), Wh.data_ptr(), Vh.data_ptr(), Ih.data_ptr(), b, n, None,
                               Ad.data_ptr(), Wd.data_ptr(), Vd.data_ptr(), None, 0, 0, 0) == B.BED_ERR_INVALID_ARG
    assert B.bed_eigh_f32_host(Ah.data_ptr(), Wh.data_ptr(), Vh.data_ptr(), None, b, 65, None,
                               Ad.data_ptr(), Wd.data_ptr(), Vd.data_ptr(), None, 0, 0, 0) == B.BED_ERR_UNSUPPORTED_N


@pytest.mark.parametrize("n,b", [(1, 3), (5, 70), (37, 300), (64, 513)])
def test_pinned_zero_copy_entry_point(n, b):
    """bed_eigh_f32_pinned (the kernel reads and writes page-locked host memory directly) gives the
    results of bed_eigh_f32 on device buffers, bitwise."""
    A = wl.covariance(b, n, seed=78 + n)
    Ah = torch.from_numpy(A).pin_memory()
    Wh = torch.full((b, n), -7.0).pin_memory()
    Vh = torch.full((b, n, n), -7.0).pin_memory()
    Ih = torch.full((b,), -1, dtype=torch.int32).pin_memory()
    s = torch.cuda.Stream()
    assert B.bed_eigh_f32_pinned(Ah.data_ptr(), Wh.data_ptr(), Vh.data_ptr(), Ih.data_ptr(), b, n, None,
                                 s.cuda_stream) == B.BED_OK
    s.synchronize()
    W, V, info = run_gpu(A)
    assert np.array_equal(Wh.numpy(), W) and np.array_equal(Vh.numpy(), V) and np.array_equal(Ih.numpy(), info)
    if n == 64:
        Wo, Vo = run_oracle(A[:40])
        assert_parity(A[:40], Wh.numpy()[:40], Vh.numpy()[:40], Ih.numpy()[:40], Wo, Vo, "pinned entry point")


def test_pinned_entry_point_rejects_unmapped_buffers():
    """Pageable host memory and device memory are refused before anything is enqueued."""
    b, n = 4, 8
    Ah = torch.from_numpy(wl.covariance(b, n, seed=5)).pin_memory()
    Wh = torch.empty(b, n).pin_memory()
    Vh = torch.empty(b, n, n).pin_memory()
    pageable = np.zeros((b, n, n), dtype=np.float32)
    Vd = torch.empty(b, n, n, device="cuda")
    ok = (Ah.data_ptr(), Wh.data_ptr(), Vh.data_ptr())
    assert B.bed_eigh_f32_pinned(pageable.ctypes.data, ok[1], ok[2], None, b, n) == B.BED_ERR_INVALID_ARG
    assert B.bed_eigh_f32_pinned(ok[0], ok[1], pageable.ctypes.data, None, b, n) == B.BED_ERR_INVALID_ARG
    assert B.bed_eigh_f32_pinned(ok[0], ok[1], Vd.data_ptr(), None, b, n) == B.BED_ERR_INVALID_ARG
    assert B.bed_eigh_f32_pinned(ok[0], ok[1], ok[2], pageable.ctypes.data, b, n) == B.BED_ERR_INVALID_ARG
    assert B.bed_eigh_f32_pinned(ok[0], ok[1], ok[2], None, b, 65) == B.BED_ERR_UNSUPPORTED_N
    assert B.bed_eigh_f32_pinned(0, 0, 0, None, 0, n) == B.BED_OK
    assert B.bed_eigh_f32_pinned(ok[0], ok[1], ok[2], None, b, n) == B.BED_OK
    torch.cuda.synchronize()


def test_many_pinned_entry_point():
    """bed_eigh_many_f32_pinned: several sizes (one of them empty) in one call agree bitwise with the
    device path; a bad buffer in any batch is refused before anything is enqueued."""
    ns, bs = [7, 64, 30, 12], [21, 40, 0, 9]
    A = [torch.from_numpy(wl.covariance(max(b, 1), n, seed=700 + n))[:b].contiguous().pin_memory()
         for n, b in zip(ns, bs)]
    W = [torch.full((b, n), -7.0).pin_memory() for n, b in zip(ns, bs)]
    V = [torch.full((b, n, n), -7.0).pin_memory() for n, b in zip(ns, bs)]
    I = [torch.full((b,), -1, dtype=torch.int32).pin_memory() for b in bs]
    side = [torch.cuda.Stream() for _ in range(2)]
    cur = torch.cuda.current_stream()
    args = lambda Wp: ([t.data_ptr() for t in A], Wp, [t.data_ptr() for t in V], [t.data_ptr() for t in I])
    pageable = np.zeros(40 * 64, dtype=np.float32)
    bad = [t.data_ptr() for t in W]
    bad[1] = pageable.ctypes.data
    assert B.bed_eigh_many_f32_pinned(ns, bs, *args(bad), None, cur.cuda_stream,
                                      [s.cuda_stream for s in side]) == B.BED_ERR_INVALID_ARG
    two = [x[:2] for x in args([t.data_ptr() for t in W])]
    assert B.bed_eigh_many_f32_pinned([7, 65], [1, 1], *two, None, cur.cuda_stream,
                                      [s.cuda_stream for s in side]) == B.BED_ERR_UNSUPPORTED_N
    torch.cuda.synchronize()
    assert all(bool((w == -7.0).all()) for w in W)  # nothing ran
    assert B.bed_eigh_many_f32_pinned(ns, bs, *args([t.data_ptr() for t in W]), None, cur.cuda_stream,
                                      [s.cuda_stream for s in side]) == B.BED_OK
    cur.synchronize()
    live = sum(1 for b in bs if b)  # batches that launch, side by side on the two streams
    for k, (n, b) in enumerate(zip(ns, bs)):
        if b == 0:
            continue
        Wg, Vg, ig = run_gpu(A[k].numpy(), B.concurrent_params(None, n, live))
        assert np.array_equal(W[k].numpy(), Wg) and np.array_equal(V[k].numpy(), Vg)
        assert np.array_equal(I[k].numpy(), ig)
    assert B.bed_eigh_many_f32_pinned([], [], [], [], [], None, None, cur.cuda_stream, []) == B.BED_OK


def test_many_async_in_flight_matches_synchronous():
    """Several batched_eigh_many_async calls in flight (more than the stream slots), waited in any
    order, give the synchronous results bitwise."""
    calls = [[torch.from_numpy(wl.covariance(30 + 7 * c, n, seed=800 + 10 * c + n)) for n in (64, 20, 33)]
             for c in range(4)]
    pend = [B.batched_eigh_many_async(m) for m in calls]
    dropped = B.batched_eigh_many_async(calls[0])
    del dropped  # an unfinished call that is dropped waits for its work
    for c in (2, 0, 3, 1):
        got = pend[c].wait(return_info=True)
        ref = B.batched_eigh_many(calls[c], return_info=True)
        for (W, V, i), (W2, V2, i2) in zip(got, ref):
            assert torch.equal(W, W2) and torch.equal(V, V2) and torch.equal(i, i2)
            assert int((i != 0).sum()) == 0


def test_uniform_workload_end_to_end_path_at_full_size():
    """The benchmark's end-to-end configuration: the uniform workload (512 matrices at each of
    n = 16, 32, 48, 64) from page-locked host memory through batched_eigh_many_async with two calls in
    flight; every result equals the device path (with the parameters a batch gets beside the others)
    bitwise, and a sample of each size matches the oracle."""
    sizes = (16, 32, 48, 64)
    host = [torch.from_numpy(wl.covariance(512, n)).pin_memory() for n in sizes]
    p1 = B.batched_eigh_many_async(host)
    p2 = B.batched_eigh_many_async(host)
    r1 = p1.wait(return_info=True)
    r2 = p2.wait(return_info=True)
    rng = np.random.default_rng(5)
    for n, A, (W, V, info), (W2, V2, info2) in zip(sizes, host, r1, r2):
        Wd, Vd, infod = run_gpu(A.numpy(), B.concurrent_params(None, n, len(sizes)))
        assert np.array_equal(W.numpy(), Wd) and np.array_equal(V.numpy(), Vd) and np.array_equal(info.numpy(), infod)
        assert torch.equal(W, W2) and torch.equal(V, V2)
        idx = np.sort(rng.choice(512, 24, replace=False))
        An = A.numpy()[idx]
        Wo, Vo = run_oracle(An)
        assert_parity(An, W.numpy()[idx], V.numpy()[idx], info.numpy()[idx], Wo, Vo, f"end-to-end path n={n}")


@pytest.mark.parametrize("chunks", [0, 2])
def test_many_batches_host_copy_path(chunks):
    """batched_eigh_many on host tensors through the copy-engine entry point (host_chunks > 0) agrees
    bitwise with the zero-copy default."""
    mats = [torch.from_numpy(wl.covariance(33, n, seed=90 + n)) for n in (64, 9, 40)]
    a = B.batched_eigh_many(mats, return_info=True)
    c = B.batched_eigh_many(mats, return_info=True, host_chunks=max(chunks, 1))
    for (W, V, i), (W2, V2, i2) in zip(a, c):
        assert torch.equal(W, W2) and torch.equal(V, V2) and torch.equal(i, i2)


# ------------------------------------------------- merge products on the tensor cores (split-3xTF32)


@pytest.mark.parametrize("leaf", [1, 2, 8])
def test_tensor_core_merges_every_n(leaf):
    """merge_tensor_cores = 1: every n (all four team sizes; with leaf 1 the deepest level of a large
    matrix has more tiles than the registers hold and takes the FP32 products) within the tolerance."""
    p = B.make_params(leaf_size=leaf, merge_tensor_cores=1)
    for n in range(1, 65):
        A = np.concatenate([wl.covariance(3, n, seed=9400 + n), wl.known_spectrum(2, n, seed=9500 + n)[0]])
        W, V, info = run_gpu(A, p)
        Wo, Vo = run_oracle(A)
        assert_parity(A, W, V, info, Wo, Vo, f"tensor-core merges leaf={leaf} n={n}")


@pytest.mark.parametrize("n", [16, 32, 48, 64])
def test_tensor_core_merges_uniform_workload(n):
    A = wl.covariance(512, n)
    W, V, info = run_gpu(A, B.make_params(merge_tensor_cores=1))
    Wo, Vo = run_oracle(A)
    assert_parity(A, W, V, info, Wo, Vo, f"tensor-core merges covariance 512 x {n}")


@pytest.mark.parametrize("name", ["zero", "identity", "diagonal", "repeated", "rank_one", "block_diagonal", "toeplitz"])
def test_tensor_core_merges_degenerate_inputs(name):
    for n in (3, 9, 17, 37, 64):
        A = wl.special_cases(n)[name][None].repeat(2, axis=0)
        W, V, info = run_gpu(A, B.make_params(merge_tensor_cores=1))
        Wo, Vo = run_oracle(A)
        assert_parity(A, W, V, info, Wo, Vo, f"tensor-core merges {name} n={n}")


@pytest.mark.parametrize("n", [5, 16, 40, 64])
def test_power_of_two_scaling_is_exact(n):
    """The kernel scales every matrix by a power of two before solving and back after: A 2^e gives
    exactly W 2^e and the same V, over the whole exponent range."""
    A = wl.covariance(8, n, seed=55)
    W0, V0, i0 = run_gpu(A)
    for e in (-100, -60, 60, 120):  # inputs and results stay in the normal range
        W, V, info = run_gpu((A * np.float32(2.0 ** e)).astype(np.float32))
        assert np.all(info == 0)
        assert np.array_equal(W, W0 * np.float32(2.0 ** e)) and np.array_equal(V, V0)


def test_large_and_small_magnitudes_hold_tolerance():
    for s in (1e-30, 1e30):
        A = (wl.covariance(8, 48, seed=56).astype(np.float64) * s).astype(np.float32)
        W, V, info = run_gpu(A)
        Wo, Vo = run_oracle(A)
        assert_parity(A, W, V, info, Wo, Vo, f"scale {s}")



# ----------------------------------------------------------------------------- bounded staging wait


@pytest.mark.parametrize("n", [16, 64])
def test_staging_wait_limit_zero_flags_timeout_and_outputs_nan(n):
    """With a staging wait limit of 0 the team gives up on the bulk copy without polling it: every
    matrix reports BED_INFO_TIMEOUT with NaN outputs, and the copy is drained before the block moves on
    (the same launch with the default limit right after gives correct results)."""
    A = wl.covariance(4, n, seed=31)  # even n and a 16-byte aligned buffer: the bulk-copy staging path
    W, V, info = run_gpu(A, B.make_params(stage_wait_us=0))
    assert np.all(info == B.BED_INFO_TIMEOUT), info
    assert np.all(np.isnan(W)) and np.all(np.isnan(V))
    W2, V2, info2 = run_gpu(A)
    Wo, Vo = run_oracle(A)
    assert_parity(A, W2, V2, info2, Wo, Vo, "default staging wait after a timed-out launch")


def test_staging_wait_limit_zero_in_the_persistent_kernel_reaches_every_matrix():
    """The ragged kernel's teams solve many matrices each: after a timed-out (but drained) copy a team
    keeps taking work, so every matrix is reached and flagged, none is left unwritten."""
    mats, ns = wl.ragged(300, nmin=2, nmax=64, seed=77)
    even = [k for k in range(len(ns)) if ns[k] % 2 == 0]
    mats = [mats[k] for k in even]
    ns = [ns[k] for k in even]
    rb = B.RaggedBatch(ns, params=B.make_params(stage_wait_us=0)).load(mats)
    rb.info.fill_(-1)
    rb.solve()
    torch.cuda.synchronize()
    info = rb.info.cpu().numpy()[: rb.count]
    assert np.all(info == B.BED_INFO_TIMEOUT), np.unique(info)
    assert torch.isnan(rb.W[: sum(ns)]).all()


def test_staging_wait_limit_is_validated():
    A = torch.zeros(1, 4, 4, device="cuda")
    for bad in (-1, 60000001):
        st = B.bed_eigh_f32(A.data_ptr(), A.data_ptr() + 64, A.data_ptr() + 128, None, 1, 4,
                            B.make_params(stage_wait_us=bad), torch.cuda.current_stream().cuda_stream)
        assert st == B.BED_ERR_INVALID_ARG
