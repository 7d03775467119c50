"""The C ABI library loads, exports what include/bed.h declares, and validates arguments (CPU only).

No call here reaches the GPU: every bed_eigh_f32 call below is rejected by argument validation (or
has batch == 0) before anything is enqueued.
"""
import ctypes as C
import os
import re

import pytest

from paper_2604_27325_gb300 import binding as B

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "bed.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bed_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = B.lib()
    names = declared_functions()
    assert names, "no declarations parsed"
    for name in names:
        assert hasattr(L, name), name
    assert sorted(B.EXPORTED) == names


def test_library_exports_only_the_declared_functions():
    """The dynamic symbol table holds exactly the functions of include/bed.h: everything else (kernel
    stubs, template instantiations and their function-local statics) is local to the library."""
    import shutil
    import subprocess

    from paper_2604_27325_gb300 import build

    nm = shutil.which("nm")
    if nm is None:
        pytest.skip("nm is not installed")
    B.lib()
    out = subprocess.run([nm, "-D", "--defined-only", build.LIB], capture_output=True, text=True, check=True).stdout
    names = sorted(line.split()[-1] for line in out.splitlines() if line.strip())
    assert names == declared_functions()


def test_constants_and_strings():
    assert B.bed_max_n() == 64
    assert B.bed_status_string(B.BED_OK) == "BED_OK"
    assert B.bed_status_string(B.BED_ERR_UNSUPPORTED_N) == "BED_ERR_UNSUPPORTED_N"
    assert B.bed_status_string(99) == "BED_UNKNOWN_STATUS"
    assert C.sizeof(B.bed_counters) == 32
    p = B.bed_default_params()
    assert (p.leaf_size, p.k_multisection, p.retire_by_vote, p.threads_per_matrix) == (0, 4, 1, 0)
    assert p.merge_tensor_cores == 0 and p.matrices_per_cta == 0 and p.n_bisect_first == 1
    assert p.section_rel_eps == 2.0**-1


FAKE = 1 << 20  # aligned, never dereferenced: every call below is rejected before a launch


@pytest.mark.parametrize("n", [0, -1, 65, 1000])
def test_unsupported_n(n):
    assert B.bed_eigh_f32(FAKE, FAKE, FAKE + 4096, None, 4, n) == B.BED_ERR_UNSUPPORTED_N


def test_invalid_arguments_rejected_before_launch():
    assert B.bed_eigh_f32(FAKE, FAKE, FAKE + 4096, None, -1, 8) == B.BED_ERR_INVALID_ARG
    assert B.bed_eigh_f32(0, FAKE, FAKE, None, 3, 8) == B.BED_ERR_INVALID_ARG
    assert B.bed_eigh_f32(FAKE, 0, FAKE, None, 3, 8) == B.BED_ERR_INVALID_ARG
    assert B.bed_eigh_f32(FAKE, FAKE, 0, None, 3, 8) == B.BED_ERR_INVALID_ARG
    assert B.bed_eigh_f32(FAKE + 2, FAKE, FAKE + 4096, None, 3, 8) == B.BED_ERR_INVALID_ARG  # misaligned
    assert B.bed_eigh_f32(FAKE, FAKE, FAKE + 4096, FAKE + 1, 3, 8) == B.BED_ERR_INVALID_ARG
    assert B.bed_eigh_f32(FAKE, FAKE, FAKE, None, 3, 8) == B.BED_ERR_INVALID_ARG  # V aliases A
    assert B.bed_eigh_f32_counted(FAKE, FAKE, FAKE + 4096, None, 3, 8, None, 0) == B.BED_ERR_INVALID_ARG


def test_empty_batch_is_ok_without_launch():
    assert B.bed_eigh_f32(0, 0, 0, None, 0, 8) == B.BED_OK


@pytest.mark.parametrize(
    "field,value",
    [("leaf_size", 9), ("leaf_size", -1), ("k_multisection", 1), ("max_halley_iters", 0),
     ("max_section_iters", -1), ("section_rel_eps", 0.0), ("section_rel_eps", 1.0), ("stop_c", 0.5),
     ("deflation_tol_scale", 0.0), ("retire_by_vote", 2), ("threads_per_matrix", 100),
     ("merge_tensor_cores", 2), ("merge_tensor_cores", -1), ("matrices_per_cta", -1),
     ("matrices_per_cta", (1 << 20) + 1), ("n_bisect_first", 0), ("n_bisect_first", 65)],
)
def test_bad_params(field, value):
    p = B.make_params(**{field: value})
    assert B.bed_eigh_f32(FAKE, FAKE, FAKE + 4096, None, 3, 8, p) == B.BED_ERR_INVALID_ARG


@pytest.mark.parametrize("leaf", [1, 2, 3, 5, 8])
def test_divide_tree_plan(leaf):
    """Sec. 2.1 divide tree: split at floor(s/2) down to <= leaf rows; children merge before parents."""
    for n in range(1, 65):
        merges = B.bed_plan_describe(n, leaf)
        # leaves = maximal blocks never split
        splits = {(lo, hi): mid for lo, mid, hi, _ in merges}
        lvl = {(lo, hi): L for lo, _, hi, L in merges}
        nleaves = 0

        def walk(lo, hi):
            nonlocal nleaves
            if hi - lo <= leaf:
                assert (lo, hi) not in splits
                nleaves += 1
                return -1
            mid = splits[(lo, hi)]
            assert mid == lo + (hi - lo) // 2
            l1, l2 = walk(lo, mid), walk(mid, hi)
            assert lvl[(lo, hi)] > max(l1, l2)
            return lvl[(lo, hi)]

        walk(0, n)
        assert len(merges) == nleaves - 1
        assert [m[3] for m in merges] == sorted(m[3] for m in merges)  # deepest level first
    with pytest.raises(ValueError):
        B.bed_plan_describe(65)
    with pytest.raises(ValueError):
        B.bed_plan_describe(8, 9)
    with pytest.raises(ValueError):
        B.bed_plan_describe(8, -1)
    # leaf size 0: the automatic choice, a tree with leaves of at most 8 rows that every n has
    for n in (2, 16, 33, 48, 64):
        auto = B.bed_plan_describe(n, 0)
        assert any(auto == B.bed_plan_describe(n, leaf) for leaf in (2, 4, 8))


def test_no_cpu_fallback():
    import torch

    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(B.BedError):
        B.batched_eigh(torch.eye(4).unsqueeze(0))


def test_ragged_validation_before_launch():
    ws = B.bed_eigh_ragged_workspace_size(10)
    assert ws >= 64 + 40 and ws % 256 == 0
    assert B.bed_eigh_ragged_workspace_size(0) >= 64
    args = dict(A_ptr=FAKE, offsets_ptr=FAKE, ns_ptr=FAKE, count=10, W_ptr=FAKE, w_offsets_ptr=FAKE,
                V_ptr=FAKE + 4096, info_ptr=None, params=None, tuning=None, workspace_ptr=FAKE, workspace_bytes=ws)
    assert B.bed_eigh_ragged_f32(**{**args, "count": 0}) == B.BED_OK
    assert B.bed_eigh_ragged_f32(**{**args, "count": -1}) == B.BED_ERR_INVALID_ARG
    assert B.bed_eigh_ragged_f32(**{**args, "workspace_bytes": ws - 1}) == B.BED_ERR_INVALID_ARG
    assert B.bed_eigh_ragged_f32(**{**args, "workspace_ptr": FAKE + 8}) == B.BED_ERR_INVALID_ARG
    assert B.bed_eigh_ragged_f32(**{**args, "offsets_ptr": FAKE + 4}) == B.BED_ERR_INVALID_ARG
    assert B.bed_eigh_ragged_f32(**{**args, "ns_ptr": 0}) == B.BED_ERR_INVALID_ARG
    assert B.bed_eigh_ragged_f32(**{**args, "V_ptr": FAKE}) == B.BED_ERR_INVALID_ARG
    t = B.bed_ragged_default_tuning()
    assert [t.team[n] for n in (1, 16, 17, 32, 33, 48, 49, 64)] == [2, 2, 1, 1, 4, 4, 0, 0]
    t.team[20] = 2  # a 64-thread team (n <= 16) cannot hold n = 20
    assert B.bed_eigh_ragged_f32(**{**args, "tuning": t}) == B.BED_ERR_INVALID_ARG
    t = B.bed_ragged_default_tuning()
    t.team[49] = 4  # the 192-thread team holds n <= 48
    assert B.bed_eigh_ragged_f32(**{**args, "tuning": t}) == B.BED_ERR_INVALID_ARG
    t = B.bed_ragged_default_tuning()
    t.team[7] = 5  # no such team type
    assert B.bed_eigh_ragged_f32(**{**args, "tuning": t}) == B.BED_ERR_INVALID_ARG
    t = B.bed_ragged_default_tuning()
    t.leaf[5] = 9
    assert B.bed_eigh_ragged_f32(**{**args, "tuning": t}) == B.BED_ERR_INVALID_ARG


def test_host_entry_points_validate_before_touching_the_device():
    """Argument errors of the page-locked host entry points come back before any CUDA call."""
    assert B.bed_eigh_f32_pinned(FAKE, FAKE, FAKE + 4096, None, 3, 65) == B.BED_ERR_UNSUPPORTED_N
    assert B.bed_eigh_f32_pinned(FAKE, FAKE, FAKE + 4096, None, -1, 8) == B.BED_ERR_INVALID_ARG
    assert B.bed_eigh_f32_pinned(FAKE, FAKE, FAKE + 4096, None, 3, 8, B.make_params(leaf_size=9)) == B.BED_ERR_INVALID_ARG
    assert B.bed_eigh_f32_pinned(0, 0, 0, None, 0, 8) == B.BED_OK
    L = B.lib()
    assert L.bed_eigh_many_f32_pinned(-1, None, None, None, None, None, None, None, None, None, 0) == B.BED_ERR_INVALID_ARG
    assert L.bed_eigh_many_f32_pinned(0, None, None, None, None, None, None, None, None, None, 0) == B.BED_OK
    assert L.bed_eigh_many_f32_pinned(2, None, None, None, None, None, None, None, None, None, 1) == B.BED_ERR_INVALID_ARG
    # sizes and counts are checked batch by batch before any buffer is looked at
    args = ([FAKE], [FAKE], [FAKE + 4096], None, None, 0, [0])
    assert B.bed_eigh_many_f32_pinned([65], [3], *args) == B.BED_ERR_UNSUPPORTED_N
    assert B.bed_eigh_many_f32_pinned([8], [-2], *args) == B.BED_ERR_INVALID_ARG
    assert B.bed_eigh_many_f32_pinned([8], [3], [FAKE], [FAKE], [FAKE + 4096], None,
                                      B.make_params(merge_tensor_cores=3), 0, [0]) == B.BED_ERR_INVALID_ARG


def test_async_api_has_no_cpu_path():
    import torch

    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(B.BedError):
        B.batched_eigh_many_async([torch.eye(4).unsqueeze(0)])
    with pytest.raises(B.BedError):
        B.batched_eigh_many([torch.eye(4).unsqueeze(0)])



def test_team_shape_rule_and_concurrent_params():
    """The threads-per-matrix rule of bed.h, and the 64-thread teams for n = 17..32 in a concurrent mix."""
    from paper_2604_27325_gb300 import autotune

    assert [B.team_threads(n) for n in (1, 16, 17, 32, 33, 48, 49, 64)] == [64, 64, 128, 128, 192, 192, 128, 128]
    assert B.team_threads(64, B.make_params(merge_tensor_cores=1)) == 256
    assert B.team_threads(20, B.make_params(threads_per_matrix=64)) == 64
    t = B.bed_ragged_default_tuning()
    for n in range(1, 65):
        p = autotune.uniform_params(n, t, concurrent=True)
        assert p.threads_per_matrix == (64 if 16 < n <= 32 else 0)
        assert p.leaf_size == t.leaf[n]
        assert autotune.uniform_params(n, t).threads_per_matrix == 0
