"""Batched divide-and-conquer symmetric eigendecomposition for small FP32 matrices on GB300 (sm_103a).

The compute path is the CUDA library ``libbed.so`` (C ABI in ``include/bed.h``); :mod:`.binding`
marshals arguments to it. Importing this package loads nothing; the library is loaded (and built if
needed) on first use.
"""


def __getattr__(name):
    if name in ("batched_eigh", "batched_eigh_many", "batched_eigh_many_async", "batched_eigh_ragged", "eigh",
                "make_params", "BedError"):
        from . import binding

        return getattr(binding, name)
    raise AttributeError(name)
