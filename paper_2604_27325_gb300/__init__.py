"""Batched divide-and-conquer symmetric eigendecomposition for small FP32 matrices on GB300."""
