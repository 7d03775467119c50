"""Comparison of the CUDA path with the FP64 oracle, in the tolerances the eigensolver is held to.

Per matrix, with |A|_2 = max |lambda| of the oracle (FP64, on the exact FP32 input):
  eigenvalues   |W_gpu - W_oracle|_inf           <= 1e-5 |A|_2
  residual      |A V - V diag(W)|_F / |A|_2      <= 1e-5 n        (FP64 arithmetic on FP32 results)
  orthogonality |V^T V - I|_F                    <= 1e-5 n
  vectors       for an eigenvalue whose gap to the rest of the spectrum is >= 1e-3 |A|_2... (gap_j):
                min_s |v_gpu,j - s v_oracle,j|_2 <= 1e-5 n |A|_2 / gap_j (Davis-Kahan scaling);
                clusters closer than that are compared through their spectral projectors.
The vector bound reads the requirement "eigenvectors agree up to sign on spectra with gaps >= 1e-3"
with the perturbation theory of the FP32 backward error.
"""
from __future__ import annotations

import os

import numpy as np

TOL = 1e-5

# worst ratios seen per test function in this session (printed by the terminal summary in conftest.py)
MARGINS: dict = {}


def compare(A, W, V, Wo, Vo, gap_floor=1e-3):
    """Returns a dict of worst-case ratios (measured / allowed), every one of which must be <= 1, and
    under "vec_raw" the largest raw distance min_s |v_gpu,j - s v_oracle,j|_2 over the eigenvalues with
    a gap >= gap_floor |A|_2 (0 when there is none)."""
    A = np.asarray(A, np.float64)
    W = np.asarray(W, np.float64)
    V = np.asarray(V, np.float64)
    b, n, _ = A.shape
    out = {"eig": 0.0, "res": 0.0, "orth": 0.0, "vec": 0.0, "proj": 0.0, "vec_raw": 0.0}
    for k in range(b):
        nrm = max(np.abs(Wo[k]).max(), np.finfo(np.float64).tiny)
        eig = np.abs(W[k] - Wo[k]).max() / (TOL * nrm)
        res = np.linalg.norm(A[k] @ V[k] - V[k] * W[k][None, :]) / nrm / (TOL * n)
        orth = np.linalg.norm(V[k].T @ V[k] - np.eye(n)) / (TOL * n)
        out["eig"] = max(out["eig"], eig)
        out["res"] = max(out["res"], res)
        out["orth"] = max(out["orth"], orth)
        # clusters of the oracle spectrum at separation gap_floor * |A|_2
        w = Wo[k]
        start = 0
        for j in range(1, n + 1):
            if j == n or w[j] - w[j - 1] >= gap_floor * nrm:
                idx = np.arange(start, j)
                lo_gap = w[start] - w[start - 1] if start > 0 else np.inf
                hi_gap = w[j] - w[j - 1] if j < n else np.inf
                gap = min(lo_gap, hi_gap)
                if gap == np.inf:  # the whole spectrum is one cluster: nothing to compare
                    start = j
                    continue
                allowed = TOL * n * nrm / gap
                if len(idx) == 1:
                    c = idx[0]
                    d = min(np.linalg.norm(V[k][:, c] - Vo[k][:, c]), np.linalg.norm(V[k][:, c] + Vo[k][:, c]))
                    out["vec"] = max(out["vec"], d / allowed)
                    out["vec_raw"] = max(out["vec_raw"], d)
                else:
                    P1 = V[k][:, idx] @ V[k][:, idx].T
                    P2 = Vo[k][:, idx] @ Vo[k][:, idx].T
                    out["proj"] = max(out["proj"], np.linalg.norm(P1 - P2, 2) / allowed)
                start = j
    return out


def record(r: dict, n: int) -> None:
    """Keeps the worst ratios of the running test (keyed by its function name)."""
    cur = os.environ.get("PYTEST_CURRENT_TEST", "outside a test").split(" ")[0]
    key = cur.split("::")[-1].split("[")[0]
    m = MARGINS.setdefault(key, {"checks": 0, "max_n": 0})
    m["checks"] += 1
    m["max_n"] = max(m["max_n"], n)
    for k, v in r.items():
        m[k] = max(m.get(k, 0.0), v)


def assert_parity(A, W, V, info, Wo, Vo, what=""):
    r = compare(A, W, V, Wo, Vo)
    record(r, np.asarray(A).shape[-1])
    bad = {k: v for k, v in r.items() if k != "vec_raw" and not (v <= 1.0)}
    assert not bad, f"{what}: tolerance exceeded (ratio measured/allowed): {bad}"
    info = np.asarray(info)
    assert np.all(info == 0), f"{what}: info flags {np.unique(info)}"
    return r
