"""Autotuner for ragged launches: picks, for every n, the team shape and leaf size by measurement.

For each n the candidates are the team types whose size class holds n (one 256-thread team, two
128-thread, four 64-thread or eight 32-thread teams per block, or one 192-thread team) times three leaf sizes of the divide
tree (Sec. 2.1-2.2: 2x2 leaves, or QL leaves of up to 4 or 8 rows). Each candidate solves a uniform batch of seeded covariance
matrices of that n through the ragged entry point; the fastest per-matrix time wins. Results are kept
as JSON keyed by the GPU's name, and :func:`load` turns them into a ``bed_ragged_tuning``.
"""
from __future__ import annotations

import json
import os
import time

import torch

from . import binding as B
from . import workloads

TEAM_CAP = {0: 64, 1: 32, 2: 16, 3: 16, 4: 48}
HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_DIR = os.path.join(HERE, "tuning")


def _device_key(device=None) -> str:
    name = torch.cuda.get_device_name(device)
    return "".join(c if c.isalnum() else "_" for c in name)


def default_path(device=None) -> str:
    return os.path.join(DEFAULT_DIR, _device_key(device) + ".json")


def _time_candidate(rb: B.RaggedBatch, reps: int) -> float:
    rb.solve()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        rb.solve()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(ns=range(1, 65), batch: int = 2048, reps: int = 10, path: str | None = None, verbose: bool = False):
    """Measure every candidate for every n; write and return the table {n: {team, leaf, us_per_matrix}}."""
    table = {}
    for n in ns:
        A = workloads.covariance(batch, n, seed=7000 + n)
        best = None
        for team, cap in TEAM_CAP.items():
            if n > cap:
                continue
            for leaf in (2, 4, 8):
                t = B.bed_ragged_default_tuning()
                t.team[n], t.leaf[n] = team, leaf
                rb = B.RaggedBatch([n] * batch, tuning=t).load(list(A))
                ms = _time_candidate(rb, reps)
                us = ms * 1e3 / batch
                if verbose:
                    print(f"n={n} team={team} leaf={leaf}: {us:.4f} us/matrix", flush=True)
                if best is None or us < best[2]:
                    best = (team, leaf, us)
        table[n] = {"team": best[0], "leaf": best[1], "us_per_matrix": best[2]}
    out = {"device": torch.cuda.get_device_name(), "sm_count": torch.cuda.get_device_properties(0).multi_processor_count,
           "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()), "batch": batch, "table": table}
    path = path or default_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    return out


def load(path: str | None = None) -> B.bed_ragged_tuning:
    """The tuned table for this GPU if one exists (else the library's built-in choice)."""
    t = B.bed_ragged_default_tuning()
    try:
        path = path or default_path()
        with open(path) as f:
            table = json.load(f)["table"]
    except (OSError, KeyError, ValueError, RuntimeError):
        return t
    for k, v in table.items():
        n = int(k)
        if 1 <= n <= 64 and n <= TEAM_CAP.get(int(v["team"]), 0) and 1 <= int(v["leaf"]) <= 8:
            t.team[n], t.leaf[n] = int(v["team"]), int(v["leaf"])
    return t


TEAM_THREADS = {0: 256, 1: 128, 2: 64, 3: 32, 4: 192}


def uniform_params(n: int, tuning: B.bed_ragged_tuning | None = None, same_team: bool = False,
                   concurrent: bool = False) -> B.bed_params:
    """Parameters of a uniform-size launch (bed_eigh_f32) with the leaf size the tuning table gives size n
    and the uniform kernel's automatic team shape; with ``same_team`` the team shape of the table too,
    so that a uniform launch runs exactly (bitwise) what the ragged kernel would for n. With
    ``concurrent`` (launches of several sizes side by side) sizes 17..32 get 64-thread teams, the choice
    bed_eigh_many_f32_pinned makes for such a mix: half the registers of the automatic 128-thread team,
    so that more of them fit beside the larger sizes' blocks."""
    t = tuning if tuning is not None else load()
    p = B.make_params(threads_per_matrix=TEAM_THREADS[int(t.team[n])] if same_team else 0, leaf_size=int(t.leaf[n]))
    return B.concurrent_params(p, n, 2) if concurrent else p


if __name__ == "__main__":
    import sys

    res = tune(verbose="-v" in sys.argv)
    print(json.dumps({k: (v["team"], v["leaf"], round(v["us_per_matrix"], 4)) for k, v in res["table"].items()}))
