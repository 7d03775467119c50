"""The autotuner measures, writes and reloads a per-n table (GPU)."""
import json

import pytest

from paper_2604_27325_gb300 import autotune
from paper_2604_27325_gb300 import binding as B

pytestmark = pytest.mark.gpu


def test_autotune_roundtrip(tmp_path):
    path = str(tmp_path / "t.json")
    out = autotune.tune(ns=[5, 20, 50], batch=128, reps=2, path=path)
    table = json.load(open(path))["table"]
    assert set(table) == {"5", "20", "50"}
    for n, v in out["table"].items():
        assert n <= autotune.TEAM_CAP[v["team"]] and 1 <= v["leaf"] <= 8 and v["us_per_matrix"] > 0
    t = autotune.load(path)
    d = B.bed_ragged_default_tuning()
    for n in (5, 20, 50):
        assert (t.team[n], t.leaf[n]) == (out["table"][n]["team"], out["table"][n]["leaf"])
    assert (t.team[6], t.leaf[6]) == (d.team[6], d.leaf[6])
