"""Autotuner host logic: coordinate descent, the persisted table and its lookup (no GPU)."""

import json
import math

from paper_1803_08333_gb300 import autotune as at


def test_coordinate_descent_finds_the_separable_minimum():
    # cost separable in the knobs: the minimum is at gemv_chunk=2048, gemm_bn=64
    cost = {"gemv_chunk": {0: 3.0, 256: 5.0, 1024: 3.0, 2048: 1.0}, "gemm_bn": {0: 2.0, 32: 4.0, 64: 0.5, 128: 2.5}}
    calls = []

    def measure(plan):
        calls.append(dict(plan))
        return sum(cost[k][plan.get(k, 0)] for k in cost)

    plan, ms, tried = at.coordinate_descent(measure, [("gemv_chunk", (256, 1024, 2048)), ("gemm_bn", (32, 64, 128))])
    assert plan == {"gemv_chunk": 2048, "gemm_bn": 64}
    assert ms == 1.5
    assert tried["default"] == 5.0 and tried["gemv_chunk=256"] == 7.0
    assert len(calls) == 1 + 3 + 3


def test_coordinate_descent_skips_invalid_candidates():
    def measure(plan):
        return math.inf if plan.get("gemm_bn") == 128 else 1.0 + (plan.get("gemm_bn", 0) == 32)

    plan, ms, _ = at.coordinate_descent(measure, [("gemm_bn", (32, 128))])
    assert plan == {} and ms == 1.0


def _table():
    t = at.Table("NVIDIA GB300")
    for n in (1920, 30720):
        for nr in (1, 16, 512):
            t.add(at.Entry(n, nr, "mixed", {"gemv_chunk": 256 * (nr % 7 + 1), "mrhs_min": 1 if nr >= 16 else 65536},
                           0.1 * nr, 0.2 * nr, {}))
    t.add(at.Entry(1920, 1, "ff", {"gemv_chunk": 4096}, 1.0, 1.0, {}))
    return t


def test_lookup_takes_the_nearest_size_then_the_nearest_column_count():
    t = _table()
    assert t.lookup(2000, 1)["gemv_chunk"] == 512       # n -> 1920, nrhs 1
    assert t.lookup(20000, 20)["mrhs_min"] == 1          # n -> 30720, nrhs -> 16
    assert t.lookup(20000, 3)["mrhs_min"] == 65536       # nrhs 3 is nearer 1 than 16 on a log scale
    assert t.lookup(30720, 4096)["gemv_chunk"] == 256 * (512 % 7 + 1)
    assert t.lookup(30720, 1, "ff")["gemv_chunk"] == 4096  # only n=1920 has ff entries
    assert at.Table("x").lookup(10, 1) is None


def test_table_round_trip_and_device_match(tmp_path):
    t = _table()
    t.add(at.Entry(1920, 1, "mixed", {"gemv_chunk": 1024}, 0.05, 0.1, {"default": 0.1}))  # replaces the old one
    assert sum(1 for e in t.entries if (e.n, e.nrhs, e.precision) == (1920, 1, "mixed")) == 1
    path = tmp_path / (at.device_slug("NVIDIA GB300") + ".json")
    t.save(str(path))
    d = json.loads(path.read_text())
    assert d["device"] == "NVIDIA GB300" and len(d["entries"]) == len(t.entries)
    u = at.Table.for_device("NVIDIA GB300", str(tmp_path))
    assert u is not None and u.lookup(1920, 1) == {"gemv_chunk": 1024}
    assert at.Table.for_device("NVIDIA B200", str(tmp_path)) is None
    assert at.device_slug("NVIDIA GB300") == "nvidia_gb300"
