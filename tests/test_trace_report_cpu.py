"""The trace breakdown (paper_1507_01926_gb300.trace_report) on hand-made traces: every round and level lands in
the bucket of its size, and the bucket sums add up to the totals."""
import numpy as np
import pytest

from paper_1507_01926_gb300 import trace_report as T


def test_breakdown_buckets_and_totals():
    live = np.array([1, 7, 8, 100, 5000, 5000, 300000], np.int32)
    rns = np.array([1000, 2000, 3000, 4000, 5000, 7000, 100000], np.int32)
    lv = np.array([1, 70000], np.int32)
    lns = np.array([9000, 30000], np.int32)
    b = T.breakdown(live, rns, lv, lns)
    assert b["rounds"] == 7 and b["levels"] == 2
    assert b["round_ms"] == pytest.approx(0.122) and b["level_ms"] == pytest.approx(0.039)
    rows = {tuple(r["live"]): r for r in b["rounds_by_live"]}
    assert rows[(0, 8)]["count"] == 2 and rows[(0, 8)]["ms"] == pytest.approx(0.003)
    assert rows[(8, 64)]["count"] == 1 and rows[(64, 256)]["count"] == 1
    assert rows[(4096, 16384)]["count"] == 2 and rows[(4096, 16384)]["us_mean"] == pytest.approx(6.0)
    assert rows[(262144, 1 << 31)]["count"] == 1
    assert sum(r["count"] for r in b["rounds_by_live"]) == 7
    assert sum(r["ms"] for r in b["rounds_by_live"]) == pytest.approx(b["round_ms"])
    lrows = {tuple(r["frontier"]): r for r in b["levels_by_frontier"]}
    assert lrows[(0, 8)]["us_mean"] == pytest.approx(9.0) and lrows[(65536, 262144)]["count"] == 1


def test_breakdown_rejects_mismatched_lengths():
    with pytest.raises(ValueError):
        T.breakdown([1, 2], [10], [], [])
