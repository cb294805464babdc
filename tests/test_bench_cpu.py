"""CPU checks of bench.py's host-side arithmetic: the algorithmic-byte model, the per-phase roofline split,
option overrides, and the sizing of the oracle's bounded CPU-baseline sample (no GPU needed)."""
import argparse
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

STATS = dict(scans_discharge=1000, scans_discharge_residual=700, pushes=100, visits_discharge=50, scans_bfs=400, visits_bfs=30,
             global_relabels=2, discharge_ms=2.0, relabel_ms=1.0)


def test_model_bytes_is_the_sum_of_its_units():
    n, m = 10, 40
    want = (4 * 1000 + 8 * 700 + 28 * 100 + 48 * 50 + 12 * 400 + 16 * 30 + 20 * m + 28 * n + 12 * n * 2)
    assert bench.model_bytes(STATS, n, m) == want


def test_phase_rooflines_split_the_kernel_bytes():
    n = 10
    ph = bench.phase_rooflines(STATS, n, peak=100.0)
    dis, bfs = ph["discharge_rounds"], ph["global_relabel_bfs"]
    assert dis["model_bytes"] == 4 * 1000 + 8 * 700 + 28 * 100 + 48 * 50
    assert bfs["model_bytes"] == 12 * 400 + 16 * 30 + 12 * n * 2
    # GB/s = bytes / (ms * 1e6); frac = that / peak
    assert dis["achieved_GBps"] == pytest.approx(dis["model_bytes"] / 2.0e6)
    assert bfs["frac"] == pytest.approx(bfs["model_bytes"] / 1.0e6 / 100.0)
    # the per-slot and per-vertex fixed costs belong to neither phase
    assert dis["model_bytes"] + bfs["model_bytes"] < bench.model_bytes(STATS, n, 40)
    zero = bench.phase_rooflines(dict(STATS, relabel_ms=0.0), n, peak=100.0)
    assert zero["global_relabel_bfs"]["achieved_GBps"] is None


def test_option_overrides(built):
    from paper_1507_01926_gb300 import mf

    o = mf.default_options()
    bench.apply_overrides(o, argparse.Namespace(options='{"bin_warp": 128, "bfs_hops": 2}'))
    assert (o.bin_warp, o.bfs_hops) == (128, 2)
    with pytest.raises(KeyError):
        bench.apply_overrides(o, argparse.Namespace(options='{"no_such_option": 1}'))
    before = mf.options_to_dict(o)
    bench.apply_overrides(o, argparse.Namespace(options=""))
    assert mf.options_to_dict(o) == before


def test_sized_oracle_sample_stops_near_its_target(built):
    from paper_1507_01926_gb300 import inputs as I

    g = I.grid3d(40, 40, 30, 900)
    r, limit = bench.sized_oracle_run(g, seconds=0.3)
    assert limit >= 20_000_000 or not r["truncated"]
    assert r["seconds"] < 5.0  # the geometric growth never overshoots by much
    assert r["stats"]["scans"] > 0


@pytest.mark.parametrize("which", ["grid", "random", "rmat", "multi"])
def test_paired_slot_count_equals_the_builder(built, which):
    """The reference arm reports the same slot count as the CSR builder without calling the solver library."""
    import numpy as np

    from paper_1507_01926_gb300 import inputs as I
    from paper_1507_01926_gb300 import mf

    if which == "multi":  # parallel and antiparallel multi-arcs and self-loops
        rng = np.random.default_rng(5)
        tail = rng.integers(0, 12, 300).astype(np.int32)
        head = rng.integers(0, 12, 300).astype(np.int32)
        n = 12
        cap = np.ones(300, np.int32)
    else:
        g = {"grid": lambda: I.grid3d(9, 8, 7, 31), "random": lambda: I.random_graph(80, 900, 32),
             "rmat": lambda: I.rmat(9, 8, 33)}[which]()
        n, tail, head, cap = g.n, g.tail, g.head, g.cap
    assert bench.paired_slot_count(tail, head) == mf.build_csr(n, tail, head, cap).m
