"""Autotuning on the GPU (mf_autotune, mf_batch_autotune, mf_set_options): the tuned options must give the
oracle's flow value and minimal source-side cut, every chosen field must come from the candidate table of
include/mf.h, a tiny time budget must leave the starting options, and the JSON cache must round-trip."""
import numpy as np
import pytest

import oracle
from paper_1507_01926_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CANDIDATES = {"gr_time_ratio": {0.0, 1.0, 2.0, 4.0}, "gr_freq": {0.25, 0.5, 1.0, 2.0}, "bin_thread": {2, 4, 8, 16},
              "bin_warp": {128, 1024, 8192}, "kernel_variant": {0, 1, 2, 3, 4}, "local_lists": {0, 1},
              "bfs_hops": {1, 4, 8, 16}, "bfs_pull": {0, 20, 50, 200}}
SHAPES = {(256, 2), (512, 1), (128, 4), (256, 1), (64, 4)}


def check_solution(mf, g, csr, r):
    ref = oracle.maxflow(g.n, g.s, g.t, g.tail, g.head, g.cap, want_flow=False)
    cut = mf.cut_bits_to_bool(r.cut_bits, g.n)
    assert r.value == ref["value"], g.name
    assert np.array_equal(cut, ref["cut"]), g.name
    f_in = np.where(csr.arc_slot >= 0, r.flow[np.maximum(csr.arc_slot, 0)], 0).astype(np.int64)
    assert not oracle.check_flow(g.n, g.s, g.t, g.tail, g.head, g.cap, f_in, r.value, cut), g.name


def in_table(mf, o, start):
    d, s = mf.options_to_dict(o), mf.options_to_dict(start)
    for k, vals in CANDIDATES.items():
        assert d[k] == s[k] or d[k] in vals, k
    assert (d["block_threads"], d["blocks_per_sm"]) == (s["block_threads"], s["blocks_per_sm"]) or \
        (d["block_threads"], d["blocks_per_sm"]) in SHAPES
    for k in ("gr_alpha", "work_beta", "max_rounds", "timeout_ms", "cut_only", "device", "simple_rounds"):
        assert d[k] == s[k], k


@pytest.mark.parametrize("which", ["grid", "rmat"])
def test_tuned_options_solve_exactly(gpu, which):
    g = I.grid2d(90, 70, 71) if which == "grid" else I.rmat(13, 8, 72)
    csr = gpu.build_csr(g.n, g.tail, g.head, g.cap)
    start = gpu.default_options()
    with gpu.Graph.from_csr(csr, g.s, g.t, start) as G:
        best, ms = G.autotune(reps=1, sweeps=2)
        assert ms > 0
        in_table(gpu, best, start)
        check_solution(gpu, g, csr, G.solve())
        assert G.stats()["block_threads"] == best.block_threads


def test_tiny_budget_keeps_the_starting_options(gpu):
    g = I.grid2d(40, 40, 73)
    csr = gpu.build_csr(g.n, g.tail, g.head, g.cap)
    start = gpu.default_options(bin_warp=256)
    with gpu.Graph.from_csr(csr, g.s, g.t, start) as G:
        best, ms = G.autotune(reps=1, sweeps=1, time_budget_ms=1e-6)
        assert gpu.options_to_dict(best) == gpu.options_to_dict(start) and ms > 0
        check_solution(gpu, g, csr, G.solve())


def test_set_options_validates_and_keeps_graph_usable(gpu):
    g = I.grid2d(50, 30, 74)
    csr = gpu.build_csr(g.n, g.tail, g.head, g.cap)
    with gpu.Graph.from_csr(csr, g.s, g.t) as G:
        with pytest.raises(gpu.MFError) as e:
            G.set_options(gpu.default_options(block_threads=33))
        assert e.value.code == -1
        with pytest.raises(gpu.MFError):
            G.set_options(gpu.default_options(device=7))
        check_solution(gpu, g, csr, G.solve())
        G.set_options(gpu.default_options(block_threads=128, blocks_per_sm=4, bin_thread=2, gr_time_ratio=0.0))
        assert G.stats()["block_threads"] in (0, 256)  # stats are those of the last solve
        check_solution(gpu, g, csr, G.solve())
        assert G.stats()["block_threads"] == 128


def test_batch_autotune_and_cache(gpu, tmp_path):
    from paper_1507_01926_gb300 import autotune as A

    insts = [I.layered(8 + 3 * k, 40 + 20 * k, 300 + k) for k in range(6)]
    csrs = [gpu.build_csr(g.n, g.tail, g.head, g.cap) for g in insts]
    key = A.workload_key("layered-test", sum(g.n for g in insts), sum(c.m for c in csrs), len(insts))
    path = str(tmp_path / "tune.json")
    with gpu.Batch(csrs, [(g.s, g.t) for g in insts]) as B:
        o1, ms1, hit1 = A.tuned(B, key, path=path, reps=1)
        assert not hit1 and ms1 > 0
        res = B.solve()
    for g, c, r in zip(insts, csrs, res):
        check_solution(gpu, g, c, r)
    with gpu.Batch(csrs, [(g.s, g.t) for g in insts]) as B:
        o2, ms2, hit2 = A.tuned(B, key, path=path)
        assert hit2 and ms2 == ms1 and gpu.options_to_dict(o2) == gpu.options_to_dict(o1)
        res = B.solve()
        assert B.stats()["block_threads"] == o1.block_threads
    for g, c, r in zip(insts, csrs, res):
        check_solution(gpu, g, c, r)
