"""GPU solver vs the CPU oracle, through the C-ABI (libmf.so).

The flow value and the minimal source-side cut S_min are unique for a maximum flow (arXiv:1507.01926,
Section 2), so they must match the oracle bit for bit. Per-arc flows are not unique; they are checked
against the definitions (capacity bounds, conservation, no residual s-t path, cut capacity = value).
The labels of a global relabel are exact BFS distances (Algorithm 2), so they must match the oracle's
BFS exactly on the same residual graph.
"""
import numpy as np
import pytest

import oracle
from paper_1507_01926_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def solve_and_compare(mf, g, options=None):
    value, flow, cut, csr, stats = mf.solve_instance(g, options)
    ref = oracle.maxflow(g.n, g.s, g.t, g.tail, g.head, g.cap, want_flow=False)
    assert value == ref["value"], f"{g.name}: value {value} != oracle {ref['value']}"
    assert np.array_equal(cut, ref["cut"]), f"{g.name}: S_min differs in {int((cut != ref['cut']).sum())} vertices"
    bad = oracle.check_flow(g.n, g.s, g.t, g.tail, g.head, g.cap, flow, value, cut)
    assert not bad, f"{g.name}: flow violates {bad}"
    return value, stats


@pytest.mark.parametrize("seed", range(60))
def test_random_small(gpu, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 200))
    m = int(rng.integers(0, 8 * n))
    g = I.random_graph(n, m, 7000 + seed, cap=(0, int(rng.integers(1, 1000))), allow_loops=bool(seed % 3 == 0))
    solve_and_compare(gpu, g)


@pytest.mark.parametrize("seed", range(8))
def test_random_dense_hubs(gpu, seed):
    """Few vertices, many parallel arcs: degrees above the thread and warp bins."""
    g = I.random_graph(12 + seed, 3000 + 500 * seed, 9100 + seed, cap=(1, 100))
    solve_and_compare(gpu, g)


def test_grid2d_64x64(gpu):
    import json
    import os

    g = I.grid2d_64x64()
    value, stats = solve_and_compare(gpu, g)
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "grid2d_64x64.json")))
    assert value == gold["value"]
    assert stats["rounds"] > 0 and stats["global_relabels"] >= 2


@pytest.mark.parametrize("shape", [(97, 131), (40, 300), (256, 256)])
def test_grid2d(gpu, shape):
    solve_and_compare(gpu, I.grid2d(shape[0], shape[1], 11 * shape[0] + shape[1]))


@pytest.mark.parametrize("shape", [(16, 16, 8), (33, 29, 17), (64, 64, 16)])
def test_grid3d(gpu, shape):
    solve_and_compare(gpu, I.grid3d(*shape, seed=sum(shape)))


@pytest.mark.parametrize("scale", [8, 11, 14])
def test_rmat(gpu, scale):
    solve_and_compare(gpu, I.rmat(scale, 16, 500 + scale))


@pytest.mark.parametrize("LW", [(5, 7), (16, 64), (40, 300)])
def test_layered(gpu, LW):
    solve_and_compare(gpu, I.layered(LW[0], LW[1], 77 + LW[0]))


def test_multiframe(gpu):
    solve_and_compare(gpu, I.multiframe(3, 99, side=48))


@pytest.mark.parametrize("bins", [(0, 0), (0, 1 << 30), (8, 8), (2, 40)])
def test_degree_bins_agree(gpu, bins):
    """Forcing every vertex through the CTA, the warp or the thread path gives the same unique results."""
    opt = gpu.default_options(bin_thread=bins[0], bin_warp=bins[1])
    for g in (I.grid2d(30, 40, 5), I.rmat(10, 8, 6), I.random_graph(20, 2000, 8, cap=(1, 50))):
        solve_and_compare(gpu, g, opt)


@pytest.mark.parametrize("variant,bt,bin_thread", [(0, 256, 8), (1, 256, 8), (2, 256, 8), (3, 512, 8), (2, 128, 8),
                                                   (4, 256, 8), (4, 256, 16), (4, 128, 12)])
def test_kernel_variants_agree(gpu, variant, bt, bin_thread):
    """Every register-budget variant of the persistent kernel gives the same unique results (variant 4 also
    with the 16-slot thread path, which the layered graphs' degree-9..16 vertices take)."""
    opt = gpu.default_options(kernel_variant=variant, block_threads=bt, bin_thread=bin_thread)
    for g in (I.grid3d(18, 20, 10, seed=variant), I.rmat(11, 8, 40 + variant), I.grid2d(40, 60, variant),
              I.layered(12, 90, 50 + variant), I.random_graph(60, 700, 60 + variant, cap=(1, 40))):
        solve_and_compare(gpu, g, opt)


@pytest.mark.parametrize("bt", [64, 128, 512])
def test_block_shapes(gpu, bt):
    opt = gpu.default_options(block_threads=bt)
    solve_and_compare(gpu, I.grid3d(20, 18, 9, seed=bt), opt)
    solve_and_compare(gpu, I.rmat(11, 8, bt), opt)


def arcs(lst, n, s, t, name="edge"):
    a = np.array(lst, dtype=np.int64).reshape(-1, 3)
    return I.Instance(n, s, t, a[:, 0].astype(np.int32), a[:, 1].astype(np.int32), a[:, 2].astype(np.int32), name)


EDGE_CASES = {
    "no_arcs": arcs([], 3, 0, 2),
    "direct_st": arcs([(0, 1, 17), (0, 1, 4), (1, 0, 9)], 2, 0, 1),
    "disconnected": arcs([(0, 1, 5), (2, 3, 5)], 4, 0, 3),
    "zero_caps": arcs([(0, 1, 0), (1, 2, 0), (0, 2, 0)], 3, 0, 2),
    "source_isolated": arcs([(1, 2, 5)], 3, 0, 2),
    "sink_unreachable": arcs([(0, 1, 5), (2, 1, 5)], 3, 0, 2),
    "self_loops": arcs([(0, 0, 9), (0, 1, 5), (1, 1, 3), (1, 2, 4)], 3, 0, 2),
    "antiparallel": arcs([(0, 1, 10), (1, 0, 10), (1, 2, 7), (2, 1, 3), (0, 2, 1)], 3, 0, 2),
    "int64_value": arcs([(0, k, 2 ** 30) for k in range(1, 6)] + [(k, 6, 2 ** 30) for k in range(1, 6)], 7, 0, 6),
    "max_pair_capacity": arcs([(0, 1, 2 ** 31 - 2), (1, 0, 1), (1, 2, 2 ** 31 - 1)], 3, 0, 2),
    "sink_is_zero_id": arcs([(2, 1, 4), (1, 0, 3), (2, 0, 2)], 3, 2, 0),
    "long_path": arcs([(k, k + 1, 1000 - k) for k in range(999)], 1000, 0, 999),
    "trapped_excess": arcs([(0, 1, 100), (1, 2, 100), (2, 3, 1), (1, 4, 50), (4, 1, 50)], 5, 0, 3),
}


@pytest.mark.parametrize("name", sorted(EDGE_CASES))
def test_edge_cases(gpu, name):
    solve_and_compare(gpu, EDGE_CASES[name])


def test_star_hub_block_path(gpu):
    """A vertex of degree 20,000 (CTA discharge) between s and t."""
    k = 20000
    lst = [(0, 1, 10 ** 6)] + [(1, 2 + i, 1 + i % 7) for i in range(k)] + [(2 + i, k + 2, 5) for i in range(k)]
    solve_and_compare(gpu, arcs(lst, k + 3, 0, k + 2))


def test_repeated_solves_identical(gpu):
    g = I.grid3d(24, 24, 12, seed=3)
    csr = gpu.build_csr(g.n, g.tail, g.head, g.cap)
    with gpu.Graph.from_csr(csr, g.s, g.t) as G:
        a = G.solve()
        b = G.solve()
    assert a.value == b.value
    assert np.array_equal(a.cut_bits, b.cut_bits)


def test_cut_only_matches(gpu):
    g = I.grid2d(50, 70, 21)
    ref = oracle.maxflow(g.n, g.s, g.t, g.tail, g.head, g.cap, want_flow=False)
    csr = gpu.build_csr(g.n, g.tail, g.head, g.cap)
    with gpu.Graph.from_csr(csr, g.s, g.t, gpu.default_options(cut_only=1)) as G:
        r = G.solve(flow=False)
        with pytest.raises(gpu.MFError):
            G.solve(flow=True)
    assert r.value == ref["value"]
    assert np.array_equal(gpu.cut_bits_to_bool(r.cut_bits, g.n), ref["cut"])


def test_device_api(gpu):
    import torch

    g = I.grid2d(40, 44, 31)
    ref = oracle.maxflow(g.n, g.s, g.t, g.tail, g.head, g.cap, want_flow=False)
    csr = gpu.build_csr(g.n, g.tail, g.head, g.cap)
    dev = torch.device("cuda:0")
    row = torch.from_numpy(csr.row_offsets).to(dev)
    head = torch.from_numpy(csr.head).to(dev)
    cap = torch.from_numpy(csr.cap).to(dev)
    rev = torch.from_numpy(csr.rev).to(dev)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        G = gpu.Graph.from_device(g.n, row, head, cap, rev, g.s, g.t, stream=stream)
        val = torch.zeros(1, dtype=torch.int64, device=dev)
        flow = torch.zeros(csr.m, dtype=torch.int32, device=dev)
        cutw = torch.zeros((g.n + 31) // 32, dtype=torch.int32, device=dev)
        G.solve_device(val, flow, cutw, stream=stream)
    stream.synchronize()
    assert int(val.item()) == ref["value"]
    cut = gpu.cut_bits_to_bool(cutw.cpu().numpy().view(np.uint32), g.n)
    assert np.array_equal(cut, ref["cut"])
    f_in = flow.cpu().numpy()[csr.arc_slot].astype(np.int64)
    assert not oracle.check_flow(g.n, g.s, g.t, g.tail, g.head, g.cap, f_in, ref["value"], cut)
    G.close()


def residual_arcs(csr, res):
    t = csr.tails()
    k = res > 0
    return t[k], csr.head[k]


@pytest.mark.parametrize("rounds", [0, 1, 2, 5, 20])
@pytest.mark.parametrize("which", ["grid3d", "rmat", "random"])
def test_global_relabel_labels_exact(gpu, rounds, which):
    """After k rounds of phase 1, a global relabel on the GPU gives exactly the oracle's BFS distances to
    t over the same residual graph (s never entered, n for unreachable)."""
    g = {"grid3d": I.grid3d(20, 20, 12, seed=4), "rmat": I.rmat(11, 12, 5),
         "random": I.random_graph(300, 2400, 6, cap=(1, 30))}[which]
    csr = gpu.build_csr(g.n, g.tail, g.head, g.cap)
    with gpu.Graph.from_csr(csr, g.s, g.t) as G:
        res, lab, ex, done = G.run_rounds(rounds, final_relabel=True)
    rt, rh = residual_arcs(csr, res)
    d = oracle.sink_distances(g.n, g.s, g.t, rt, rh)
    assert np.array_equal(lab, d), f"{int((lab != d).sum())} labels differ"


@pytest.mark.parametrize("opts", [dict(local_lists=0, bfs_pull=50), dict(local_lists=0, bfs_pull=0),
                                  dict(bfs_hops=1), dict(bfs_hops=8)])
def test_wide_seed_level_labels_and_cut(gpu, opts):
    """The sink of this grid has 528 arcs, more than a CTA of 128 threads: the first level of every BFS from it
    (and of the cut BFS from s) is expanded by the whole grid, and the level loop starts at depth 1. With
    level-synchronous levels (top-down, bottom-up) and label-correcting ones the labels after a global
    relabel must be the oracle's BFS distances, and the solve must give the oracle's value and S_min."""
    g = I.grid3d(24, 22, 10, seed=14)
    csr = gpu.build_csr(g.n, g.tail, g.head, g.cap)
    o = gpu.default_options(block_threads=128, **opts)
    for rounds in (0, 7):
        with gpu.Graph.from_csr(csr, g.s, g.t, o) as G:
            res, lab, _, _ = G.run_rounds(rounds, final_relabel=True)
        rt, rh = residual_arcs(csr, res)
        assert np.array_equal(lab, oracle.sink_distances(g.n, g.s, g.t, rt, rh))
    solve_and_compare(gpu, g, o)


@pytest.mark.parametrize("rounds", [1, 3, 10, 40])
def test_preflow_invariants_mid_solve(gpu, rounds):
    """After any number of rounds: residuals in range, pair sums preserved, and every excess equals the net
    inflow implied by the residuals (a preflow, Section 2.1)."""
    g = I.grid3d(24, 20, 10, seed=rounds)
    csr = gpu.build_csr(g.n, g.tail, g.head, g.cap)
    with gpu.Graph.from_csr(csr, g.s, g.t) as G:
        res, lab, ex, done = G.run_rounds(rounds, final_relabel=False)
    assert (res >= 0).all()
    assert np.array_equal(res.astype(np.int64) + res[csr.rev], csr.cap.astype(np.int64) + csr.cap[csr.rev])
    t = csr.tails()
    net_in = np.zeros(g.n, np.int64)
    np.add.at(net_in, t, res.astype(np.int64) - csr.cap)
    others = np.ones(g.n, bool)
    others[g.s] = False
    assert np.array_equal(net_in[others], ex[others])
    assert (ex[others] >= 0).all()


def test_invalid_graphs_rejected_on_device(gpu):
    row = np.array([0, 1, 2, 2], np.int64)
    head = np.array([1, 0], np.int32)
    cap = np.array([3, 0], np.int32)
    with pytest.raises(gpu.MFError) as e:  # rev[0] points to itself
        gpu.Graph(3, row, head, cap, np.array([0, 0], np.int64), 0, 2)
    assert e.value.code == -1
    with pytest.raises(gpu.MFError) as e:  # head[rev[a]] != tail(a)
        gpu.Graph(3, row, np.array([1, 2], np.int32), cap, np.array([1, 0], np.int64), 0, 2)
    assert e.value.code == -2
    with pytest.raises(gpu.MFError) as e:
        gpu.Graph(3, row, head, np.array([2 ** 31 - 1, 1], np.int32), np.array([1, 0], np.int64), 0, 2)
    assert e.value.code == -4
    with pytest.raises(gpu.MFError) as e:
        gpu.Graph(3, np.array([0, 1, 3, 2], np.int64), head, cap, np.array([1, 0], np.int64), 0, 2)
    assert e.value.code == -1
    with pytest.raises(gpu.MFError) as e:
        gpu.Graph(3, row, head, np.array([-1, 0], np.int32), np.array([1, 0], np.int64), 0, 2)
    assert e.value.code == -1


def test_round_limit_reports_error(gpu):
    g = I.grid2d(30, 30, 2)
    csr = gpu.build_csr(g.n, g.tail, g.head, g.cap)
    with gpu.Graph.from_csr(csr, g.s, g.t, gpu.default_options(max_rounds=2)) as G:
        with pytest.raises(gpu.MFError) as e:
            G.solve()
        assert e.value.code == -7
        # the graph stays usable after an error
    with gpu.Graph.from_csr(csr, g.s, g.t) as G:
        assert G.solve().value == oracle.maxflow(g.n, g.s, g.t, g.tail, g.head, g.cap)["value"]


@pytest.mark.parametrize("hops", [1, 4])
def test_trace_matches_stats(gpu, hops):
    """mf_solve_trace: one entry per round and per BFS level (grid barrier), consistent with the solve's
    counters. With one BFS level per barrier the frontier sizes add up to the expanded vertices; with more,
    CTAs also expand vertices they reached within the level, so the frontiers add up to at most that."""
    g = I.grid3d(30, 30, 16, seed=9)
    csr = gpu.build_csr(g.n, g.tail, g.head, g.cap)
    # (bottom-up levels count the vertices they reach, not the frontier: off here)
    with gpu.Graph.from_csr(csr, g.s, g.t, gpu.default_options(bfs_hops=hops, bfs_pull=0)) as G:
        live, gr, levels, rns, lns = G.solve_trace(times=True)
        st = G.stats()
    assert len(live) == st["rounds"] and len(levels) == st["bfs_levels"]
    # durations: every round and level took some time, and together no more than the solve
    assert (rns > 0).all() and (lns > 0).all()
    assert (int(rns.sum()) + int(lns.sum())) * 1e-6 <= st["solve_ms"] * 1.01 + 0.05
    assert gr[0] == 1 and int(gr.sum()) <= st["global_relabels"]
    assert (live > 0).all()
    if hops == 1:
        assert int(levels.sum()) == st["visits_bfs"]
    else:
        assert 0 < int(levels.sum()) <= st["visits_bfs"]


@pytest.mark.parametrize("which", ["grid2d", "grid3d", "rmat", "layered", "random", "hub"])
def test_simple_rounds_parity(gpu, which):
    """The simple synchronous rounds of Section 3 (one push pass, then at most one relabel per round)."""
    g = {"grid2d": I.grid2d(60, 80, 1), "grid3d": I.grid3d(24, 20, 12, seed=2), "rmat": I.rmat(12, 8, 3),
         "layered": I.layered(20, 120, 4), "random": I.random_graph(200, 1600, 5, cap=(0, 300)),
         "hub": I.random_graph(15, 4000, 6, cap=(1, 80))}[which]
    solve_and_compare(gpu, g, gpu.default_options(simple_rounds=1))


def test_simple_rounds_are_deterministic(gpu):
    """Without contested arcs or read races, repeated solves give the same per-arc flow (and the same
    number of rounds), on the same graph object and on a fresh one."""
    g = I.grid3d(28, 24, 14, seed=11)
    csr = gpu.build_csr(g.n, g.tail, g.head, g.cap)
    opt = gpu.default_options(simple_rounds=1)
    runs = []
    for _ in range(2):
        with gpu.Graph.from_csr(csr, g.s, g.t, opt) as G:
            for _ in range(2):
                r = G.solve()
                runs.append((r.value, r.flow.copy(), r.cut_bits.copy(), G.stats()["rounds"]))
    for v, f, c, k in runs[1:]:
        assert v == runs[0][0] and k == runs[0][3]
        assert np.array_equal(f, runs[0][1]) and np.array_equal(c, runs[0][2])


def test_device_wait_timeout_reported_and_graph_reusable(gpu):
    """Failure detection without a fault: with a 1 ms limit on device-side waits, a solve whose single
    CTA-wide discharge of a 4-million-arc hub takes far longer than that makes the other CTAs' barrier
    waits run out; the solve returns MF_ERR_TIMEOUT and the same graph then solves normally."""
    k = 1 << 22
    hub, t = 1, k + 2
    tail = np.concatenate([[0], np.full(k, hub), np.arange(2, k + 2)]).astype(np.int32)
    head = np.concatenate([[hub], np.arange(2, k + 2), np.full(k, t)]).astype(np.int32)
    cap = np.ones(2 * k + 1, np.int32)
    cap[0] = k
    g = I.Instance(k + 3, 0, t, tail, head, cap, "hub")
    csr = gpu.build_csr(g.n, g.tail, g.head, g.cap)
    with gpu.Graph.from_csr(csr, g.s, g.t, gpu.default_options(timeout_ms=1)) as G:
        with pytest.raises(gpu.MFError) as e:
            G.solve(flow=False, cut=False)
        assert e.value.code == -8
    with gpu.Graph.from_csr(csr, g.s, g.t) as G:
        assert G.solve(flow=False, cut=False).value == k
