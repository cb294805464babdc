"""Batched solving (mf_batch_*): many independent instances in one persistent launch.

Each instance's flow value and minimal source-side cut must equal the oracle's (they are unique), and
each instance's flow must satisfy the flow definitions on its own arcs.
"""
import numpy as np
import pytest

import oracle
from paper_1507_01926_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def check_batch(mf, insts, options=None):
    csrs = [mf.build_csr(g.n, g.tail, g.head, g.cap) for g in insts]
    with mf.Batch(csrs, [(g.s, g.t) for g in insts], options) as B:
        res = B.solve()
        st = B.stats()
    for g, c, r in zip(insts, csrs, res):
        ref = oracle.maxflow(g.n, g.s, g.t, g.tail, g.head, g.cap, want_flow=False)
        cut = mf.cut_bits_to_bool(r.cut_bits, g.n)
        assert r.value == ref["value"], g.name
        assert np.array_equal(cut, ref["cut"]), g.name
        f_in = np.where(c.arc_slot >= 0, r.flow[np.maximum(c.arc_slot, 0)], 0).astype(np.int64)
        assert not oracle.check_flow(g.n, g.s, g.t, g.tail, g.head, g.cap, f_in, r.value, cut), g.name
    return res, st


def test_batch_mixed_families(gpu):
    insts = [I.grid2d(20, 30, 1), I.layered(10, 50, 2), I.random_graph(40, 300, 3, cap=(1, 40)),
             I.grid3d(10, 9, 8, 4), I.rmat(9, 8, 5), I.multiframe(2, 6, side=20), I.grid2d(3, 3, 7)]
    check_batch(gpu, insts)


@pytest.mark.parametrize("seed", range(6))
def test_batch_many_uneven_layered(gpu, seed):
    rng = np.random.default_rng(seed)
    insts = [I.layered(int(rng.integers(2, 40)), int(rng.integers(1, 200)), 100 * seed + k) for k in range(40)]
    check_batch(gpu, insts)


def test_batch_equals_single_solves(gpu):
    insts = [I.grid2d(33, 17, 11), I.layered(12, 64, 12), I.random_graph(100, 900, 13, cap=(1, 500))]
    res, _ = check_batch(gpu, insts)
    for g, r in zip(insts, res):
        v, _, cut, _, _ = gpu.solve_instance(g)
        assert v == r.value
        assert np.array_equal(cut, gpu.cut_bits_to_bool(r.cut_bits, g.n))


def test_batch_of_one_and_edge_instances(gpu):
    from test_gpu_parity import EDGE_CASES

    check_batch(gpu, [EDGE_CASES["direct_st"]])
    check_batch(gpu, [EDGE_CASES[k] for k in sorted(EDGE_CASES)])


def test_batch_cut_only(gpu):
    insts = [I.grid2d(25, 25, 31), I.layered(8, 40, 32)]
    csrs = [gpu.build_csr(g.n, g.tail, g.head, g.cap) for g in insts]
    with gpu.Batch(csrs, [(g.s, g.t) for g in insts], gpu.default_options(cut_only=1)) as B:
        res = B.solve(flow=False)
    for g, r in zip(insts, res):
        ref = oracle.maxflow(g.n, g.s, g.t, g.tail, g.head, g.cap, want_flow=False)
        assert r.value == ref["value"]
        assert np.array_equal(gpu.cut_bits_to_bool(r.cut_bits, g.n), ref["cut"])


def test_batch_rejects_bad_instance(gpu):
    good = I.grid2d(5, 5, 1)
    c = gpu.build_csr(good.n, good.tail, good.head, good.cap)
    bad = gpu.CSR(c.n, c.row_offsets, c.head.copy(), c.cap, c.rev, c.arc_slot, 0)
    bad.head[0] = c.n  # out of its instance
    with pytest.raises(gpu.MFError) as e:
        gpu.Batch([c, bad], [(good.s, good.t)] * 2)
    assert e.value.code == -1
    with pytest.raises(gpu.MFError) as e:
        gpu.Batch([c], [(good.s, good.s)])
    assert e.value.code == -3


@pytest.mark.parametrize("hops", [1, 8, 32])
def test_batch_of_grids_local_lists_and_hops(gpu, hops):
    """A batch whose instances are all grids (every vertex thread-sized): the CTA-local lists and the
    label-correcting BFS act across instances; each instance must still get the oracle's value and S_min."""
    insts = [I.grid2d(20 + 7 * k, 30 + 3 * k, 800 + k) for k in range(5)]
    insts += [I.grid3d(10 + k, 9, 6 + k, 810 + k) for k in range(3)] + [I.multiframe(3, 820, side=24)]
    check_batch(gpu, insts, gpu.default_options(bfs_hops=hops))


@pytest.mark.parametrize("instance_relabel", [0, 1])
@pytest.mark.parametrize("ratio", [0.0, 2.0])
def test_batch_partial_relabels_agree(gpu, instance_relabel, ratio):
    """Instances of very different sizes need global relabels at different times; with instance_relabel each
    keeps its own schedule and a relabel covers only the instances that asked, carrying the others' working
    sets over. Frequent relabels (gr_freq 8, and the round-count trigger) make many of them partial; every
    instance must still get the oracle's value and S_min, and a valid flow."""
    insts = [I.grid2d(120, 90, 900), I.layered(60, 300, 901), I.multiframe(4, 902, side=40)]
    insts += [I.grid2d(4 + k, 5, 910 + k) for k in range(10)] + [I.layered(3, 8, 930 + k) for k in range(10)]
    opts = gpu.default_options(instance_relabel=instance_relabel, gr_freq=8.0, gr_time_ratio=ratio)
    _, st = check_batch(gpu, insts, opts)
    if instance_relabel:
        assert st["global_relabels_partial"] > 0
    else:
        assert st["global_relabels_partial"] == 0
    assert st["global_relabels_partial"] < st["global_relabels"]  # the first of each phase covers all


def test_simple_rounds_flow_independent_of_the_mix(gpu):
    """Deterministic mode in a batch: with the simple synchronous rounds and per-instance relabel schedules, an
    instance's per-arc flow is the same solved in a batch of one and packed with other instances (which need more
    or fewer rounds and relabels than it does)."""
    opts = gpu.default_options(simple_rounds=1, instance_relabel=1)
    target = I.grid2d(50, 41, 950)
    others = [I.multiframe(3, 951, side=30), I.layered(20, 60, 952), I.grid2d(90, 80, 953), I.grid2d(6, 7, 954)]
    (alone,), _ = check_batch(gpu, [target], opts)
    for mix in ([target] + others, others[:2] + [target] + others[2:]):
        res, st = check_batch(gpu, mix, opts)
        mixed = res[mix.index(target)]
        assert mixed.value == alone.value
        assert np.array_equal(mixed.cut_bits, alone.cut_bits)
        assert np.array_equal(mixed.flow, alone.flow), "per-arc flow differs between alone and mixed"
