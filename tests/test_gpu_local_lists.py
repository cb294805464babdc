"""CTA-local working sets and BFS frontiers (mf_options.local_lists) and several BFS levels per grid barrier
(mf_options.bfs_hops): on graphs whose vertices are all thread-sized, a CTA keeps the few vertices it stages
for the next round or level in shared memory, and a BFS may expand them further before the barrier
(label-correcting). The flow value and the minimal source-side cut are unique, so every setting must give
the oracle's, and the flow must satisfy the flow definitions; global-relabel labels must equal exact BFS
distances."""
import numpy as np
import pytest

import oracle
from paper_1507_01926_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CASES = {
    "grid2d_96x80": lambda: I.grid2d(96, 80, 91),
    "grid3d_40x36x28": lambda: I.grid3d(40, 36, 28, 92),
    "multiframe_6": lambda: I.multiframe(6, 93, side=48),
    "layered_small": lambda: I.layered(30, 64, 94),  # degrees above bin_thread: the setting has no effect
}


@pytest.mark.parametrize("local,hops", [(0, 1), (1, 1), (1, 4), (1, 64)])
@pytest.mark.parametrize("name", sorted(CASES))
def test_exact_with_and_without_local_lists(gpu, name, local, hops):
    g = CASES[name]()
    csr = gpu.build_csr(g.n, g.tail, g.head, g.cap)
    ref = oracle.maxflow(g.n, g.s, g.t, g.tail, g.head, g.cap, want_flow=False)
    opts = [gpu.default_options(local_lists=local, bfs_hops=hops)]
    if local:  # a smaller CTA keeps fewer entries; more CTAs per SM
        opts.append(gpu.default_options(local_lists=1, bfs_hops=hops, block_threads=128, blocks_per_sm=4,
                                        kernel_variant=2))
        opts.append(gpu.default_options(local_lists=1, bfs_hops=hops, cut_only=1))
    for o in opts:
        with gpu.Graph.from_csr(csr, g.s, g.t, o) as G:
            for _ in range(2):
                if o.cut_only:
                    r = G.solve(flow=False)
                    assert r.value == ref["value"], name
                    assert np.array_equal(gpu.cut_bits_to_bool(r.cut_bits, g.n), ref["cut"]), name
                    continue
                r = G.solve()
                cut = gpu.cut_bits_to_bool(r.cut_bits, g.n)
                assert r.value == ref["value"], name
                assert np.array_equal(cut, ref["cut"]), name
                f_in = np.where(csr.arc_slot >= 0, r.flow[np.maximum(csr.arc_slot, 0)], 0).astype(np.int64)
                assert not oracle.check_flow(g.n, g.s, g.t, g.tail, g.head, g.cap, f_in, r.value, cut), name


@pytest.mark.parametrize("local,hops", [(0, 1), (1, 1), (1, 2), (1, 4), (1, 64)])
@pytest.mark.parametrize("rounds", [0, 1, 7, 40])
def test_relabel_labels_exact_with_local_lists(gpu, rounds, local, hops):
    g = I.grid3d(24, 24, 20, 95)
    csr = gpu.build_csr(g.n, g.tail, g.head, g.cap)
    with gpu.Graph.from_csr(csr, g.s, g.t, gpu.default_options(local_lists=local, bfs_hops=hops)) as G:
        res, lab, ex, done = G.run_rounds(rounds, final_relabel=True)
    k = res > 0
    d = oracle.sink_distances(g.n, g.s, g.t, csr.tails()[k], csr.head[k])
    assert np.array_equal(lab, d), f"{int((lab != d).sum())} labels differ"
