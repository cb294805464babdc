"""Bottom-up BFS levels (mf_options.bfs_pull): a level-synchronous BFS level whose frontier is large runs
bottom-up (every vertex not reached yet looks for an arc into the frontier). The labels of a global relabel
are the exact BFS distances either way, and the flow value and minimal source-side cut must equal the
oracle's; bfs_pull = 2**20 makes almost every level bottom-up."""
import numpy as np
import pytest

import oracle
from paper_1507_01926_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CASES = {
    "rmat": lambda: I.rmat(12, 10, 701),
    "random": lambda: I.random_graph(500, 5000, 702, cap=(1, 30)),
    "grid3d": lambda: I.grid3d(20, 18, 12, 703),
    "layered": lambda: I.layered(16, 60, 704),
}


@pytest.mark.parametrize("pull", [0, 20, 1 << 20])
@pytest.mark.parametrize("name", sorted(CASES))
def test_solve_exact(gpu, name, pull):
    g = CASES[name]()
    csr = gpu.build_csr(g.n, g.tail, g.head, g.cap)
    ref = oracle.maxflow(g.n, g.s, g.t, g.tail, g.head, g.cap, want_flow=False)
    for opt in (gpu.default_options(bfs_pull=pull, bfs_hops=1), gpu.default_options(bfs_pull=pull, cut_only=1)):
        with gpu.Graph.from_csr(csr, g.s, g.t, opt) as G:
            r = G.solve(flow=not opt.cut_only)
            cut = gpu.cut_bits_to_bool(r.cut_bits, g.n)
            assert r.value == ref["value"], name
            assert np.array_equal(cut, ref["cut"]), name
            if not opt.cut_only:
                f_in = np.where(csr.arc_slot >= 0, r.flow[np.maximum(csr.arc_slot, 0)], 0).astype(np.int64)
                assert not oracle.check_flow(g.n, g.s, g.t, g.tail, g.head, g.cap, f_in, r.value, cut), name


@pytest.mark.parametrize("pull", [0, 1 << 20])
@pytest.mark.parametrize("rounds", [0, 3, 25])
@pytest.mark.parametrize("name", ["rmat", "random", "grid3d"])
def test_relabel_labels_exact(gpu, name, rounds, pull):
    g = CASES[name]()
    csr = gpu.build_csr(g.n, g.tail, g.head, g.cap)
    with gpu.Graph.from_csr(csr, g.s, g.t, gpu.default_options(bfs_pull=pull, bfs_hops=1)) as G:
        res, lab, ex, done = G.run_rounds(rounds, final_relabel=True)
    k = res > 0
    d = oracle.sink_distances(g.n, g.s, g.t, csr.tails()[k], csr.head[k])
    assert np.array_equal(lab, d), f"{int((lab != d).sum())} labels differ"
