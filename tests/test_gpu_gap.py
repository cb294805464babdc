"""Gap relabeling (mf_options.gap_every): between rounds, when no vertex holds some label g below n, the
vertices labelled between g and n cannot reach the sink and are lifted to n. The flow value and the
minimal source-side cut are unique, so every setting must give the oracle's, with a flow that satisfies
the flow definitions; a batch and the simple rounds ignore the option."""
import numpy as np
import pytest

import oracle
from paper_1507_01926_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CASES = {
    "grid2d": lambda: I.grid2d(70, 50, 601),
    "grid3d": lambda: I.grid3d(24, 20, 16, 602),
    "rmat": lambda: I.rmat(12, 8, 603),
    "random": lambda: I.random_graph(400, 3000, 604, cap=(1, 30)),
    "layered": lambda: I.layered(24, 80, 605),
}


def check(gpu, g, csr, r):
    ref = oracle.maxflow(g.n, g.s, g.t, g.tail, g.head, g.cap, want_flow=False)
    cut = gpu.cut_bits_to_bool(r.cut_bits, g.n)
    assert r.value == ref["value"], g.name
    assert np.array_equal(cut, ref["cut"]), g.name
    f_in = np.where(csr.arc_slot >= 0, r.flow[np.maximum(csr.arc_slot, 0)], 0).astype(np.int64)
    assert not oracle.check_flow(g.n, g.s, g.t, g.tail, g.head, g.cap, f_in, r.value, cut), g.name


@pytest.mark.parametrize("every", [1, 3, 64])
def test_gap_relabeling_exact(gpu, every):
    lifted = 0
    for name in sorted(CASES):
        g = CASES[name]()
        csr = gpu.build_csr(g.n, g.tail, g.head, g.cap)
        # the time-based relabel trigger off, so that labels drift and gaps open between global relabels
        with gpu.Graph.from_csr(csr, g.s, g.t, gpu.default_options(gap_every=every, gr_time_ratio=0.0)) as G:
            for _ in range(2):
                check(gpu, g, csr, G.solve())
                st = G.stats()
                assert st["gap_lifted"] >= 0
                lifted += st["gap_lifted"]
    assert lifted > 0, "no gap opened in any case: the path was not exercised"


def test_gap_option_ignored_where_it_does_not_apply(gpu):
    insts = [I.layered(6 + k, 30, 610 + k) for k in range(3)]
    csrs = [gpu.build_csr(g.n, g.tail, g.head, g.cap) for g in insts]
    with gpu.Batch(csrs, [(g.s, g.t) for g in insts], gpu.default_options(gap_every=1)) as B:
        for g, c, r in zip(insts, csrs, B.solve()):
            check(gpu, g, c, r)
        assert B.stats()["gap_lifted"] == 0
    g = I.grid2d(30, 30, 620)
    csr = gpu.build_csr(g.n, g.tail, g.head, g.cap)
    with gpu.Graph.from_csr(csr, g.s, g.t, gpu.default_options(gap_every=1, simple_rounds=1)) as G:
        check(gpu, g, csr, G.solve())
        assert G.stats()["gap_lifted"] == 0
