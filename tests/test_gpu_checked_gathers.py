"""The solver built with every gather index checked (libmf_check.so, MF_CHECK_BOUNDS).

In that build an index outside its array (a head, a reverse slot, a row offset, a vertex taken from a list)
is recorded in the error word with the source line and the index, replaced by a safe index, and the solve
ends with MF_ERR_INTERNAL at its next grid barrier: a wrong gather shows up as an error instead of a silent
out-of-bounds access. These tests run the checked build on the parity cases of every solver path (improved
and simple rounds, the degree bins, CTA-local lists, bottom-up BFS levels, gap relabeling, cut-only, batches
and the service with per-instance phases) and require the oracle's results with no error.
"""
import numpy as np
import pytest

import oracle
from paper_1507_01926_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def checked(gpu):
    from paper_1507_01926_gb300 import build as mfbuild

    path = mfbuild.build(check=True)
    before = gpu.use_library(path)
    yield gpu
    gpu.use_library(before)


def check_solve(mf, g, **opts):
    value, flow, cut, csr, st = mf.solve_instance(g, mf.default_options(**opts) if opts else None)
    ref = oracle.maxflow(g.n, g.s, g.t, g.tail, g.head, g.cap, want_flow=False)
    assert value == ref["value"] and np.array_equal(cut, ref["cut"]), g.name
    assert not oracle.check_flow(g.n, g.s, g.t, g.tail, g.head, g.cap, flow, value, cut), g.name


CASES = {
    "grid2d": lambda: I.grid2d(40, 37, 1),
    "grid3d": lambda: I.grid3d(20, 18, 12, 2),
    "rmat": lambda: I.rmat(10, 8, 3),
    "layered": lambda: I.layered(12, 60, 4),
    "random": lambda: I.random_graph(300, 3000, 5, cap=(1, 50)),
    "multiframe": lambda: I.multiframe(3, 6, side=24),
}
OPTIONS = {
    "defaults": {},
    "simple rounds": dict(simple_rounds=1),
    "warp and CTA bins": dict(bin_thread=2, bin_warp=4),
    "no local lists, bottom-up levels": dict(local_lists=0, bfs_pull=2),
    "gap relabeling": dict(gap_every=4),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("opt", list(OPTIONS))
def test_checked_single_graph(checked, case, opt):
    check_solve(checked, CASES[case](), **OPTIONS[opt])


def test_checked_cut_only(checked):
    g = I.grid2d(33, 29, 7)
    csr = checked.build_csr(g.n, g.tail, g.head, g.cap)
    with checked.Graph.from_csr(csr, g.s, g.t, checked.default_options(cut_only=1)) as G:
        r = G.solve(flow=False)
    ref = oracle.maxflow(g.n, g.s, g.t, g.tail, g.head, g.cap, want_flow=False)
    assert r.value == ref["value"]
    assert np.array_equal(checked.cut_bits_to_bool(r.cut_bits, g.n), ref["cut"])


@pytest.mark.parametrize("opts", [{}, dict(instance_relabel=0), dict(gr_freq=8.0)])
def test_checked_batch(checked, opts):
    insts = [I.grid2d(30, 30, 10), I.layered(20, 40, 11), I.multiframe(2, 12, side=20)]
    insts += [I.grid2d(4 + k, 5, 20 + k) for k in range(6)]
    csrs = [checked.build_csr(g.n, g.tail, g.head, g.cap) for g in insts]
    with checked.Batch(csrs, [(g.s, g.t) for g in insts], checked.default_options(**opts)) as B:
        res = B.solve()
    for g, c, r in zip(insts, csrs, res):
        ref = oracle.maxflow(g.n, g.s, g.t, g.tail, g.head, g.cap, want_flow=False)
        assert r.value == ref["value"], g.name
        assert np.array_equal(checked.cut_bits_to_bool(r.cut_bits, g.n), ref["cut"]), g.name


def test_checked_service(checked):
    insts = [I.grid2d(int(s), int(s), 30 + k) for k, s in enumerate([20, 45, 33])] + [I.multiframe(2, 40, side=30)]
    csrs = [checked.build_csr(g.n, g.tail, g.head, g.cap) for g in insts]
    with checked.Service(1 << 30) as svc:
        tks = [svc.submit(c, g.s, g.t) for c, g in zip(csrs, insts)]
        for t in tks:
            assert svc.wait(t, 120000) is not None
        res = [svc.poll(t) for t in tks]
    for g, c, r in zip(insts, csrs, res):
        ref = oracle.maxflow(g.n, g.s, g.t, g.tail, g.head, g.cap, want_flow=False)
        assert r.value == ref["value"], g.name
        assert np.array_equal(checked.cut_bits_to_bool(r.cut_bits, g.n), ref["cut"]), g.name
