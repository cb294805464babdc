"""Graph-captured solves (mf_options.use_graph): the launch sequence of a solve (control-block reset, the
persistent kernel, the status read-back) is captured into a CUDA graph once and replayed.

A replay must give the oracle's flow value and minimal source-side cut (both unique) and a flow that
satisfies the flow definitions, on every replay, after a change of outputs or options (which captures
anew) and for batches; on the legacy default stream the sequence is launched directly.
"""
import numpy as np
import pytest

import oracle
from paper_1507_01926_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def check(mf, g, csr, value, flow, cut_bits):
    ref = oracle.maxflow(g.n, g.s, g.t, g.tail, g.head, g.cap, want_flow=False)
    cut = mf.cut_bits_to_bool(cut_bits, g.n)
    assert value == ref["value"], g.name
    assert np.array_equal(cut, ref["cut"]), g.name
    f_in = np.where(csr.arc_slot >= 0, flow[np.maximum(csr.arc_slot, 0)], 0).astype(np.int64)
    assert not oracle.check_flow(g.n, g.s, g.t, g.tail, g.head, g.cap, f_in, value, cut), g.name


@pytest.mark.parametrize("which", ["grid2d", "rmat", "layered"])
def test_replays_solve_exactly(gpu, which):
    g = {"grid2d": lambda: I.grid2d(64, 48, 81), "rmat": lambda: I.rmat(12, 8, 82),
         "layered": lambda: I.layered(20, 150, 83)}[which]()
    csr = gpu.build_csr(g.n, g.tail, g.head, g.cap)
    with gpu.Graph.from_csr(csr, g.s, g.t, gpu.default_options(use_graph=1)) as G:
        rounds = set()
        for _ in range(3):
            r = G.solve()
            check(gpu, g, csr, r.value, r.flow, r.cut_bits)
            st = G.stats()
            assert st["rounds"] > 0 and st["solve_ms"] > 0
            rounds.add(st["rounds"])
        # options change the kernel arguments: the next solve captures anew
        G.set_options(gpu.default_options(use_graph=1, bin_thread=2, gr_time_ratio=0.0))
        r = G.solve()
        check(gpu, g, csr, r.value, r.flow, r.cut_bits)
        # and back to direct launches
        G.set_options(gpu.default_options())
        r = G.solve()
        check(gpu, g, csr, r.value, r.flow, r.cut_bits)


def test_device_outputs_and_streams(gpu):
    import torch

    g = I.grid3d(24, 20, 16, 84)
    csr = gpu.build_csr(g.n, g.tail, g.head, g.cap)
    dev = torch.device("cuda", 0)
    opt = gpu.default_options(use_graph=1)
    row = torch.from_numpy(csr.row_offsets).to(dev)
    head = torch.from_numpy(csr.head).to(dev)
    cap = torch.from_numpy(csr.cap).to(dev)
    rev = torch.from_numpy(csr.rev).to(dev)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    G = gpu.Graph.from_device(g.n, row, head, cap, rev, g.s, g.t, opt, stream=s1)
    try:
        outs = []
        for _ in range(2):
            outs.append((torch.zeros(1, dtype=torch.int64, device=dev), torch.zeros(csr.m, dtype=torch.int32, device=dev),
                         torch.zeros((g.n + 31) // 32, dtype=torch.int32, device=dev)))
        # same outputs twice (replay), other outputs (new capture), another stream (new capture), the legacy
        # default stream (direct launch)
        for k, st in ((0, s1), (0, s1), (1, s1), (1, s2), (0, torch.cuda.default_stream())):
            v, f, c = outs[k]
            v.zero_()
            f.fill_(-1)
            c.zero_()
            torch.cuda.synchronize()
            G.solve_device(v, f, c, stream=st)
            torch.cuda.synchronize()
            check(gpu, g, csr, int(v.item()), f.cpu().numpy(), c.cpu().numpy().view(np.uint32))
    finally:
        G.close()


def test_batch_replays(gpu):
    insts = [I.layered(6 + 2 * k, 30 + 25 * k, 400 + k) for k in range(5)] + [I.grid2d(30, 20, 410)]
    csrs = [gpu.build_csr(g.n, g.tail, g.head, g.cap) for g in insts]
    with gpu.Batch(csrs, [(g.s, g.t) for g in insts], gpu.default_options(use_graph=1)) as B:
        for _ in range(3):
            res = B.solve()
            for g, c, r in zip(insts, csrs, res):
                check(gpu, g, c, r.value, r.flow, r.cut_bits)
        vals = [r.value for r in B.solve(flow=False, cut=False)]
        assert vals == [r.value for r in res]
