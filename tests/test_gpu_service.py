"""Serving with continuous batching (mf_service_create / mf_submit / mf_poll / mf_wait).

Every result must equal the oracle's unique outputs (value, S_min) whether the request is solved alone or
in a mix with others, and its flow must satisfy the flow definitions.
"""
import numpy as np
import pytest

import oracle
from paper_1507_01926_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def check(mf, g, csr, r):
    ref = oracle.maxflow(g.n, g.s, g.t, g.tail, g.head, g.cap, want_flow=False)
    cut = mf.cut_bits_to_bool(r.cut_bits, g.n)
    assert r.value == ref["value"], g.name
    assert np.array_equal(cut, ref["cut"]), g.name
    f_in = np.where(csr.arc_slot >= 0, r.flow[np.maximum(csr.arc_slot, 0)], 0).astype(np.int64)
    assert not oracle.check_flow(g.n, g.s, g.t, g.tail, g.head, g.cap, f_in, r.value, cut), g.name


def test_alone_equals_mixed(gpu):
    target = I.multiframe(3, 41, side=48)
    others = [I.grid2d(int(s), int(s), 100 + k) for k, s in enumerate([20, 64, 33, 90, 45])]
    others += [I.multiframe(2, 200 + k, side=32) for k in range(3)]
    tc = gpu.build_csr(target.n, target.tail, target.head, target.cap)
    with gpu.Service(1 << 30) as svc:
        tk = svc.submit(tc, target.s, target.t)
        assert svc.wait(tk) > 0
        alone = svc.poll(tk)
        check(gpu, target, tc, alone)
        csrs = [gpu.build_csr(g.n, g.tail, g.head, g.cap) for g in others]
        tks = [svc.submit(c, g.s, g.t) for c, g in zip(csrs[:4], others[:4])]
        tk2 = svc.submit(tc, target.s, target.t)
        tks += [svc.submit(c, g.s, g.t) for c, g in zip(csrs[4:], others[4:])]
        for t in tks + [tk2]:
            assert svc.wait(t, 120000) is not None
        mixed = svc.poll(tk2)
        check(gpu, target, tc, mixed)
        assert mixed.value == alone.value
        assert np.array_equal(mixed.cut_bits, alone.cut_bits)
        for t, c, g in zip(tks, csrs, others):
            check(gpu, g, c, svc.poll(t))


def test_poll_pending_unknown_and_budget(gpu):
    g = I.grid2d(30, 30, 5)
    c = gpu.build_csr(g.n, g.tail, g.head, g.cap)
    with gpu.Service(1 << 22) as svc:  # 4 MiB: fits this instance, not a big one
        tk = svc.submit(c, g.s, g.t)
        r = None
        for _ in range(100000):
            r = svc.poll(tk)
            if r is not None:
                break
            svc.wait(tk, 10)
        assert r is not None
        check(gpu, g, c, r)
        with pytest.raises(gpu.MFError) as e:
            svc.poll(tk)  # forgotten after the result was handed out
        assert e.value.code == -12
        big = I.grid2d(300, 300, 6)
        bc = gpu.build_csr(big.n, big.tail, big.head, big.cap)
        with pytest.raises(gpu.MFError) as e:
            svc.submit(bc, big.s, big.t)
        assert e.value.code == -6


def test_budget_serialises_but_completes(gpu):
    """With a budget that fits one request at a time, all requests still complete correctly."""
    insts = [I.grid2d(150, 150, 300 + k) for k in range(6)]
    csrs = [gpu.build_csr(g.n, g.tail, g.head, g.cap) for g in insts]
    one = 61 * insts[0].n + 32 * csrs[0].m + 65536
    with gpu.Service(int(one * 1.5)) as svc:
        tks = [svc.submit(c, g.s, g.t) for c, g in zip(csrs, insts)]
        for t, c, g in zip(tks, csrs, insts):
            assert svc.wait(t, 120000) is not None
            check(gpu, g, c, svc.poll(t))


def test_alone_equals_mixed_per_arc_flow_in_simple_rounds(gpu):
    """Deterministic mode: with the simple synchronous rounds (Section 3) and per-instance relabel schedules
    (instance_relabel), a request's whole result, per-arc flow included, is the same solved alone and in a mix
    with other requests of other sizes and kinds."""
    opts = gpu.default_options(simple_rounds=1, instance_relabel=1)
    target = I.multiframe(3, 61, side=40)
    others = [I.grid2d(int(s), int(s), 400 + k) for k, s in enumerate([24, 70, 45])] + [I.multiframe(2, 410, side=30)]
    tc = gpu.build_csr(target.n, target.tail, target.head, target.cap)
    csrs = [gpu.build_csr(g.n, g.tail, g.head, g.cap) for g in others]
    with gpu.Service(1 << 30, opts) as svc:
        tk = svc.submit(tc, target.s, target.t)
        assert svc.wait(tk, 120000) is not None
        alone = svc.poll(tk)
        check(gpu, target, tc, alone)
        results = []
        for order in (0, 1):  # the target first, then last, in one admission group each time
            group = [(tc, target)] + list(zip(csrs, others))
            if order:
                group = group[1:] + group[:1]
            tks = [svc.submit(c, g.s, g.t) for c, g in group]
            for t in tks:
                assert svc.wait(t, 120000) is not None
            res = [svc.poll(t) for t in tks]
            results.append(res[0] if order == 0 else res[-1])
            for (c, g), r in zip(group, res):
                check(gpu, g, c, r)
        for mixed in results:
            assert mixed.value == alone.value
            assert np.array_equal(mixed.cut_bits, alone.cut_bits)
            assert np.array_equal(mixed.flow, alone.flow), "per-arc flow differs between alone and mixed"
