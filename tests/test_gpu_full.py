"""Full-size workloads on the GPU, with the default options and with the options the bench times (the
autotuner's packaged GB300 choices).

The flow value and the minimal source-side cut must equal the oracle's stored results
(tests/golden/*.json, written by tests/golden/make_golden.py from the oracle alone); the per-arc flow
must satisfy the flow definitions (oracle.check_flow: capacity bounds, conservation, no residual s-t
path, cut capacity = value, cut = residual reachability from s).
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from paper_1507_01926_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def digest(cut):
    return hashlib.sha256(np.packbits(cut.astype(np.uint8), bitorder="little").tobytes()).hexdigest()


@pytest.mark.parametrize("name", ["grid2d_64x64", "grid3d_256x256x128", "rmat_s22_ef16"])
def test_full_size_against_golden(gpu, name):
    gold = json.load(open(os.path.join(GOLD, f"{name}.json")))
    g = getattr(I, name)()
    assert (g.n, g.m, g.s, g.t) == (gold["n"], gold["m"], gold["s"], gold["t"]), "generator drifted"
    value, flow, cut, csr, stats = gpu.solve_instance(g)
    assert value == gold["value"]
    assert int(cut.sum()) == gold["cut_size"]
    assert digest(cut) == gold["cut_sha256"]
    bad = oracle.check_flow(g.n, g.s, g.t, g.tail, g.head, g.cap, flow, value, cut)
    assert not bad, bad


def test_grid3d_256x256x128_cut_only_and_repeat(gpu):
    gold = json.load(open(os.path.join(GOLD, "grid3d_256x256x128.json")))
    g = I.grid3d_256x256x128()
    csr = gpu.build_csr(g.n, g.tail, g.head, g.cap)
    with gpu.Graph.from_csr(csr, g.s, g.t, gpu.default_options(cut_only=1)) as G:
        for _ in range(2):
            r = G.solve(flow=False)
            assert r.value == gold["value"]
            assert digest(gpu.cut_bits_to_bool(r.cut_bits, g.n)) == gold["cut_sha256"]


@pytest.mark.parametrize("name,family", [("grid3d_256x256x128", "grid3d"), ("rmat_s22_ef16", "rmat")])
def test_full_size_with_the_bench_options(gpu, name, family):
    """The launch configuration bench.py times: the packaged tuned options of the workload."""
    from paper_1507_01926_gb300 import autotune

    gold = json.load(open(os.path.join(GOLD, f"{name}.json")))
    g = getattr(I, name)()
    csr = gpu.build_csr(g.n, g.tail, g.head, g.cap)
    hit = autotune.lookup(autotune.workload_key(family, g.n, csr.m), "NVIDIA GB300", path=os.devnull)
    assert hit is not None, "no packaged options for this workload"
    opt = hit[0]
    opt.device = 0
    with gpu.Graph.from_csr(csr, g.s, g.t, opt) as G:
        r = G.solve()
    cut = gpu.cut_bits_to_bool(r.cut_bits, g.n)
    assert r.value == gold["value"]
    assert int(cut.sum()) == gold["cut_size"] and digest(cut) == gold["cut_sha256"]
    f_in = np.where(csr.arc_slot >= 0, r.flow[np.maximum(csr.arc_slot, 0)], 0).astype(np.int64)
    bad = oracle.check_flow(g.n, g.s, g.t, g.tail, g.head, g.cap, f_in, r.value, cut)
    assert not bad, bad
