"""Full-size multi-instance workloads on the GPU against the oracle's stored results.

* The batch of 2048 layered graphs, solved in one persistent launch with the options the bench times (the
  autotuner's packaged GB300 choice for this batch): every instance's flow value and minimal source-side cut
  must equal the oracle's (tests/golden/layered_batch_2048.json), and the per-arc flows of a strided sample
  of instances must satisfy the flow definitions.
* The first 1000 requests of the serving stream (2D grids of side up to 1024, multi-frame grids of up to 64
  frames; the largest side and frame count the whole stream draws are among them), through the
  continuous-batching service under the bench's 64 GB budget: every request's value and S_min must equal
  the oracle's (tests/golden/serving_stream_1000.json).

The stored results are written by tests/golden/make_golden.py from the oracle alone.
"""
import hashlib
import json
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_1507_01926_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
GOLD = os.path.join(os.path.dirname(__file__), "golden")
JOBS = min(32, os.cpu_count() or 1)


def digest(cut):
    return hashlib.sha256(np.packbits(cut.astype(np.uint8), bitorder="little").tobytes()).hexdigest()


def rows(name):
    g = json.load(open(os.path.join(GOLD, f"{name}.json")))
    return [dict(zip(g["fields"], r)) for r in g["rows"]]


def test_layered_batch_2048_against_golden(gpu):
    from paper_1507_01926_gb300 import autotune

    gold = rows("layered_batch_2048")
    params = I.layered_batch_params(2048)

    def csr_of(i):
        L, W = params[i]
        g = I.layered_batch_instance(i, L, W)
        assert (g.n, g.m, g.s, g.t) == (gold[i]["n"], gold[i]["m"], gold[i]["s"], gold[i]["t"]), "generator drifted"
        c = gpu.build_csr(g.n, g.tail, g.head, g.cap)
        c.arc_slot = None
        return c, (g.s, g.t)

    with ThreadPoolExecutor(JOBS) as ex:
        built = list(ex.map(csr_of, range(2048)))
    csrs, sts = [b[0] for b in built], [b[1] for b in built]
    nv, ns = sum(c.n for c in csrs), sum(c.m for c in csrs)
    hit = autotune.lookup(autotune.workload_key("layered", nv, ns, len(csrs)), "NVIDIA GB300", path=os.devnull)
    assert hit is not None, "no packaged options for the layered batch"
    opt = hit[0]
    opt.device = 0
    sample = set(range(0, 2048, 32))
    with gpu.Batch(csrs, sts, opt) as B:
        res = B.solve(flow=True, cut=True)
    bad = [i for i, r in enumerate(res) if r.value != gold[i]["value"]
           or digest(gpu.cut_bits_to_bool(r.cut_bits, csrs[i].n)) != gold[i]["cut_sha256"]]
    assert not bad, f"{len(bad)} instances differ from the oracle, first {bad[:5]}"
    for i in sorted(sample):  # per-arc flows by the flow definitions
        L, W = params[i]
        g = I.layered_batch_instance(i, L, W)
        c = gpu.build_csr(g.n, g.tail, g.head, g.cap)
        f_in = np.where(c.arc_slot >= 0, res[i].flow[np.maximum(c.arc_slot, 0)], 0).astype(np.int64)
        cut = gpu.cut_bits_to_bool(res[i].cut_bits, g.n)
        assert not oracle.check_flow(g.n, g.s, g.t, g.tail, g.head, g.cap, f_in, res[i].value, cut), i


def test_serving_stream_prefix_against_golden(gpu):
    gold = rows("serving_stream_1000")
    reqs = I.serving_stream_requests(len(gold))

    def csr_of(i):
        _, kind, size = reqs[i]
        g = I.serving_stream_instance(i, kind, size)
        assert (g.n, g.m, g.s, g.t) == (gold[i]["n"], gold[i]["m"], gold[i]["s"], gold[i]["t"]), "generator drifted"
        c = gpu.build_csr(g.n, g.tail, g.head, g.cap)
        c.arc_slot = None
        return i, c, g.s, g.t

    outstanding, bad, window = {}, [], 128
    with gpu.Service(64 << 30) as svc, ThreadPoolExecutor(JOBS) as ex:
        def drain(limit):
            while len(outstanding) > limit:
                i = min(outstanding)
                tk, n = outstanding.pop(i)
                assert svc.wait(tk, 600000) is not None, f"request {i} did not finish"
                r = svc.poll(tk, flow=False, cut=True)
                if r.value != gold[i]["value"] or digest(gpu.cut_bits_to_bool(r.cut_bits, n)) != gold[i]["cut_sha256"]:
                    bad.append(i)

        # built ahead by JOBS threads (at most 2 * JOBS at a time), submitted in stream order, at most `window`
        # requests open in the service
        futs = {i: ex.submit(csr_of, i) for i in range(min(2 * JOBS, len(gold)))}
        for i in range(len(gold)):
            _, c, s, t = futs.pop(i).result()
            if i + 2 * JOBS < len(gold):
                futs[i + 2 * JOBS] = ex.submit(csr_of, i + 2 * JOBS)
            outstanding[i] = (svc.submit(c, s, t), c.n)
            drain(window)
        drain(0)
    assert not bad, f"{len(bad)} requests differ from the oracle, first {bad[:5]}"
