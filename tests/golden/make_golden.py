"""Writes the stored expected results of the large workloads by running the CPU oracle.

Usage: python tests/golden/make_golden.py [--jobs J] [grid3d_256x256x128] [layered_batch_2048] ...

Only the oracle and the seeded input generators are called; nothing comes from the GPU path. For each
single-instance workload the file ``tests/golden/<name>.json`` records the instance shape (n, m, s, t), the
maximum flow value and the minimal source-side cut S_min as its size plus a SHA-256 of the bitmap packed
little-endian (bit v of byte v // 8 is 1 iff v is in S_min). The flow value and S_min are unique for a
maximum flow (arXiv:1507.01926, Section 2), so any correct solver must reproduce them exactly.

The multi-instance workloads store one row per instance with the same fields:

* ``layered_batch_2048``: all 2048 layered graphs of the batch workload (instance i has the (L, W) that
  ``inputs.layered_batch_params`` draws for it);
* ``serving_stream_1000``: the first 1000 requests of the serving stream (2D grids of side up to 1024 and
  multi-frame grids of up to 64 frames; the largest side and frame count the whole stream draws both occur
  among them).

Every instance's oracle flow is also checked against the flow definitions before its row is written. The
instances are independent, so they are spread over J worker processes (default: all host cores).
"""
import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1507_01926_gb300 import inputs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

WORKLOADS = {
    "grid2d_64x64": inputs.grid2d_64x64,
    "grid3d_256x256x128": inputs.grid3d_256x256x128,
    "rmat_s22_ef16": inputs.rmat_s22_ef16,
}

BATCH_COUNT = 2048
STREAM_PREFIX = 1000
ROW_FIELDS = ["i", "kind", "size", "n", "m", "s", "t", "value", "cut_size", "cut_sha256", "oracle_seconds"]


def cut_digest(cut_bool: np.ndarray) -> str:
    return hashlib.sha256(np.packbits(cut_bool.astype(np.uint8), bitorder="little").tobytes()).hexdigest()


def solve_checked(g):
    """The oracle's maximum flow of g, checked against the flow definitions; (result, cut digest)."""
    r = oracle.maxflow(g.n, g.s, g.t, g.tail, g.head, g.cap, want_flow=True, want_cut=True)
    bad = oracle.check_flow(g.n, g.s, g.t, g.tail, g.head, g.cap, r["flow"], r["value"], r["cut"])
    if bad:
        raise RuntimeError(f"{g.name}: oracle flow failed its own checks: {bad}")
    return r, cut_digest(r["cut"])


def single(name):
    g = WORKLOADS[name]()
    t0 = time.time()
    r, dig = solve_checked(g)
    out = dict(workload=g.name, n=g.n, m=g.m, s=g.s, t=g.t, value=r["value"],
               cut_size=int(r["cut"].sum()), cut_sha256=dig,
               oracle_stats=r["stats"], oracle_seconds=round(r["seconds"], 3))
    with open(os.path.join(HERE, f"{name}.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(name, out, f"{time.time() - t0:.1f}s", flush=True)


def instance(task):
    """Builds one instance of a multi-instance workload from its descriptor."""
    kind, i, a, b = task
    if kind == "layered":
        return inputs.layered_batch_instance(i, a, b)
    return inputs.serving_stream_instance(i, kind, a)


def row_of(task):
    kind, i, a, b = task
    g = instance(task)
    r, dig = solve_checked(g)
    size = [a, b] if kind == "layered" else a
    return [i, kind, size, g.n, g.m, g.s, g.t, r["value"], int(r["cut"].sum()), dig, round(r["seconds"], 3)]


def multi(name, tasks, weight, jobs, note):
    """Solves every task with the oracle in `jobs` processes (largest first) and writes one row each."""
    t0 = time.time()
    order = sorted(range(len(tasks)), key=lambda k: -weight[k])
    rows = [None] * len(tasks)
    ctx = mp.get_context("spawn")
    with ctx.Pool(jobs) as pool:
        for k, row in zip(order, pool.imap(row_of, [tasks[k] for k in order], chunksize=1)):
            rows[k] = row
    path = os.path.join(HERE, f"{name}.json")
    with open(path, "w") as f:
        f.write("{\n")
        f.write(f' "workload": {json.dumps(name)},\n "note": {json.dumps(note)},\n')
        f.write(f' "count": {len(rows)},\n "fields": {json.dumps(ROW_FIELDS)},\n "rows": [\n')
        f.write(",\n".join("  " + json.dumps(r) for r in rows))
        f.write("\n ]\n}\n")
    print(name, f"{len(rows)} instances, oracle {sum(r[-1] for r in rows):.0f} s in total, "
                f"{time.time() - t0:.0f} s wall with {jobs} processes", flush=True)


def layered_batch(jobs):
    params = inputs.layered_batch_params(BATCH_COUNT)
    tasks = [("layered", i, L, W) for i, (L, W) in enumerate(params)]
    multi(f"layered_batch_{BATCH_COUNT}", tasks, [L * W for _, _, L, W in tasks], jobs,
          "instance i: layered graph with the (L, W) drawn for it, size = [L, W]")


def serving_prefix(jobs):
    reqs = inputs.serving_stream_requests(STREAM_PREFIX)
    tasks = [(kind, i, size, 0) for i, (_, kind, size) in enumerate(reqs)]
    weight = [(size * size if kind == "grid" else 16 * 16384 * size) for kind, _, size, _ in tasks]
    multi(f"serving_stream_{STREAM_PREFIX}", tasks, weight, jobs,
          "request i of the serving stream: kind grid (size = side) or frames (size = F)")


MULTI = {f"layered_batch_{BATCH_COUNT}": layered_batch, f"serving_stream_{STREAM_PREFIX}": serving_prefix}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("names", nargs="*")
    args = ap.parse_args()
    oracle.build_lib()
    inputs.build_lib()
    for name in args.names or (list(WORKLOADS) + list(MULTI)):
        if name in WORKLOADS:
            single(name)
        elif name in MULTI:
            MULTI[name](args.jobs)
        else:
            raise SystemExit(f"unknown workload {name}")


if __name__ == "__main__":
    main()
