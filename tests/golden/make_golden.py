"""Writes the stored expected results of the large workloads by running the CPU oracle.

Usage: python tests/golden/make_golden.py [grid3d_256x256x128] [rmat_s22_ef16] ...

Only the oracle and the seeded input generators are called; nothing comes from the GPU path. For each
workload the file ``tests/golden/<name>.json`` records the instance shape (n, m, s, t), the maximum
flow value and the minimal source-side cut S_min as its size plus a SHA-256 of the bitmap packed
little-endian (bit v of byte v // 8 is 1 iff v is in S_min). The flow value and S_min are unique for
a maximum flow (arXiv:1507.01926, Section 2), so any correct solver must reproduce them exactly.
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1507_01926_gb300 import inputs  # noqa: E402

WORKLOADS = {
    "grid2d_64x64": inputs.grid2d_64x64,
    "grid3d_256x256x128": inputs.grid3d_256x256x128,
    "rmat_s22_ef16": inputs.rmat_s22_ef16,
}


def cut_digest(cut_bool: np.ndarray) -> str:
    return hashlib.sha256(np.packbits(cut_bool.astype(np.uint8), bitorder="little").tobytes()).hexdigest()


def main(names):
    for name in names:
        g = WORKLOADS[name]()
        t0 = time.time()
        r = oracle.maxflow(g.n, g.s, g.t, g.tail, g.head, g.cap, want_flow=True, want_cut=True)
        bad = oracle.check_flow(g.n, g.s, g.t, g.tail, g.head, g.cap, r["flow"], r["value"], r["cut"])
        if bad:
            raise SystemExit(f"{name}: oracle flow failed its own checks: {bad}")
        out = dict(workload=g.name, n=g.n, m=g.m, s=g.s, t=g.t, value=r["value"],
                   cut_size=int(r["cut"].sum()), cut_sha256=cut_digest(r["cut"]),
                   oracle_stats=r["stats"], oracle_seconds=round(r["seconds"], 3))
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}.json")
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
            f.write("\n")
        print(name, out, f"{time.time() - t0:.1f}s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or list(WORKLOADS))
