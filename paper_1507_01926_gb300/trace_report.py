"""Where the time of a solve goes: a traced solve (mf_solve_trace with durations) split by working-set size.

Every push-relabel round and every BFS level ends with a grid barrier, so a solve is a sequence of short
phases whose cost depends on how many vertices they touch. `breakdown` sums the phase durations CTA 0
recorded into buckets of working-set (round) or frontier (BFS level) size; the command line runs it on the
256x256x128 3D grid with the options the bench uses, or another grid (GPU required):

    python -m paper_1507_01926_gb300.trace_report [--solves K] [--grid3d X Y Z]
"""
from __future__ import annotations

import json

import numpy as np

EDGES = (0, 8, 64, 256, 1024, 4096, 16384, 65536, 262144, 1 << 31)


def _buckets(sizes, ns, edges, what):
    sizes = np.asarray(sizes, np.int64)
    us = np.asarray(ns, np.int64) * 1e-3
    rows = []
    for a, b in zip(edges[:-1], edges[1:]):
        m = (sizes >= a) & (sizes < b)
        if m.any():
            rows.append({what: [int(a), int(b)], "count": int(m.sum()), "ms": float(us[m].sum()) / 1e3,
                         "us_mean": float(us[m].mean()), "us_p90": float(np.percentile(us[m], 90))})
    return rows


def breakdown(live, round_ns, level_sizes, level_ns, edges=EDGES) -> dict:
    """Rounds by working-set size and BFS levels by frontier size: count, total ms, mean and p90 us each."""
    if len(live) != len(round_ns) or len(level_sizes) != len(level_ns):
        raise ValueError("sizes and durations differ in length")
    return {
        "rounds": len(live),
        "round_ms": float(np.sum(np.asarray(round_ns, np.int64))) / 1e6,
        "rounds_by_live": _buckets(live, round_ns, edges, "live"),
        "levels": len(level_sizes),
        "level_ms": float(np.sum(np.asarray(level_ns, np.int64))) / 1e6,
        "levels_by_frontier": _buckets(level_sizes, level_ns, edges, "frontier"),
    }


def main(argv=None) -> int:
    import argparse

    from . import autotune, inputs, mf

    ap = argparse.ArgumentParser(description="Traced solve of a 3D grid, split by working-set size")
    ap.add_argument("--solves", type=int, default=1, help="traced solves (one JSON line each)")
    ap.add_argument("--grid3d", type=int, nargs=3, default=None, metavar=("X", "Y", "Z"),
                    help="another grid than the 256x256x128 bench workload (same generator, seed 1)")
    a = ap.parse_args(argv)
    g = inputs.grid3d(*a.grid3d, seed=1) if a.grid3d else inputs.grid3d_256x256x128()
    csr = mf.build_csr(g.n, g.tail, g.head, g.cap)
    hit = autotune.lookup(autotune.workload_key("grid3d", g.n, csr.m), autotune.device_name(0))
    opt = hit[0] if hit else mf.default_options()
    with mf.Graph.from_csr(csr, g.s, g.t, opt) as G:
        G.solve(flow=False, cut=False)  # warm-up
        for _ in range(a.solves):
            live, _, lv, rns, lns = G.solve_trace(capacity=1 << 21, level_capacity=1 << 21, times=True)
            st = G.stats()
            out = {"workload": g.name, "solve_ms": st["solve_ms"], "global_relabels": st["global_relabels"],
                   **breakdown(live, rns, lv, lns)}
            print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
