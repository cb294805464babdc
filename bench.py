"""Benchmark: max-flow / min-cut on one GB300 through libmf's C-ABI.

The line's metric is measured on the 256x256x128 6-connected grid (8,388,610 vertices, 50,331,648 CSR slots):
one step = one complete mf_solve (reset from the capacities, phase 1 = maximum preflow by synchronous discharge
rounds and BFS global relabels, phase 2 = excess returned to s, cut BFS, per-slot flow and cut bitmap outputs,
all in device memory). The metric is arc-scans/s (slots examined by discharge passes and BFS expansions per
second of solve time); solve ms and the solve-time ratio to the oracle's full solve are reported beside it.

The same line carries the two multi-instance workloads:
  "batch": the 2048 layered graphs, batched (one persistent launch) against plain (one launch per instance) on
           the same instances, with the parity of every instance against the oracle's stored results;
  "serve": the 20,000-request Poisson stream through the continuous-batching service at 0.7 of the saturated
           throughput, with p50/p99 latency and the parity of the first 1000 requests.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload all|grid3d|batch|serve]

N > 1 runs under torchrun, one replica per GPU of the grid solve (the path does not shard; each rank solves its
own copy; the batch and serving parts run at N = 1 only). --impl reference times the CPU oracle (sequential
FIFO push-relabel) on a bounded sample of the 3D-grid workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "grid3d_256x256x128: 6-connected, capacity U[1,1000] per direction, s->face z=0 and face z=127->t at 1e6"
METRIC = "arc-scans/s"

# Algorithmic bytes (what the method must move), per unit:
B_SCAN_DIS = 4      # discharge arc scan, every examined slot: its residual 4
B_SCAN_DIS_RES = 8  # ... and one with positive residual: head 4 + d(w) 4 (+ the active bit)
B_PUSH = 28         # push: rev 4 + two residual writes 8 + int64 atomic read-modify-write 16
B_VISIT_DIS = 48    # active-vertex visit: row offsets 8 + d 4 + e 8 + d' 4 + addedExcess 16 + list 8
B_SCAN_BFS = 12     # BFS arc scan: head 4 + reverse residual 4 + d(w) 4
B_VISIT_BFS = 16    # BFS frontier vertex: row offsets 8 + list 8
B_SLOT_FIXED = 20   # per solve and slot: residual reset (cap 4 + write 4) + flow output (cap 4 + res 4 + out 4)
B_VERTEX_FIXED = 28  # per solve and vertex: state reset (d 4 + e 8 + addedExcess 8 + stamps 4) + cut 4
B_VERTEX_GR = 12    # per global relabel and vertex: label reset 4 + rebuild (label 4 + excess ... 4)
HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e, nominal (the measured copy peak is the roofline's denominator)


def model_bytes(st: dict, n: int, m: int) -> int:
    return int(B_SCAN_DIS * st["scans_discharge"] + B_SCAN_DIS_RES * st["scans_discharge_residual"]
               + B_PUSH * st["pushes"] + B_VISIT_DIS * st["visits_discharge"] + B_SCAN_BFS * st["scans_bfs"] + B_VISIT_BFS * st["visits_bfs"] + B_SLOT_FIXED * m
               + B_VERTEX_FIXED * n + B_VERTEX_GR * n * st["global_relabels"])


def phase_rooflines(st: dict, n: int, peak: float) -> dict:
    """Algorithmic GB/s of the two parts of the hot path, timed by the kernel's own clock (CTA 0's view of
    the time spent in discharge rounds and in global relabels, barrier waits included)."""
    dis = (B_SCAN_DIS * st["scans_discharge"] + B_SCAN_DIS_RES * st["scans_discharge_residual"]
           + B_PUSH * st["pushes"] + B_VISIT_DIS * st["visits_discharge"])
    bfs = B_SCAN_BFS * st["scans_bfs"] + B_VISIT_BFS * st["visits_bfs"] + B_VERTEX_GR * n * st["global_relabels"]
    out = {}
    for name, b, ms in (("discharge_rounds", dis, st["discharge_ms"]), ("global_relabel_bfs", bfs, st["relabel_ms"])):
        gbs = b / (ms * 1e6) if ms > 0 else None
        out[name] = {"model_bytes": int(b), "ms": ms, "achieved_GBps": gbs, "frac": gbs / peak if gbs else None}
    return out


def paired_slot_count(tail, head) -> int:
    """Slots of the paired-slot CSR of an arc list (include/mf.h): self-loops dropped, the k-th arc u -> v
    shares its slot pair with the k-th arc v -> u, every other arc gets a pair of its own; so an unordered
    pair {u, v} takes 2 * max(#(u -> v), #(v -> u)) slots."""
    tail = np.asarray(tail, np.int64)
    head = np.asarray(head, np.int64)
    keep = tail != head
    tail, head = tail[keep], head[keep]
    lo, hi = np.minimum(tail, head), np.maximum(tail, head)
    n = int(max(hi.max(), 0)) + 1 if hi.size else 1
    fwd = tail < head
    key = lo * n + hi
    cf = np.unique(key[fwd], return_counts=True)
    cb = np.unique(key[~fwd], return_counts=True)
    keys = np.union1d(cf[0], cb[0])
    a = np.zeros(keys.size, np.int64)
    b = np.zeros(keys.size, np.int64)
    a[np.searchsorted(keys, cf[0])] = cf[1]
    b[np.searchsorted(keys, cb[0])] = cb[1]
    return int(2 * np.maximum(a, b).sum())


def workload_config(g, slots: int, world: int, name: str) -> dict:
    """The `config` object of a bench line, the same for both arms."""
    return {"workload": name, "n": g.n, "slots": slots, "arcs": g.m, "global_batch": world,
            "parallelism": f"replicas x{world}", "l2": "inputs larger than L2 (about 1.3 GB of device state per solve)"}


def apply_overrides(opt, args):
    """Sets the mf_options fields given by --options (a JSON object) on opt."""
    if args.options:
        for k, v in json.loads(args.options).items():
            if not hasattr(opt, k):
                raise KeyError(k)
            setattr(opt, k, v)
    return opt


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def load_workload(shape=None):
    from paper_1507_01926_gb300 import inputs, mf

    if shape is None or tuple(shape) == (256, 256, 128):
        g = inputs.grid3d_256x256x128()
    else:
        g = inputs.grid3d(*shape, seed=inputs.BASE_SEED + 1)
    csr = mf.build_csr(g.n, g.tail, g.head, g.cap)
    return g, csr


def kernel_source_hash() -> str:
    """Identifies the solver kernel version the stored ncu counters belong to."""
    import hashlib

    csrc = os.path.join(ROOT, "paper_1507_01926_gb300", "csrc")
    data = b"".join(open(os.path.join(csrc, f), "rb").read() for f in ("mf_solver.cuh", "mf_device.cuh"))
    return hashlib.sha256(data).hexdigest()[:16]


def golden_record():
    p = os.path.join(ROOT, "tests", "golden", "grid3d_256x256x128.json")
    if os.path.exists(p):
        return json.load(open(p))
    return None


def sized_oracle_run(g, seconds: float):
    """Runs the oracle's phase 1 on the full workload with an arc-scan limit grown geometrically until one run
    takes about `seconds` (the scan rate changes as a solve proceeds: its first global relabel scans every arc
    quickly, the discharge rounds after it are slower per scan, so a short probe overestimates the rate).
    Returns (last run, its scan limit); the sizing runs take about as long again."""
    import oracle

    limit = 20_000_000
    for _ in range(8):
        r = oracle.maxflow(g.n, g.s, g.t, g.tail, g.head, g.cap, want_flow=False, want_cut=False, work_limit=limit)
        if not r["truncated"] or r["seconds"] >= 0.6 * seconds:
            break
        limit = int(limit * min(4.0, max(1.5, 0.8 * seconds / max(r["seconds"], 1e-3))))
    return r, limit


def cpu_baseline(g, seconds: float = 12.0):
    """The oracle, as it stands, on a bounded sample: phase 1 on the full workload, stopped after a number of
    arc scans sized to about `seconds` of single-core work. Reports arc-scans/s."""
    r, _ = sized_oracle_run(g, seconds)
    done = r["stats"]["scans"]
    return {"value": done / r["seconds"], "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"sequential FIFO push-relabel phase 1 on the full {g.name}, stopped after {done} arc scans "
                      f"({r['seconds']:.1f} s, {'complete' if not r['truncated'] else 'truncated'})",
            "seconds": r["seconds"], "scans": done}


def aggregate_ranks(total_ms: float, scans: float, device):
    """Whole-job figures over the ranks of the process group: the slowest rank's timed milliseconds and the
    arc scans of all ranks (replicas: every rank solves its own copy)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(total_ms), float(scans)], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    from paper_1507_01926_gb300 import inputs

    import oracle

    g = inputs.grid3d_256x256x128()
    per_step = max(2.0, min(10.0, 150.0 / max(1, args.steps + args.warmup)))
    _, limit = sized_oracle_run(g, per_step)
    for _ in range(args.warmup):
        oracle.maxflow(g.n, g.s, g.t, g.tail, g.head, g.cap, want_flow=False, want_cut=False, work_limit=limit)
    scans, secs = 0, 0.0
    for _ in range(args.steps):
        r = oracle.maxflow(g.n, g.s, g.t, g.tail, g.head, g.cap, want_flow=False, want_cut=False, work_limit=limit)
        scans += r["stats"]["scans"]
        secs += r["seconds"]
    value = scans / secs
    sample = (f"each step: sequential FIFO push-relabel phase 1 on the full {g.name}, stopped after about {limit} "
              f"arc scans ({secs / max(args.steps, 1):.1f} s)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * secs / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32/i64",
            "data": "synthetic", "config": workload_config(g, paired_slot_count(g.tail, g.head), world, WORKLOAD),
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)
    return 0


def golden_rows(name):
    """Per-instance stored oracle results of a multi-instance workload (tests/golden), or None."""
    p = os.path.join(ROOT, "tests", "golden", f"{name}.json")
    if not os.path.exists(p):
        return None
    g = json.load(open(p))
    return [dict(zip(g["fields"], r)) for r in g["rows"]]


def cut_digest(bits, n) -> str:
    """SHA-256 of a cut bitmap (uint32 words, bit v of word v // 32) as packed little-endian bytes of n bits,
    the form of the stored oracle results."""
    import hashlib

    b = np.unpackbits(np.asarray(bits, np.uint32).view(np.uint8), bitorder="little")[:n]
    return hashlib.sha256(np.packbits(b, bitorder="little").tobytes()).hexdigest()


def host_jobs() -> int:
    return max(1, min(32, os.cpu_count() or 1))


class Feeder:
    """Builds instances i = 0, 1, ... (their paired-slot CSRs) on the host cores ahead of their use, at most
    `ahead` at a time; get(i) must be called in increasing order."""

    def __init__(self, make, count: int, jobs: int, ahead: int):
        from concurrent.futures import ThreadPoolExecutor

        self.make, self.count, self.ahead = make, count, ahead
        self.ex = ThreadPoolExecutor(jobs)
        self.futs = {i: self.ex.submit(make, i) for i in range(min(ahead, count))}

    def get(self, i: int):
        item = self.futs.pop(i).result()
        if i + self.ahead < self.count:
            self.futs[i + self.ahead] = self.ex.submit(self.make, i + self.ahead)
        return item

    def close(self):
        self.ex.shutdown(wait=True, cancel_futures=True)


def batch_section(args) -> dict:
    """The batch of 2048 uneven layered graphs (L ~ logU[16,256] layers of W ~ logU[64,4096] vertices).
    Batched = all instances in one persistent launch (mf_batch_solve, graph-captured replay, the autotuner's
    packaged choice for this batch); plain = one mf_solve launch per instance, on the same instances, with the
    faster of the defaults and the batch's options (picked on a strided sample). Reports solves/s of both, the
    ratio, the batch kernel's roofline and the parity of every instance with the oracle's stored results."""
    import torch

    from paper_1507_01926_gb300 import autotune, inputs, mf

    torch.cuda.set_device(0)
    params = inputs.layered_batch_params(args.batch_count)

    def make(i):
        L, W = params[i]
        g = inputs.layered_batch_instance(i, L, W)
        c = mf.build_csr(g.n, g.tail, g.head, g.cap)
        c.arc_slot = None
        return c, (g.s, g.t)

    t0 = time.perf_counter()
    from concurrent.futures import ThreadPoolExecutor

    with ThreadPoolExecutor(host_jobs()) as ex:
        built = list(ex.map(make, range(len(params))))
    csrs, sts = [b[0] for b in built], [b[1] for b in built]
    del built
    prep_s = time.perf_counter() - t0
    nv, ns = sum(c.n for c in csrs), sum(c.m for c in csrs)
    key = autotune.workload_key("layered", nv, ns, len(csrs))
    hit = autotune.lookup(key, autotune.device_name(0))
    opt = hit[0] if hit else mf.default_options()
    opt.device = 0
    opt.use_graph = 0 if args.no_graph else 1
    apply_overrides(opt, args)
    gold = golden_rows(f"layered_batch_{len(csrs)}")
    # batched: the whole batch in one launch
    t0 = time.perf_counter()
    B = mf.Batch(csrs, sts, opt)
    create_s = time.perf_counter() - t0
    first = B.solve(flow=False, cut=True)  # warm-up, and the parity check of every instance
    matched = None
    if gold is not None:
        matched = sum(1 for i, r in enumerate(first)
                      if r.value == gold[i]["value"] and cut_digest(r.cut_bits, csrs[i].n) == gold[i]["cut_sha256"])
    del first
    times, stats = [], []
    for _ in range(max(1, args.batch_steps)):
        t0 = time.perf_counter()
        B.solve(flow=False, cut=False)
        times.append(time.perf_counter() - t0)
        stats.append(B.stats())
    B.close()
    full_s = statistics.median(times)
    st = stats[len(stats) // 2]
    # plain: one launch per instance; options picked on a strided sample
    popt = mf.default_options(device=0)
    sample = list(range(0, len(csrs), max(1, len(csrs) // 64)))

    def plain(idx, o):
        secs, vals = 0.0, []
        for i in idx:
            with mf.Graph.from_csr(csrs[i], *sts[i], o) as G:
                torch.cuda.synchronize()
                t = time.perf_counter()
                vals.append(G.solve(flow=False, cut=False).value)
                secs += time.perf_counter() - t
        return secs, vals

    pick = {}
    for tag, o in (("defaults", popt), ("batch options", opt)):
        o2 = mf.options_from_dict(mf.options_to_dict(o))
        o2.use_graph = 0
        pick[tag] = (plain(sample, o2)[0], o2)
    plain_tag = min(pick, key=lambda k: pick[k][0])
    plain_s, plain_vals = plain(range(len(csrs)), pick[plain_tag][1])
    plain_matched = None
    if gold is not None:
        plain_matched = sum(1 for i, v in enumerate(plain_vals) if v == gold[i]["value"])
    peak, peak_kind = peaks()
    mb = model_bytes(st, nv, ns)
    batched_rate, plain_rate = len(csrs) / full_s, len(csrs) / plain_s
    return {"workload": f"{len(csrs)} layered graphs, L~logU[16,256] layers of W~logU[64,4096], 4 next-layer arcs + "
                        f"1 in-layer arc per vertex, capacity U[1,10000], terminals 1e6",
            "instances": len(csrs), "vertices": nv, "slots": ns,
            "batched_solves_per_s": batched_rate, "batched_s": full_s, "batched_s_all": [round(x, 3) for x in times],
            "plain_solves_per_s": plain_rate, "plain_s": plain_s, "plain_instances": len(csrs),
            "plain_options": plain_tag, "plain_sample_s_by_options": {k: v[0] for k, v in pick.items()},
            "batched_vs_plain": batched_rate / plain_rate,
            "parity": {"instances": len(csrs), "value_and_cut_match_oracle": matched,
                       "plain_values_match_oracle": plain_matched,
                       "golden": f"tests/golden/layered_batch_{len(csrs)}.json" if gold else None},
            "rounds": st["rounds"], "global_relabels": st["global_relabels"],
            "global_relabels_partial": st["global_relabels_partial"], "kernel_ms": st["solve_ms"],
            "host_prep_s": prep_s, "create_s": create_s,
            "roofline": {"bound": "hbm", "achieved": mb / st["solve_ms"] * 1e-6, "peak": peak, "unit": "GB/s",
                         "frac": mb / st["solve_ms"] * 1e-6 / peak, "traffic": None, "peak_kind": peak_kind,
                         "kernel": "mf::solve_kernel", "model_bytes_per_launch": mb,
                         "scans_per_launch": st["scans_discharge"] + st["scans_bfs"],
                         "phases": phase_rooflines(st, nv, peak)},
            "options": {"tuned": ("cached autotuner choice" if hit else "defaults (no cached choice)")
                        + (f", overridden by {args.options}" if args.options else ""),
                        "use_graph": int(opt.use_graph),
                        **{f: getattr(opt, f) for f in ("gr_time_ratio", "gr_freq", "bin_thread", "bin_warp",
                                                        "block_threads", "blocks_per_sm", "kernel_variant",
                                                        "instance_relabel")}}}


def stream_run(svc, feeder, count, arrivals, gold, check_upto):
    """Submits requests 0..count-1 at their arrival times (seconds from the start; the submitting thread
    sleeps until each), collects every result in order on a second thread, and checks value and cut of the
    first check_upto requests against the stored oracle results. Returns latencies (ms, submission to
    completion as the service measures them), the wall time from the first submission to the last completion,
    the submission lag behind the arrival times (ms), and the number of checked requests that matched."""
    import queue

    q = queue.Queue()
    lat, out = [0.0] * count, {"matched": 0, "checked": 0, "error": None}

    def collect():
        try:
            for _ in range(count):
                i, tk, n = q.get()
                lat[i] = svc.wait(tk)
                want_cut = gold is not None and i < check_upto
                r = svc.poll(tk, flow=False, cut=want_cut)
                if want_cut:
                    out["checked"] += 1
                    if r.value == gold[i]["value"] and cut_digest(r.cut_bits, n) == gold[i]["cut_sha256"]:
                        out["matched"] += 1
            out["t_end"] = time.perf_counter()
        except Exception as e:  # reported by the caller
            out["error"] = repr(e)

    th = threading.Thread(target=collect, daemon=True)
    th.start()
    lag = []
    t_start = time.perf_counter()
    for i in range(count):
        c, (s, t) = feeder.get(i)
        now = time.perf_counter() - t_start
        if arrivals[i] > now:
            time.sleep(arrivals[i] - now)
            now = time.perf_counter() - t_start
        lag.append(1000.0 * max(0.0, now - arrivals[i]))
        q.put((i, svc.submit(c, s, t), c.n))
    th.join()
    if out["error"]:
        raise RuntimeError(out["error"])
    return lat, out["t_end"] - t_start, lag, out


def serve_section(args) -> dict:
    """The serving stream: requests arriving as a Poisson process, half 2D grids of side logU[32,1024], half
    multi-frame grids of F ~ U[4,64] frames of 128x128, through the continuous-batching service under a 64 GB
    device budget. First the saturated throughput X on the first --serve-prefix requests (all submitted as
    soon as they are built), then the whole stream of --requests at 0.7 X; reports solves/s and p50/p99
    latency, and checks value and cut of the requests that have stored oracle results."""
    import torch

    from paper_1507_01926_gb300 import inputs, mf

    torch.cuda.set_device(0)
    N = args.requests
    P = min(args.serve_prefix, N)
    reqs = inputs.serving_stream_requests(N, rate_per_s=1.0)
    gold = golden_rows("serving_stream_1000")
    check_upto = len(gold) if gold else 0

    def make(i):
        _, kind, size = reqs[i]
        g = inputs.serving_stream_instance(i, kind, size)
        c = mf.build_csr(g.n, g.tail, g.head, g.cap)
        c.arc_slot = None
        return c, (g.s, g.t)

    budget = 64 << 30
    sopt = apply_overrides(mf.service_default_options(device=0), args)
    jobs = host_jobs()
    # saturated throughput on the prefix
    feeder = Feeder(make, P, jobs, 4 * jobs)
    with mf.Service(budget, sopt) as svc:
        lat0, wall0, _, chk0 = stream_run(svc, feeder, P, [0.0] * P, gold, check_upto)
    feeder.close()
    X = P / wall0
    rate = args.serve_load * X
    feeder = Feeder(make, N, jobs, 4 * jobs)
    arrivals = [a / rate for a, _, _ in reqs]
    with mf.Service(budget, sopt) as svc:
        lat, wall, lag, chk = stream_run(svc, feeder, N, arrivals, gold, check_upto)
    feeder.close()
    nv = sum((s * s if k == "grid" else 16384 * s + 2) for _, k, s in reqs)
    return {"workload": f"serving stream of {N} requests: Poisson arrivals, half 2D grids of side logU[32,1024], "
                        f"half multi-frame grids of U[4,64] frames of 128x128; 64 GB device budget",
            "requests": N, "vertices": nv, "budget_bytes": budget,
            "saturated": {"requests": P, "solves_per_s": X, "p50_ms": float(np.percentile(lat0, 50)),
                          "p99_ms": float(np.percentile(lat0, 99))},
            "load": args.serve_load, "rate_per_s": rate, "solves_per_s": N / wall, "seconds": wall,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "p50_ms_grids": float(np.percentile([x for x, r in zip(lat, reqs) if r[1] == "grid"], 50)),
            "p50_ms_frames": float(np.percentile([x for x, r in zip(lat, reqs) if r[1] == "frames"], 50)),
            "submit_lag_ms": {"p50": float(np.percentile(lag, 50)), "p99": float(np.percentile(lag, 99)),
                              "max": float(max(lag))},
            "parity": {"checked": chk["checked"], "value_and_cut_match_oracle": chk["matched"],
                       "checked_saturated": chk0["checked"], "matched_saturated": chk0["matched"],
                       "golden": "tests/golden/serving_stream_1000.json" if gold else None},
            "latency": "submission to completion, measured by the service (mf_wait)",
            "options": "service defaults (mf_service_default_options: lanes of 128-thread CTAs)"
                       + (f", overridden by {args.options}" if args.options else "")}


def run_batch(args):
    line = {"metric": "batched solves/s (layered batch)", "unit": "solves/s", "n_gpus": 1, "higher_is_better": True,
            "data": "synthetic", **batch_section(args)}
    line["value"] = line["batched_solves_per_s"]
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    line = {"metric": "served solves/s with p50/p99 latency (Poisson stream)", "unit": "solves/s", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic", **serve_section(args)}
    line["value"] = line["solves_per_s"]
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--grid3d", type=int, nargs=3, default=[256, 256, 128], metavar=("X", "Y", "Z"),
                    help="size of the 3D grid workload (profiling runs use a smaller case)")
    ap.add_argument("--workload", default="all", choices=["all", "grid3d", "batch", "serve"],
                    help="all (default): the 3D grid line with the batch and serving results in it")
    ap.add_argument("--batch-count", type=int, default=2048)
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--requests", type=int, default=20000)
    ap.add_argument("--serve-prefix", type=int, default=1000, help="requests of the saturated run that sets X")
    ap.add_argument("--serve-load", type=float, default=0.7, help="arrival rate of the stream as a fraction of X")
    ap.add_argument("--no-graph", action="store_true", help="batch workload: launch directly, no CUDA graphs")
    ap.add_argument("--options", default="", help="JSON object of mf_options fields applied over the chosen options")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)

    import torch

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    import __graft_entry__

    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_1507_01926_gb300 import mf

    g, csr = load_workload(args.grid3d)
    # the autotuner's cached choice for this workload on this device (the packaged GB300 table when the
    # user's cache has none), else the defaults
    from paper_1507_01926_gb300 import autotune

    hit = autotune.lookup(autotune.workload_key("grid3d", g.n, csr.m), autotune.device_name(torch.cuda.current_device()))
    opt = hit[0] if hit else mf.default_options()
    opt.device = torch.cuda.current_device()
    apply_overrides(opt, args)
    stream = torch.cuda.Stream()
    row = torch.from_numpy(csr.row_offsets).to(dev)
    head = torch.from_numpy(csr.head).to(dev)
    cap = torch.from_numpy(csr.cap).to(dev)
    rev = torch.from_numpy(csr.rev).to(dev)
    torch.cuda.synchronize()
    G = mf.Graph.from_device(g.n, row, head, cap, rev, g.s, g.t, opt, stream=stream)
    del row, head, cap, rev
    val = torch.zeros(1, dtype=torch.int64, device=dev)
    flow = torch.zeros(csr.m, dtype=torch.int32, device=dev)
    cutw = torch.zeros((g.n + 31) // 32, dtype=torch.int32, device=dev)

    def step():
        G.solve_device(val, flow, cutw, stream=stream)

    for _ in range(max(3, args.warmup)):
        step()
    stream.synchronize()
    warm_stats = G.stats()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    per_step, stats = [], []
    with ClockSampler(torch.cuda.current_device()) as clk:
        for i in range(args.steps):
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
            stats.append(G.stats())
        stream.synchronize()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    per_step = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(per_step)
    scans = sum(s["scans_discharge"] + s["scans_bfs"] for s in stats)
    if world > 1:
        total_ms_max, scans_all = aggregate_ranks(total_ms, scans, dev)
    else:
        total_ms_max, scans_all = total_ms, float(scans)
    value = scans_all / (total_ms_max / 1000.0)
    flow_value = int(val.item())
    grec = golden_record() if tuple(args.grid3d) == (256, 256, 128) else None
    gold = grec["value"] if grec else None

    # roofline of the (only) kernel: the persistent solve kernel, one launch per step
    peak, peak_kind = peaks()
    mb = [model_bytes(s, g.n, csr.m) for s in stats]
    achieved = (sum(mb) / len(mb)) / (statistics.mean(per_step) / 1000.0) / 1e9
    traffic = None
    tp = os.path.join(ROOT, "profiles", "solve_kernel_grid3d_256x256x128.json")
    if os.path.exists(tp) and tuple(args.grid3d) == (256, 256, 128):
        rec = json.load(open(tp))
        if rec.get("kernel_source_sha256_16") == kernel_source_hash():
            traffic = rec.get("dram_bytes_per_launch")  # counters of this very kernel version

    if rank != 0:
        G.close()
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    # end to end through the C-ABI with host buffers: create (H2D) + solve + outputs (D2H) + destroy
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()  # noqa: E731
    h_row, h_head, h_cap, h_rev = pin(csr.row_offsets), pin(csr.head), pin(csr.cap), pin(csr.rev)
    h_flow = torch.zeros(csr.m, dtype=torch.int32).pin_memory().numpy()
    h_cut = torch.zeros((g.n + 31) // 32, dtype=torch.int32).pin_memory().numpy().view(np.uint32)
    e2e_t, e2e_scans = [], 0
    import ctypes

    L = mf.lib()
    for i in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = ctypes.c_void_p()
        mf._check(L.mf_create_graph(g.n, csr.m, mf._ptr(h_row), mf._ptr(h_head), mf._ptr(h_cap), mf._ptr(h_rev),
                                    g.s, g.t, ctypes.byref(opt), ctypes.byref(h)))
        v = ctypes.c_int64()
        mf._check(L.mf_solve(h, ctypes.byref(v), mf._ptr(h_flow), mf._ptr(h_cut)))
        s = mf.Stats()
        L.mf_get_stats(h, ctypes.byref(s))
        L.mf_destroy_graph(h)
        dt = time.perf_counter() - t0
        assert v.value == flow_value
        if i > 0:  # first call warms the allocator and the pinned path
            e2e_t.append(dt)
            e2e_scans += s.scans_discharge + s.scans_bfs
    h2d = 8 * (g.n + 1) + 4 * csr.m + 4 * csr.m + 8 * csr.m
    d2h = 8 + 4 * csr.m + 4 * ((g.n + 31) // 32)
    e2e = None
    if e2e_t:
        e2e = {"value": e2e_scans / sum(e2e_t), "unit": METRIC, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": 1000 * statistics.mean(e2e_t),
               "includes": "mf_create_graph (H2D from pinned memory + on-device validation) + mf_solve (flow, cut D2H)"}

    cpu = None if args.no_cpu_baseline else cpu_baseline(g)
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "i32/i64", "data": "synthetic",
        "config": workload_config(g, csr.m, world, WORKLOAD if tuple(args.grid3d) == (256, 256, 128) else g.name),
        "solve_ms": statistics.median(per_step), "solve_ms_all": [round(x, 3) for x in per_step],
        "preflow_ms": statistics.median(s["preflow_ms"] for s in stats),
        "flow_value": flow_value, "flow_value_matches_oracle": (gold == flow_value) if gold is not None else None,
        "solve_time_vs_oracle": ({"oracle_full_solve_s": grec["oracle_seconds"],
                                  "gpu_full_solve_s": statistics.median(per_step) / 1000.0,
                                  "ratio": grec["oracle_seconds"] / (statistics.median(per_step) / 1000.0),
                                  "note": "the like-for-like comparison: the oracle's arc scans count the entries of "
                                          "its own adjacency (two per input arc), the GPU's the slots of the paired-"
                                          "slot CSR (antiparallel arcs share a slot pair)"}
                                 if grec else None),
        "rounds": stats[-1]["rounds"], "global_relabels": stats[-1]["global_relabels"],
        "scans_per_solve": scans / args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_kind": peak_kind, "kernel": "mf::solve_kernel",
                     "peak_nominal": HBM_NOMINAL_GBS, "frac_nominal": achieved / HBM_NOMINAL_GBS,
                     "traffic_GBps": (traffic / (statistics.mean(per_step) / 1000.0) / 1e9) if traffic else None,
                     "model_bytes_per_launch": statistics.mean(mb),
                     "phases": phase_rooflines(stats[len(stats) // 2], g.n, peak)},
        "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks, "gpu_launches": args.steps,
        "grid": [warm_stats["grid_blocks"], warm_stats["block_threads"]],
        "options": {"tuned": ("cached autotuner choice" if hit else "defaults (no cached choice)")
                        + (f", overridden by {args.options}" if args.options else ""),
                    **{f: getattr(opt, f) for f in ("gr_time_ratio", "gr_freq", "bin_thread", "bin_warp",
                                                    "block_threads", "blocks_per_sm", "kernel_variant",
                                                    "local_lists", "bfs_hops")}},
    }
    G.close()
    del val, flow, cutw
    torch.cuda.empty_cache()
    if args.workload == "all" and world == 1:
        line["batch"] = batch_section(args)
        line["serve"] = serve_section(args)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
