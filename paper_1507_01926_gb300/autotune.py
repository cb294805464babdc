"""Cached autotuning of solver options (mf_autotune / mf_batch_autotune in include/mf.h).

The search itself runs in libmf (coordinate descent over candidate relabel triggers, degree bins, launch
shapes and register budgets, every candidate timed on the GPU and checked to reproduce the flow values).
This module only keeps its choices: a JSON file maps a device name and a workload key to the chosen
options and their median solve time, so that a workload family is tuned once per device and later runs
start from the cached options.

Cache layout::

    {"<device name>": {"<workload key>": {"options": {<mf_options fields>}, "ms": <median solve ms>}}}

A lookup that misses the user's cache falls back to ``tuned_gb300.json`` beside this module: the choices
of the same search on a GB300 for the three standing workloads (the 256x256x128 3D grid, R-MAT scale 22 and
the batch of 2048 layered graphs), written by ``python -m paper_1507_01926_gb300.autotune --out
paper_1507_01926_gb300/tuned_gb300.json <workload>`` (each entry's ``tuned_on`` field records the instances,
reps and sweeps it was tuned with).
"""
from __future__ import annotations

import json
import os
import tempfile

from . import mf

DEFAULT_CACHE = os.environ.get("MF_TUNE_CACHE",
                               os.path.join(os.path.expanduser("~"), ".cache", "paper_1507_01926_gb300_tune.json"))
PACKAGED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_gb300.json")


def workload_key(family: str, n: int, m: int, count: int = 1) -> str:
    """Key of a workload family and size class: sizes are rounded to powers of two, so that instances of one
    family and similar size share their tuned options."""

    def p2(x):
        return max(int(x), 1).bit_length()

    return f"{family}/n2^{p2(n)}/m2^{p2(m)}/x{p2(count)}"


def device_name(device: int = 0) -> str:
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.get_device_name(device)
    except Exception:
        pass
    return f"cuda:{device}"


def load_cache(path: str = DEFAULT_CACHE) -> dict:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(data: dict, path: str = DEFAULT_CACHE) -> None:
    """Writes the cache atomically (a temporary file renamed over the old one)."""
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=d, prefix=".tune", suffix=".json")
    with os.fdopen(fd, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(key: str, device: str, path: str = DEFAULT_CACHE, packaged: bool = True):
    """(Options, ms) cached for (device, key) in `path`, else (packaged=True) in the packaged GB300 table,
    else None."""
    e = load_cache(path).get(device, {}).get(key)
    if not e and packaged:
        e = load_cache(PACKAGED).get(device, {}).get(key)
    if not e:
        return None
    return mf.options_from_dict(e["options"]), float(e["ms"])


def store(key: str, device: str, options: mf.Options, ms: float, path: str = DEFAULT_CACHE) -> None:
    data = load_cache(path)
    data.setdefault(device, {})[key] = {"options": mf.options_to_dict(options), "ms": float(ms)}
    save_cache(data, path)


def tuned(target, key: str, path: str = DEFAULT_CACHE, reps: int = 3, sweeps: int = 1,
          time_budget_ms: float = 0.0, device: int = 0, retune: bool = False):
    """Options for `target` (an mf.Graph or mf.Batch) under workload `key`: the cached choice when there is
    one (applied with set_options), else a fresh mf_autotune run whose result is cached. Returns
    (Options, median ms, from_cache)."""
    dev = device_name(device)
    hit = None if retune else lookup(key, dev, path)
    if hit is not None:
        opts, ms = hit
        opts.device = device
        target.set_options(opts)
        return opts, ms, True
    opts, ms = target.autotune(reps=reps, sweeps=sweeps, time_budget_ms=time_budget_ms)
    store(key, dev, opts, ms, path)
    return opts, ms, False


def _standing_workload(name: str, batch_sample: int = 2048):
    """(key, target factory, note) of a standing workload: the 256x256x128 3D grid, R-MAT scale 22, or the
    batch of 2048 layered graphs (tuned on its first `batch_sample` instances, stored under the full batch's
    key)."""
    from . import inputs as I

    if name == "layered":
        params = I.layered_batch_params()
        n_all = m_all = 0
        csrs, sts = [], []
        for i, (L, W) in enumerate(params):
            g = I.layered_batch_instance(i, L, W)
            c = mf.build_csr(g.n, g.tail, g.head, g.cap)
            n_all, m_all = n_all + c.n, m_all + c.m
            if i < batch_sample:
                c.arc_slot = None
                csrs.append(c)
                sts.append((g.s, g.t))
        key = workload_key("layered", n_all, m_all, len(params))
        which = "all" if len(csrs) == len(params) else f"first {len(csrs)} of the"
        return key, (lambda: mf.Batch(csrs, sts)), f"{which} 2048 layered graphs, mf_batch_autotune"
    g = {"grid3d": I.grid3d_256x256x128, "rmat": I.rmat_s22_ef16}[name]()
    c = mf.build_csr(g.n, g.tail, g.head, g.cap)
    return workload_key(name, g.n, c.m), (lambda: mf.Graph.from_csr(c, g.s, g.t)), f"{g.name}, mf_autotune"


def main(argv=None) -> int:
    """Tunes the named standing workloads on cuda:0 and stores the choices (GPU required)."""
    import argparse

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("workloads", nargs="+", choices=["grid3d", "rmat", "layered"])
    ap.add_argument("--out", default=DEFAULT_CACHE)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--sweeps", type=int, default=2)
    ap.add_argument("--batch-sample", type=int, default=2048, help="layered instances the batch is tuned on")
    a = ap.parse_args(argv)
    dev = device_name(0)
    for name in a.workloads:
        key, make, note = _standing_workload(name, a.batch_sample)
        with make() as target:
            opts, ms = target.autotune(reps=a.reps, sweeps=a.sweeps)
        store(key, dev, opts, ms, a.out)
        data = load_cache(a.out)
        data[dev][key]["tuned_on"] = f"{note} reps={a.reps} sweeps={a.sweeps}"
        save_cache(data, a.out)
        print(json.dumps({"workload": name, "key": key, "ms": ms, "options": mf.options_to_dict(opts)}), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
