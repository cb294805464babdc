"""CPU oracle for maximum flow / minimum cut (ctypes wrapper over ``oracle.c``).

TEST INFRASTRUCTURE ONLY. Tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may call it; the solver package never imports it. It shares no code with the GPU path.

Everything here follows arXiv:1507.01926: Section 2 (flows, residual graphs, max-flow = min-cut,
S_min = residual reachability from s), Section 2.1 (push-relabel, FIFO order, global relabeling,
maximum preflow then flow), Section 3 and Algorithms 1-2 (global-relabel schedule and reverse BFS).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

ERRORS = {-1: "invalid argument", -2: "out of memory", -3: "work limit reached",
          -4: "cut identity failed", -5: "excess left after phase 2", -6: "invariant failed (checked mode)"}

# checked mode: what the failure code of maxflow_checked means (oracle.c, check_state)
CHECK_FAILURES = {1: "negative residual", 2: "arc pair capacity not kept", 3: "negative excess",
                  4: "excess differs from net inflow", 5: "invalid label: d(u) > d(w) + 1 on a residual arc"}


def build_lib(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc -O2, single-threaded, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_lib())
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        lib.orc_maxflow.argtypes = [i32, i64, vp, vp, vp, i32, i32, i64, vp, vp, vp]
        lib.orc_maxflow.restype = i64
        lib.orc_maxflow_checked.argtypes = [i32, i64, vp, vp, vp, i32, i32, i32, vp, vp, vp, vp]
        lib.orc_maxflow_checked.restype = i64
        lib.orc_edmonds_karp.argtypes = [i32, i64, vp, vp, vp, i32, i32, vp]
        lib.orc_edmonds_karp.restype = i64
        lib.orc_bruteforce_cut.argtypes = [i32, i64, vp, vp, vp, i32, i32, vp]
        lib.orc_bruteforce_cut.restype = i64
        lib.orc_sink_distances.argtypes = [i32, i64, vp, vp, i32, i32, vp]
        lib.orc_sink_distances.restype = ctypes.c_int
        lib.orc_check_flow.argtypes = [i32, i64, vp, vp, vp, i32, i32, vp, i64, vp]
        lib.orc_check_flow.restype = ctypes.c_int
        _lib = lib
    return _lib


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    pass


def _check(rc):
    if rc < 0:
        raise OracleError(ERRORS.get(int(rc), f"error {rc}"))
    return rc


def maxflow(n, s, t, tail, head, cap, want_flow=True, want_cut=True, work_limit=0):
    """Two-phase FIFO push-relabel. Returns dict(value, flow (int64[m]) or None, cut (bool[n]) or
    None, stats dict, seconds)."""
    tail, head, cap = _i32(tail), _i32(head), _i32(cap)
    m = tail.shape[0]
    flow = np.zeros(m, np.int64) if want_flow else None
    cut = np.zeros(n, np.uint8) if want_cut else None
    st = np.zeros(8, np.int64)
    t0 = time.perf_counter()
    v = _L().orc_maxflow(n, m, _p(tail), _p(head), _p(cap), s, t, int(work_limit), _p(flow), _p(cut), _p(st))
    sec = time.perf_counter() - t0
    keys = ["scans", "pushes", "relabels", "global_relabels", "p1_scans", "p1_pushes", "p1_relabels",
            "p1_global_relabels"]
    stats = dict(zip(keys, (int(x) for x in st)))
    if v == -3 and work_limit > 0:
        return dict(value=None, flow=None, cut=None, stats=stats, seconds=sec, truncated=True)
    _check(v)
    return dict(value=int(v), flow=flow, cut=None if cut is None else cut.astype(bool), stats=stats,
                seconds=sec, truncated=False)


def maxflow_checked(n, s, t, tail, head, cap, plant=False):
    """maxflow with the push-relabel invariants checked after every global relabel, relabel and discharge
    (residual bounds, pair capacities, excess = net inflow, label validity d(u) <= d(w) + 1 on residual
    arcs; Section 2.1). plant=True plants a mistake in relabel (one too high) to show that the checker
    catches it. Returns dict(value or None, cut or None, checks, failed: 0 or the CHECK_FAILURES code)."""
    tail, head, cap = _i32(tail), _i32(head), _i32(cap)
    m = tail.shape[0]
    cut = np.zeros(n, np.uint8)
    st = np.zeros(8, np.int64)
    chk = np.zeros(2, np.int64)
    v = _L().orc_maxflow_checked(n, m, _p(tail), _p(head), _p(cap), s, t, 1 if plant else 0, None, _p(cut),
                                 _p(st), _p(chk))
    failed = int(chk[1])
    if v == -6:
        return dict(value=None, cut=None, checks=int(chk[0]), failed=failed)
    _check(v)
    return dict(value=int(v), cut=cut.astype(bool), checks=int(chk[0]), failed=failed)


def edmonds_karp(n, s, t, tail, head, cap):
    """Returns (value, cut bool[n]) by shortest augmenting paths."""
    tail, head, cap = _i32(tail), _i32(head), _i32(cap)
    cut = np.zeros(n, np.uint8)
    v = _check(_L().orc_edmonds_karp(n, tail.shape[0], _p(tail), _p(head), _p(cap), s, t, _p(cut)))
    return int(v), cut.astype(bool)


def bruteforce_cut(n, s, t, tail, head, cap):
    """Returns (min cut capacity, S_min bool[n]) by enumerating all source sides (n <= 22)."""
    tail, head, cap = _i32(tail), _i32(head), _i32(cap)
    smin = np.zeros(n, np.uint8)
    v = _check(_L().orc_bruteforce_cut(n, tail.shape[0], _p(tail), _p(head), _p(cap), s, t, _p(smin)))
    return int(v), smin.astype(bool)


def sink_distances(n, s, t, rtail, rhead):
    """Exact global-relabel labels for the residual graph whose residual arcs are rtail -> rhead."""
    rtail, rhead = _i32(rtail), _i32(rhead)
    d = np.zeros(n, np.int32)
    _check(_L().orc_sink_distances(n, rtail.shape[0], _p(rtail), _p(rhead), s, t, _p(d)))
    return d


CHECK_BITS = {1: "capacity bounds", 2: "conservation", 4: "source outflow != value", 8: "sink inflow != value",
              16: "residual s-t path", 32: "cut misses s or holds t", 64: "cut capacity != value",
              128: "cut != residual reachability from s"}


def check_flow(n, s, t, tail, head, cap, flow, value, cut=None):
    """Returns the list of violated definitions (empty list = a valid maximum flow with matching cut)."""
    tail, head, cap = _i32(tail), _i32(head), _i32(cap)
    flow = np.ascontiguousarray(flow, dtype=np.int64)
    c = None if cut is None else np.ascontiguousarray(cut, dtype=np.uint8)
    bad = _check(_L().orc_check_flow(n, tail.shape[0], _p(tail), _p(head), _p(cap), s, t, _p(flow), int(value),
                                     _p(c)))
    return [msg for bit, msg in CHECK_BITS.items() if bad & bit]
