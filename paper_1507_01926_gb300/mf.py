"""Python binding of libmf (include/mf.h): argument marshalling only.

Every step of the solve runs in the CUDA kernels of ``libmf.so``; this module converts numpy arrays or
torch tensors to pointers and raises ``MFError`` on a non-zero status. If ``libmf.so`` has not been
built, importing the library fails loudly (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmf.so")

MF_OK, MF_PENDING = 0, 1
ERR_NAMES = {-1: "MF_ERR_INVALID_ARG", -2: "MF_ERR_BAD_PAIRING", -3: "MF_ERR_S_EQ_T", -4: "MF_ERR_CAP_OVERFLOW",
             -5: "MF_ERR_OOM", -6: "MF_ERR_OVER_BUDGET", -7: "MF_ERR_ITER_LIMIT", -8: "MF_ERR_TIMEOUT",
             -9: "MF_ERR_CUDA", -10: "MF_ERR_INTERNAL", -11: "MF_ERR_TOO_LARGE", -12: "MF_ERR_UNKNOWN_TICKET"}


class MFError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("gr_freq", ctypes.c_double), ("gr_alpha", ctypes.c_int32), ("work_beta", ctypes.c_int32),
                ("bin_thread", ctypes.c_int32), ("bin_warp", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("max_rounds", ctypes.c_int64), ("timeout_ms", ctypes.c_int32),
                ("cut_only", ctypes.c_int32), ("device", ctypes.c_int32), ("gr_time_ratio", ctypes.c_double),
                ("kernel_variant", ctypes.c_int32), ("simple_rounds", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("local_lists", ctypes.c_int32), ("bfs_hops", ctypes.c_int32), ("gap_every", ctypes.c_int32),
                ("bfs_pull", ctypes.c_int32), ("union_max_requests", ctypes.c_int32),
                ("instance_relabel", ctypes.c_int32)]


class TuneSpec(ctypes.Structure):
    _fields_ = [("reps", ctypes.c_int32), ("sweeps", ctypes.c_int32), ("time_budget_ms", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int64), ("rounds_phase1", ctypes.c_int64), ("global_relabels", ctypes.c_int64),
                ("bfs_levels", ctypes.c_int64), ("scans_discharge", ctypes.c_int64), ("scans_bfs", ctypes.c_int64),
                ("pushes", ctypes.c_int64), ("relabels", ctypes.c_int64), ("visits_discharge", ctypes.c_int64),
                ("visits_bfs", ctypes.c_int64), ("solve_ms", ctypes.c_double),
                ("preflow_ms", ctypes.c_double), ("relabel_ms", ctypes.c_double), ("discharge_ms", ctypes.c_double),
                ("rounds_by_size", ctypes.c_int64 * 4), ("round_work_ms", ctypes.c_double),
                ("round_tail_ms", ctypes.c_double), ("round_wait_ms", ctypes.c_double),
                ("level_work_ms", ctypes.c_double), ("level_wait_ms", ctypes.c_double),
                ("grid_blocks", ctypes.c_int32), ("block_threads", ctypes.c_int32), ("gap_lifted", ctypes.c_int64),
                ("scans_discharge_residual", ctypes.c_int64), ("global_relabels_partial", ctypes.c_int64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["rounds_by_size"] = list(d["rounds_by_size"])
        return d


class _CSR(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int64), ("row_offsets", ctypes.POINTER(ctypes.c_int64)),
                ("head", ctypes.POINTER(ctypes.c_int32)), ("cap", ctypes.POINTER(ctypes.c_int32)),
                ("rev", ctypes.POINTER(ctypes.c_int64)), ("arc_slot", ctypes.POINTER(ctypes.c_int64)),
                ("dropped_self_loops", ctypes.c_int64)]


class GraphDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int64), ("row_offsets", ctypes.c_void_p),
                ("head", ctypes.c_void_p), ("cap", ctypes.c_void_p), ("rev", ctypes.c_void_p),
                ("s", ctypes.c_int32), ("t", ctypes.c_int32)]


_lib = None
EXPORTS = ["mf_default_options", "mf_service_default_options", "mf_struct_sizes", "mf_last_error", "mf_build_csr", "mf_free_csr", "mf_create_graph",
           "mf_create_graph_device", "mf_solve", "mf_solve_device", "mf_get_stats", "mf_run_rounds",
           "mf_solve_trace", "mf_destroy_graph", "mf_batch_create", "mf_batch_solve", "mf_batch_get_stats",
           "mf_batch_destroy", "mf_service_create", "mf_submit", "mf_poll", "mf_wait", "mf_service_destroy",
           "mf_set_options", "mf_autotune", "mf_batch_set_options", "mf_batch_autotune"]


def use_library(path: str | None):
    """Makes every later call of this module go to the library at `path` (None: back to libmf.so); used by the
    tests of the build with checked gathers (libmf_check.so). Returns the path in use before."""
    global _lib, LIB_PATH
    before = LIB_PATH
    LIB_PATH = path or os.path.join(_HERE, "libmf.so")
    _lib = None
    return before


def lib():
    """Loads libmf.so (raises OSError if it is missing or cannot be loaded)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.mf_default_options.argtypes = [ctypes.POINTER(Options)]
        L.mf_default_options.restype = None
        L.mf_service_default_options.argtypes = [ctypes.POINTER(Options)]
        L.mf_service_default_options.restype = None
        L.mf_last_error.restype = ctypes.c_char_p
        L.mf_build_csr.argtypes = [i32, i64, vp, vp, vp, ctypes.POINTER(_CSR)]
        L.mf_free_csr.argtypes = [ctypes.POINTER(_CSR)]
        L.mf_free_csr.restype = None
        L.mf_create_graph.argtypes = [i32, i64, vp, vp, vp, vp, i32, i32, ctypes.POINTER(Options),
                                      ctypes.POINTER(vp)]
        L.mf_create_graph_device.argtypes = [i32, i64, vp, vp, vp, vp, i32, i32, ctypes.POINTER(Options), vp,
                                             ctypes.POINTER(vp)]
        L.mf_solve.argtypes = [vp, vp, vp, vp]
        L.mf_solve_device.argtypes = [vp, vp, vp, vp, vp]
        L.mf_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
        L.mf_run_rounds.argtypes = [vp, i64, i32, vp, vp, vp, vp]
        L.mf_solve_trace.argtypes = [vp, vp, vp, i64, vp, vp, i64, vp, vp, vp]
        L.mf_destroy_graph.argtypes = [vp]
        L.mf_destroy_graph.restype = None
        L.mf_batch_create.argtypes = [i32, vp, ctypes.POINTER(Options), ctypes.POINTER(vp)]
        L.mf_batch_solve.argtypes = [vp, vp, vp, vp]
        L.mf_batch_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
        L.mf_batch_destroy.argtypes = [vp]
        L.mf_batch_destroy.restype = None
        L.mf_service_create.argtypes = [ctypes.c_size_t, ctypes.POINTER(Options), ctypes.POINTER(vp)]
        L.mf_submit.argtypes = [vp, ctypes.POINTER(GraphDesc), ctypes.POINTER(i64)]
        L.mf_poll.argtypes = [vp, i64, vp, vp, vp]
        L.mf_wait.argtypes = [vp, i64, i32, ctypes.POINTER(ctypes.c_double)]
        L.mf_service_destroy.argtypes = [vp]
        L.mf_service_destroy.restype = None
        for f in (L.mf_set_options, L.mf_batch_set_options):
            f.argtypes = [vp, ctypes.POINTER(Options)]
        for f in (L.mf_autotune, L.mf_batch_autotune):
            f.argtypes = [vp, ctypes.POINTER(TuneSpec), ctypes.POINTER(Options), ctypes.POINTER(ctypes.c_double)]
        L.mf_struct_sizes.argtypes = [ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.mf_struct_sizes.restype = None
        ob, sb = i32(), i32()
        L.mf_struct_sizes(ctypes.byref(ob), ctypes.byref(sb))
        if (ob.value, sb.value) != (ctypes.sizeof(Options), ctypes.sizeof(Stats)):
            raise OSError(f"{LIB_PATH} was built with mf_options/mf_stats of {ob.value}/{sb.value} bytes, the binding "
                          f"expects {ctypes.sizeof(Options)}/{ctypes.sizeof(Stats)}: rebuild it")
        _lib = L
    return _lib


def _check(rc: int):
    if rc < 0:
        raise MFError(rc, lib().mf_last_error().decode(errors="replace"))
    return rc


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(a.data_ptr())  # torch tensor


def _stream_ptr(stream):
    if stream is None:
        import torch

        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def default_options(**overrides) -> Options:
    o = Options()
    lib().mf_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def service_default_options(**overrides) -> Options:
    """mf_service_default_options (what mf_service_create uses without options), with overrides."""
    o = Options()
    lib().mf_service_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def options_to_dict(o: Options) -> dict:
    return {k: getattr(o, k) for k, _ in Options._fields_}


def options_from_dict(d: dict) -> Options:
    o = default_options()
    for k, v in d.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _autotune(fn, h, reps, sweeps, time_budget_ms):
    spec = TuneSpec(int(reps), int(sweeps), float(time_budget_ms))
    best = Options()
    ms = ctypes.c_double()
    _check(fn(h, ctypes.byref(spec), ctypes.byref(best), ctypes.byref(ms)))
    return best, float(ms.value)


@dataclass
class CSR:
    """Paired-slot CSR (see include/mf.h)."""

    n: int
    row_offsets: np.ndarray  # int64[n+1]
    head: np.ndarray         # int32[m]
    cap: np.ndarray          # int32[m]
    rev: np.ndarray          # int64[m]
    arc_slot: np.ndarray     # int64[m_in]
    dropped_self_loops: int

    @property
    def m(self) -> int:
        return int(self.head.shape[0])

    def tails(self) -> np.ndarray:
        return np.repeat(np.arange(self.n, dtype=np.int32), np.diff(self.row_offsets))


def build_csr(n, tail, head, cap) -> CSR:
    tail = np.ascontiguousarray(tail, np.int32)
    head = np.ascontiguousarray(head, np.int32)
    cap = np.ascontiguousarray(cap, np.int32)
    c = _CSR()
    _check(lib().mf_build_csr(n, tail.shape[0], _ptr(tail), _ptr(head), _ptr(cap), ctypes.byref(c)))
    try:
        m = int(c.m)

        def grab(p, k):
            return np.ctypeslib.as_array(p, shape=(k,)).copy() if k else np.zeros(0, p._type_)

        return CSR(n, grab(c.row_offsets, n + 1), grab(c.head, m), grab(c.cap, m), grab(c.rev, m),
                   grab(c.arc_slot, tail.shape[0]), int(c.dropped_self_loops))
    finally:
        lib().mf_free_csr(ctypes.byref(c))


def cut_bits_to_bool(bits, n) -> np.ndarray:
    b = np.asarray(bits, dtype=np.uint32).view(np.uint8)
    return np.unpackbits(b, bitorder="little")[:n].astype(bool)


@dataclass
class Result:
    value: int
    flow: np.ndarray | None      # int32[m] per slot
    cut_bits: np.ndarray | None  # uint32[ceil(n/32)]


class Graph:
    """A max-flow instance resident on the GPU (mf_create_graph / mf_solve)."""

    def __init__(self, n, row_offsets, head, cap, rev, s, t, options: Options | None = None, _handle=None):
        self.n, self.s, self.t = int(n), int(s), int(t)
        self._h = ctypes.c_void_p()
        if _handle is not None:
            self._h = _handle
            self.m = int(head.shape[0]) if head is not None else 0
            return
        row_offsets = np.ascontiguousarray(row_offsets, np.int64)
        head = np.ascontiguousarray(head, np.int32)
        cap = np.ascontiguousarray(cap, np.int32)
        rev = np.ascontiguousarray(rev, np.int64)
        self.m = int(head.shape[0])
        _check(lib().mf_create_graph(self.n, self.m, _ptr(row_offsets), _ptr(head), _ptr(cap), _ptr(rev), self.s,
                                     self.t, ctypes.byref(options) if options else None, ctypes.byref(self._h)))

    @classmethod
    def from_csr(cls, csr: CSR, s, t, options: Options | None = None) -> "Graph":
        return cls(csr.n, csr.row_offsets, csr.head, csr.cap, csr.rev, s, t, options)

    @classmethod
    def from_device(cls, n, row_offsets, head, cap, rev, s, t, options: Options | None = None, stream=None):
        """From torch CUDA tensors (int64 row_offsets/rev, int32 head/cap)."""
        h = ctypes.c_void_p()
        m = int(head.shape[0])
        _check(lib().mf_create_graph_device(int(n), m, _ptr(row_offsets), _ptr(head), _ptr(cap), _ptr(rev), int(s),
                                            int(t), ctypes.byref(options) if options else None,
                                            _stream_ptr(stream), ctypes.byref(h)))
        g = cls(n, None, head, None, None, s, t, _handle=h)
        return g

    def solve(self, flow=True, cut=True) -> Result:
        v = ctypes.c_int64()
        f = np.zeros(self.m, np.int32) if flow else None
        c = np.zeros((self.n + 31) // 32, np.uint32) if cut else None
        _check(lib().mf_solve(self._h, ctypes.byref(v), _ptr(f), _ptr(c)))
        return Result(int(v.value), f, c)

    def solve_device(self, value=None, flow=None, cut_bits=None, stream=None):
        """Outputs into torch CUDA tensors (int64[1], int32[m], int32/uint32[ceil(n/32)]), each optional."""
        _check(lib().mf_solve_device(self._h, _stream_ptr(stream), _ptr(value), _ptr(flow), _ptr(cut_bits)))

    def solve_trace(self, capacity: int = 1 << 22, level_capacity: int = 1 << 22, times: bool = False):
        """One traced solve: (live int32[rounds], relabel int32[rounds], bfs frontier sizes int32[levels]), and
        with times=True also the durations in ns of every round and every BFS level (int32 each)."""
        live = np.zeros(capacity, np.int32)
        gr = np.zeros(capacity, np.int32)
        lv = np.zeros(level_capacity, np.int32)
        rns = np.zeros(capacity, np.int32) if times else None
        lns = np.zeros(level_capacity, np.int32) if times else None
        nr, nl = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().mf_solve_trace(self._h, _ptr(live), _ptr(gr), capacity, ctypes.byref(nr), _ptr(lv),
                                    level_capacity, ctypes.byref(nl), _ptr(rns), _ptr(lns)))
        k = min(int(nr.value), capacity)
        kl = min(int(nl.value), level_capacity)
        if times:
            return live[:k], gr[:k], lv[:kl], rns[:k], lns[:kl]
        return live[:k], gr[:k], lv[:kl]

    def stats(self) -> dict:
        s = Stats()
        _check(lib().mf_get_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def set_options(self, options: Options):
        _check(lib().mf_set_options(self._h, ctypes.byref(options)))

    def autotune(self, reps: int = 3, sweeps: int = 1, time_budget_ms: float = 0.0):
        """mf_autotune: times candidate options on this graph and keeps the fastest; returns (Options, median ms)."""
        return _autotune(lib().mf_autotune, self._h, reps, sweeps, time_budget_ms)

    def run_rounds(self, rounds: int, final_relabel: bool = True):
        """Phase-1 state after `rounds` rounds: (residual int32[m], label int32[n], excess int64[n], rounds)."""
        res = np.zeros(self.m, np.int32)
        lab = np.zeros(self.n, np.int32)
        ex = np.zeros(self.n, np.int64)
        done = ctypes.c_int64()
        _check(lib().mf_run_rounds(self._h, int(rounds), 1 if final_relabel else 0, _ptr(res), _ptr(lab), _ptr(ex),
                                   ctypes.byref(done)))
        return res, lab, ex, int(done.value)

    def close(self):
        if self._h:
            lib().mf_destroy_graph(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_instance(inst, options: Options | None = None, flow=True, cut=True):
    """Builds the CSR of an input arc list (tail/head/cap arrays, n, s, t) and solves it on the GPU.
    Returns (value, per-input-arc flow int64 or None, cut bool[n] or None, csr, stats)."""
    csr = build_csr(inst.n, inst.tail, inst.head, inst.cap)
    with Graph.from_csr(csr, inst.s, inst.t, options) as g:
        r = g.solve(flow=flow, cut=cut)
        st = g.stats()
    fin = None
    if flow:
        fin = np.where(csr.arc_slot >= 0, r.flow[np.maximum(csr.arc_slot, 0)], 0).astype(np.int64)
    cut_b = cut_bits_to_bool(r.cut_bits, inst.n) if cut else None
    return r.value, fin, cut_b, csr, st


def _descs(csrs, sts):
    """GraphDesc array for (CSR, (s, t)) pairs; returns (array, keepalive)."""
    arr = (GraphDesc * len(csrs))()
    keep = []
    for k, (c, (s, t)) in enumerate(zip(csrs, sts)):
        row = np.ascontiguousarray(c.row_offsets, np.int64)
        head = np.ascontiguousarray(c.head, np.int32)
        cap = np.ascontiguousarray(c.cap, np.int32)
        rev = np.ascontiguousarray(c.rev, np.int64)
        keep += [row, head, cap, rev]
        arr[k] = GraphDesc(c.n, c.m, row.ctypes.data, head.ctypes.data, cap.ctypes.data, rev.ctypes.data, s, t)
    return arr, keep


class Batch:
    """Many independent instances solved by one persistent launch (mf_batch_*)."""

    def __init__(self, csrs, sts, options: Options | None = None):
        self.csrs = list(csrs)
        self.sts = list(sts)
        arr, keep = _descs(self.csrs, self.sts)
        self._h = ctypes.c_void_p()
        _check(lib().mf_batch_create(len(self.csrs), arr, ctypes.byref(options) if options else None,
                                     ctypes.byref(self._h)))

    def solve(self, flow=True, cut=True):
        """Returns a list of Result (per-instance value, slot flows, cut bits)."""
        k = len(self.csrs)
        vals = np.zeros(k, np.int64)
        flows = [np.zeros(c.m, np.int32) for c in self.csrs] if flow else None
        cuts = [np.zeros((c.n + 31) // 32, np.uint32) for c in self.csrs] if cut else None
        fp = (ctypes.c_void_p * k)(*[f.ctypes.data for f in flows]) if flow else None
        cp = (ctypes.c_void_p * k)(*[c.ctypes.data for c in cuts]) if cut else None
        _check(lib().mf_batch_solve(self._h, _ptr(vals), fp, cp))
        return [Result(int(vals[i]), flows[i] if flow else None, cuts[i] if cut else None) for i in range(k)]

    def stats(self) -> dict:
        s = Stats()
        _check(lib().mf_batch_get_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def set_options(self, options: Options):
        _check(lib().mf_batch_set_options(self._h, ctypes.byref(options)))

    def autotune(self, reps: int = 3, sweeps: int = 1, time_budget_ms: float = 0.0):
        """mf_batch_autotune: as Graph.autotune, checking the values of every instance."""
        return _autotune(lib().mf_batch_autotune, self._h, reps, sweeps, time_budget_ms)

    def close(self):
        if self._h:
            lib().mf_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Service:
    """Continuous-batching solver service (mf_service_create / mf_submit / mf_poll / mf_wait)."""

    def __init__(self, budget_bytes: int, options: Options | None = None):
        self._h = ctypes.c_void_p()
        self._inst = {}
        _check(lib().mf_service_create(int(budget_bytes), ctypes.byref(options) if options else None,
                                       ctypes.byref(self._h)))

    def submit(self, csr: CSR, s: int, t: int) -> int:
        arr, keep = _descs([csr], [(s, t)])
        tk = ctypes.c_int64()
        _check(lib().mf_submit(self._h, arr, ctypes.byref(tk)))
        self._inst[int(tk.value)] = (csr.n, csr.m)
        return int(tk.value)

    def wait(self, ticket: int, timeout_ms: int = -1):
        """Latency in ms once the ticket is done, None on timeout."""
        lat = ctypes.c_double()
        rc = _check(lib().mf_wait(self._h, ticket, timeout_ms, ctypes.byref(lat)))
        return None if rc == MF_PENDING else lat.value

    def poll(self, ticket: int, flow=True, cut=True):
        """Result once ready (the ticket is then forgotten), None while pending."""
        known = ticket in self._inst
        n, m = self._inst.get(ticket, (0, 0))
        v = ctypes.c_int64()
        f = np.zeros(m, np.int32) if flow and known else None
        c = np.zeros((n + 31) // 32, np.uint32) if cut and known else None
        rc = _check(lib().mf_poll(self._h, ticket, ctypes.byref(v), _ptr(f), _ptr(c)))
        if rc == MF_PENDING:
            return None
        self._inst.pop(ticket, None)
        return Result(int(v.value), f, c)

    def close(self):
        if self._h:
            lib().mf_service_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
