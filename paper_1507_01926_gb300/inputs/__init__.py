"""Seeded synthetic max-flow instances shared by the solver's tests, the bench and the oracle.

This module holds only structure and random numbers (see ``gen.c``): vertex numbering, arc lists and
capacities of the workload families. It contains none of the max-flow arithmetic.

Workload recipes (seed = 150701926 + k with k = 0..4 in the order below; instance i of a batch or stream
uses seed * 2**20 + i):

* ``grid2d_64x64``: 64x64 4-connected grid, neighbour capacity U[1,100] per direction, every pixel gets s->p
  (probability 1/2) or p->t with capacity U[1,1000].
* ``grid3d_256x256x128``: 256x256x128 6-connected grid, capacity U[1,1000] per direction, s -> face z=0 and
  face z=127 -> t at 10^6.
* ``rmat_s22_ef16``: R-MAT scale 22, edge factor 16, (a,b,c,d) = (.57,.19,.19,.05), self-loops and
  duplicates dropped, capacity U[1,1000]; s = max out-degree, t = max in-degree among the rest.
* ``layered_batch_params`` / ``layered_batch_instance``: 2048 layered graphs, L ~ logU[16,256], W ~ logU[64,4096], 4 next-layer arcs + 1
  in-layer arc per vertex, capacity U[1,10000], terminals at 10^6.
* ``serving_stream_requests`` / ``serving_stream_instance``: a stream of requests, half 2D grids
  (side ~ logU[32,1024], terminals as in grid2d_64x64), half
  multi-frame grids (F ~ U[4,64] frames of 128x128, in-frame U[1,1000], frame-to-frame permutation
  arcs U[1,100], terminals as in grid2d_64x64), Poisson arrivals.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libmfgen.so")

BASE_SEED = 150701926


def build_lib(force: bool = False) -> str:
    """Compile gen.c into libmfgen.so next to it (gcc, no architecture-specific flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-fopenmp", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Arcs(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32),
        ("s", ctypes.c_int32),
        ("t", ctypes.c_int32),
        ("m", ctypes.c_int64),
        ("tail", ctypes.POINTER(ctypes.c_int32)),
        ("head", ctypes.POINTER(ctypes.c_int32)),
        ("cap", ctypes.POINTER(ctypes.c_int32)),
    ]


_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_lib())
        P = ctypes.POINTER(_Arcs)
        i32, i64, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        lib.mfg_grid2d.argtypes = [i32, i32, u64, i32, i32, i32, i32, P]
        lib.mfg_grid3d.argtypes = [i32, i32, i32, u64, i32, i32, i32, P]
        lib.mfg_rmat.argtypes = [i32, i32, u64, i32, i32, i32, i32, i32, P]
        lib.mfg_layered.argtypes = [i32, i32, u64, i32, i32, i32, P]
        lib.mfg_multiframe.argtypes = [i32, i32, u64, i32, i32, i32, i32, i32, i32, P]
        lib.mfg_random.argtypes = [i32, i64, u64, i32, i32, i32, P]
        for f in ("mfg_grid2d", "mfg_grid3d", "mfg_rmat", "mfg_layered", "mfg_multiframe", "mfg_random"):
            getattr(lib, f).restype = ctypes.c_int
        lib.mfg_free.argtypes = [P]
        lib.mfg_draw.argtypes = [u64, u64, u64]
        lib.mfg_draw.restype = u64
        lib.mfg_unif.argtypes = [u64, u64, u64, i64, i64]
        lib.mfg_unif.restype = i64
        lib.mfg_logunif.argtypes = [u64, u64, u64, i64, i64]
        lib.mfg_logunif.restype = i64
        lib.mfg_u01.argtypes = [u64, u64, u64]
        lib.mfg_u01.restype = ctypes.c_double
        _lib = lib
    return _lib


@dataclass
class Instance:
    """A max-flow instance as a directed input arc list (tail, head, cap) over vertices 0..n-1."""

    n: int
    s: int
    t: int
    tail: np.ndarray
    head: np.ndarray
    cap: np.ndarray
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.tail.shape[0])


def _take(fn, *args, name=""):
    a = _Arcs()
    rc = fn(*args, ctypes.byref(a))
    if rc != 0:
        raise ValueError(f"generator {fn.__name__} failed with code {rc} for args {args}")
    try:
        m = int(a.m)

        def grab(p):
            if m == 0:
                return np.zeros(0, np.int32)
            return np.ctypeslib.as_array(p, shape=(m,)).copy()

        return Instance(int(a.n), int(a.s), int(a.t), grab(a.tail), grab(a.head), grab(a.cap), name)
    finally:
        _L().mfg_free(ctypes.byref(a))


def grid2d(h, w, seed, nbr=(1, 100), term=(1, 1000)) -> Instance:
    return _take(_L().mfg_grid2d, h, w, seed, nbr[0], nbr[1], term[0], term[1], name=f"grid2d_{h}x{w}")


def grid3d(x, y, z, seed, cap=(1, 1000), term_cap=1_000_000) -> Instance:
    return _take(_L().mfg_grid3d, x, y, z, seed, cap[0], cap[1], term_cap, name=f"grid3d_{x}x{y}x{z}")


def rmat(scale, edge_factor, seed, abc=(57, 19, 19), cap=(1, 1000)) -> Instance:
    return _take(_L().mfg_rmat, scale, edge_factor, seed, abc[0], abc[1], abc[2], cap[0], cap[1],
                 name=f"rmat_s{scale}_ef{edge_factor}")


def layered(L, W, seed, cap=(1, 10000), term_cap=1_000_000) -> Instance:
    return _take(_L().mfg_layered, L, W, seed, cap[0], cap[1], term_cap, name=f"layered_{L}x{W}")


def multiframe(F, seed, side=128, nbr=(1, 1000), frame=(1, 100), term=(1, 1000)) -> Instance:
    return _take(_L().mfg_multiframe, F, side, seed, nbr[0], nbr[1], frame[0], frame[1], term[0], term[1],
                 name=f"multiframe_{F}x{side}x{side}")


def random_graph(n, m, seed, cap=(1, 100), allow_loops=False) -> Instance:
    return _take(_L().mfg_random, n, m, seed, cap[0], cap[1], 1 if allow_loops else 0, name=f"random_{n}_{m}")


def draw_unif(seed, stream, i, a, b) -> int:
    return int(_L().mfg_unif(seed, stream, i, a, b))


def draw_logunif(seed, stream, i, a, b) -> int:
    return int(_L().mfg_logunif(seed, stream, i, a, b))


def draw_u01(seed, stream, i) -> float:
    return float(_L().mfg_u01(seed, stream, i))


# ---------------------------------------------------------------- standing workloads

def grid2d_64x64() -> Instance:
    """64x64 2D grid (4,098 vertices)."""
    g = grid2d(64, 64, BASE_SEED + 0)
    g.name = "grid2d_64x64"
    return g


def grid3d_256x256x128() -> Instance:
    """256x256x128 3D grid (8,388,610 vertices)."""
    g = grid3d(256, 256, 128, BASE_SEED + 1)
    g.name = "grid3d_256x256x128"
    return g


def rmat_s22_ef16() -> Instance:
    """R-MAT scale 22, edge factor 16."""
    g = rmat(22, 16, BASE_SEED + 2)
    g.name = "rmat_s22_ef16"
    return g


def layered_batch_params(count: int = 2048):
    """(L, W) of each layered instance of the batch, from the batch seed."""
    seed = BASE_SEED + 3
    return [(draw_logunif(seed, 1, 2 * i, 16, 256), draw_logunif(seed, 1, 2 * i + 1, 64, 4096))
            for i in range(count)]


def layered_batch_instance(i: int, L: int, W: int) -> Instance:
    g = layered(L, W, (BASE_SEED + 3) * (1 << 20) + i)
    g.name = f"layered_{i}_{L}x{W}"
    return g


def serving_stream_requests(count: int = 20000, rate_per_s: float = 1.0):
    """Request descriptors of the serving stream: (arrival_s, kind, size) with kind 'grid' (size = side)
    or 'frames' (size = F). Inter-arrival times are exponential with the given rate."""
    seed = BASE_SEED + 4
    out = []
    tnow = 0.0
    for i in range(count):
        u = draw_u01(seed, 1, i)
        tnow += -np.log1p(-u) / rate_per_s
        if _L().mfg_draw(seed, 2, i) >> 63:
            out.append((tnow, "frames", draw_unif(seed, 3, i, 4, 64)))
        else:
            out.append((tnow, "grid", draw_logunif(seed, 3, i, 32, 1024)))
    return out


def serving_stream_instance(i: int, kind: str, size: int) -> Instance:
    seed = (BASE_SEED + 4) * (1 << 20) + i
    if kind == "grid":
        return grid2d(size, size, seed)
    return multiframe(size, seed)
