"""Multi-core CPU baseline -- test infrastructure only; not the oracle.

A frontier Bellman-Ford SSSP, a level-synchronous BFS and a lock-free
union-find CC on all host cores (OpenMP), the kind of multi-core code the
paper generates from the same programs for its CPU comparison (Sec. 4).  It
gives the benchmark's CPU-baseline leg a multi-core figure beside the
sequential oracle's.  Results follow the oracle's readings and status codes;
``tests/test_omp_baseline.py`` checks them against the oracle.  Only the
tests and the benchmark's CPU-baseline leg load it.

``build()`` returns None where the host compiler has no OpenMP: the baseline
is then reported as unavailable, and nothing else depends on it.
"""
from __future__ import annotations

import ctypes
import fcntl
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "omp_frontier.c")
_LIB = os.path.join(_HERE, "libomp_frontier.so")
_lib = None

OK = 0
INVALID = 1
NEGATIVE_WEIGHT = 2
OVERFLOW = 3
NOMEM = 4


def build(force: bool = False) -> str | None:
    """Compile the baseline with gcc -O3 -fopenmp; None if that fails."""
    with open(_LIB + ".lock", "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        if os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC) and not force:
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        r = subprocess.run(["gcc", "-O3", "-std=c11", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp],
                           capture_output=True)
        if r.returncode != 0:
            return None
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        path = build()
        if path is None:
            raise RuntimeError("the OpenMP baseline did not build (no OpenMP in the host compiler)")
        lib = ctypes.CDLL(path)
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.ofr_sssp.restype = ctypes.c_int
        lib.ofr_sssp.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, ctypes.c_int32, i32p]
        lib.ofr_bfs.restype = ctypes.c_int
        lib.ofr_bfs.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, ctypes.c_int32, i32p]
        lib.ofr_cc.restype = ctypes.c_int
        lib.ofr_cc.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p]
        lib.ofr_graph_build.restype = ctypes.c_int
        lib.ofr_graph_build.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p,
                                        ctypes.POINTER(ctypes.c_void_p)]
        lib.ofr_graph_free.restype = None
        lib.ofr_graph_free.argtypes = [ctypes.c_void_p]
        lib.ofr_graph_sssp.restype = ctypes.c_int
        lib.ofr_graph_sssp.argtypes = [ctypes.c_void_p, ctypes.c_int32, i32p]
        lib.ofr_graph_bfs.restype = ctypes.c_int
        lib.ofr_graph_bfs.argtypes = [ctypes.c_void_p, ctypes.c_int32, i32p]
        lib.ofr_threads.restype = ctypes.c_int
        lib.ofr_threads.argtypes = []
        lib.ofr_set_threads.restype = None
        lib.ofr_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _arr(x):
    return None if x is None else np.ascontiguousarray(x, dtype=np.int32)


def threads() -> int:
    """Threads each parallel region uses (OMP_NUM_THREADS, else the host's cores)."""
    return int(_load().ofr_threads())


def set_threads(t: int) -> None:
    _load().ofr_set_threads(int(t))


def sssp(n, src, dst, w, s):
    """Shortest distances from s.  Returns (status, dist int32[n])."""
    src, dst, w = _arr(src), _arr(dst), _arr(w)
    dist = np.empty(n, np.int32)
    rc = _load().ofr_sssp(n, src.shape[0], _p(src), _p(dst), _p(w), s, _p(dist))
    return rc, dist


def bfs(n, src, dst, s):
    """Hop levels from s.  Returns (status, level int32[n])."""
    src, dst = _arr(src), _arr(dst)
    level = np.empty(n, np.int32)
    rc = _load().ofr_bfs(n, src.shape[0], _p(src), _p(dst), s, _p(level))
    return rc, level


def cc(n, src, dst):
    """Minimum-id labels of the weakly connected components.  Returns (status, label)."""
    src, dst = _arr(src), _arr(dst)
    label = np.empty(n, np.int32)
    rc = _load().ofr_cc(n, src.shape[0], _p(src), _p(dst), _p(label))
    return rc, label


class Graph:
    """An adjacency built once (on all threads) for many SSSP and BFS queries."""

    def __init__(self, n, src, dst, w=None):
        src, dst, w = _arr(src), _arr(dst), _arr(w)
        self.n = n
        self._h = ctypes.c_void_p()
        self.status = _load().ofr_graph_build(n, src.shape[0], _p(src), _p(dst), _p(w), ctypes.byref(self._h))

    def sssp(self, s):
        dist = np.empty(self.n, np.int32)
        return _load().ofr_graph_sssp(self._h, s, _p(dist)), dist

    def bfs(self, s):
        level = np.empty(self.n, np.int32)
        return _load().ofr_graph_bfs(self._h, s, _p(level)), level

    def close(self):
        if self._h:
            _load().ofr_graph_free(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
