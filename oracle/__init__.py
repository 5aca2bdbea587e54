"""CPU oracle -- test infrastructure only.

Plain, sequential definitions of what the fixpoint relaxation sweep computes
(Sec. 2, Algorithms 1-3): Dijkstra for SSSP, FIFO-queue BFS, union-find CC
labelled by the minimum vertex id, the Jacobi Bellman-Ford round count of
the synchronous variant, and one double-buffered relaxation round from a given
state (the all-active sweep).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the CUDA library never
does, and the two share no code.

``oracle/omp.py`` (the multi-core OpenMP baseline that the benchmark reports
beside the oracle's timing) is not part of the oracle: nothing here uses it,
and its tests compare it with the functions below.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(Floyd-Warshall, brute-force path enumeration, scipy.sparse.csgraph, closed
forms and invariants).  Nothing is left unpinned.
"""
from __future__ import annotations

import ctypes
import fcntl
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

OK = 0
INVALID = 1
NEGATIVE_WEIGHT = 2
OVERFLOW = 3
NOMEM = 4
UNREACHED = 2**31 - 1


def build(force: bool = False, extra_flags=(), out: str | None = None) -> str:
    """Compile the oracle with gcc (sequential, -O2).  ``out`` names a variant build."""
    target = out or _LIB
    with open(target + ".lock", "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        fresh = os.path.exists(target) and os.path.getmtime(target) >= os.path.getmtime(_SRC)
        if fresh and not force and not extra_flags:
            return target
        tmp = target + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", *extra_flags, _SRC,
                        "-o", tmp], check=True, capture_output=True)
        os.replace(tmp, target)
    return target


def _bind(lib):
    i32p = ctypes.POINTER(ctypes.c_int32)
    lib.or_sssp.restype = ctypes.c_int
    lib.or_sssp.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, ctypes.c_int32, i32p]
    lib.or_bfs.restype = ctypes.c_int
    lib.or_bfs.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, ctypes.c_int32, i32p]
    lib.or_cc.restype = ctypes.c_int
    lib.or_cc.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p]
    lib.or_jacobi_rounds.restype = ctypes.c_int64
    lib.or_jacobi_rounds.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p,
                                     ctypes.c_int32, ctypes.c_int, ctypes.c_int64, i32p]
    lib.or_sweep.restype = ctypes.c_int
    lib.or_sweep.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, i32p, i32p,
                             ctypes.POINTER(ctypes.c_int64)]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build()))
    return _lib


def load_variant(path: str):
    """Load a separately built oracle library (used by the planted-mistake tests)."""
    return _bind(ctypes.CDLL(path))


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _arr(x):
    return None if x is None else np.ascontiguousarray(x, dtype=np.int32)


def sssp(n, src, dst, w, s, lib=None):
    """Shortest distances from s (Alg. 1/2 fixpoint).  Returns (status, dist int32[n])."""
    lib = lib or _load()
    src, dst, w = _arr(src), _arr(dst), _arr(w)
    dist = np.empty(n, np.int32)
    rc = lib.or_sssp(n, src.shape[0], _p(src), _p(dst), _p(w), s, _p(dist))
    return rc, dist


def bfs(n, src, dst, s, lib=None):
    """Hop levels from s (Alg. 3 fixpoint).  Returns (status, level int32[n])."""
    lib = lib or _load()
    src, dst = _arr(src), _arr(dst)
    level = np.empty(n, np.int32)
    rc = lib.or_bfs(n, src.shape[0], _p(src), _p(dst), s, _p(level))
    return rc, level


def cc(n, src, dst, lib=None):
    """Minimum-id component labels of the symmetrised graph.  Returns (status, label)."""
    lib = lib or _load()
    src, dst = _arr(src), _arr(dst)
    label = np.empty(n, np.int32)
    rc = lib.or_cc(n, src.shape[0], _p(src), _p(dst), _p(label))
    return rc, label


def jacobi_rounds(n, src, dst, w, s, unit=False, max_rounds=None, lib=None):
    """Round count of double-buffered Bellman-Ford (no-change round included) and its result."""
    lib = lib or _load()
    src, dst, w = _arr(src), _arr(dst), _arr(w)
    dist = np.empty(n, np.int32)
    cap = max_rounds if max_rounds is not None else n + 2
    r = lib.or_jacobi_rounds(n, src.shape[0], _p(src), _p(dst), _p(w), s, 1 if unit else 0,
                             cap, _p(dist))
    return int(r), dist


def sweep(n, src, dst, w, cur, nxt, lib=None):
    """One double-buffered relaxation round (Alg. 1/2 body once) from state
    (cur, nxt).  Returns (status, new next int32[n], lowered-vertex count)."""
    lib = lib or _load()
    src, dst, w, cur = _arr(src), _arr(dst), _arr(w), _arr(cur)
    out = np.array(nxt, dtype=np.int32, copy=True)
    low = ctypes.c_int64(0)
    rc = lib.or_sweep(n, src.shape[0], _p(src), _p(dst), _p(w), _p(cur), _p(out), ctypes.byref(low))
    return rc, out, low.value
