"""Connected-components ORACLE (test infrastructure, not part of the product).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg (and
its ``--impl reference`` arm) may import this package. The library in
``paper_1612_01178_gb300`` never imports it and has no CPU fallback.

It computes the definition in Section II of the paper, with the representative
vertex fixed as the minimum vertex ID of the component:

    label[v] = min { w : w reachable from v in the undirected graph }

by two independent sequential algorithms in ``oracle.c`` (ascending-scan BFS
labelling and min-root union-find). The tests pin both against brute force on all
small graphs, closed forms, SciPy and invariants. Nothing here is shared with the
CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False, src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile oracle.c (plain C, -O2, no vectorisation tricks) into a shared library."""
    stale = force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src)
    if stale:
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", src, "-o", tmp])
        os.replace(tmp, out)
    return out


def _declare(lib):
    i64, i32p, i64p = ctypes.c_int64, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
    for name in ("oracle_uf_csr", "oracle_bfs_csr"):
        f = getattr(lib, name)
        f.argtypes = [i64, i64p, i32p, i32p]
        f.restype = i64
    for name in ("oracle_uf_coo", "oracle_bfs_coo"):
        f = getattr(lib, name)
        f.argtypes = [i64, i64, i32p, i32p, i32p]
        f.restype = i64
    lib.oracle_label_of.argtypes = [i64, i64p, i32p, i64, i32p, i32p]
    lib.oracle_label_of.restype = i64
    return lib


def load_library(path: str):
    """Load an oracle build (the tests also load deliberately broken copies of it)."""
    return _declare(ctypes.CDLL(path))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
    return _lib


def _p32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _p64(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _csr_args(row_ptr, col):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    V = rp.shape[0] - 1
    if V < 0:
        raise ValueError("row_ptr must have V+1 entries")
    if int(rp[-1]) != cl.shape[0]:
        raise ValueError("row_ptr[V] must equal len(col)")
    return V, rp, cl


def _check(n: int, what: str) -> int:
    if n < 0:
        raise ValueError(f"{what}: malformed graph (endpoint outside [0, V) or bad offsets)")
    return int(n)


def labels_uf_csr(row_ptr, col, lib=None):
    """Min-ID component labels of a CSR graph by union-find. Returns (labels, n_components)."""
    lib = lib or _load()
    V, rp, cl = _csr_args(row_ptr, col)
    out = np.empty(V, np.int32)
    n = lib.oracle_uf_csr(V, _p64(rp), _p32(cl), _p32(out))
    return out, _check(n, "oracle_uf_csr")


def labels_bfs_csr(row_ptr, col, lib=None):
    """Min-ID component labels of a CSR graph by ascending-scan BFS. Returns (labels, n_components)."""
    lib = lib or _load()
    V, rp, cl = _csr_args(row_ptr, col)
    out = np.empty(V, np.int32)
    n = lib.oracle_bfs_csr(V, _p64(rp), _p32(cl), _p32(out))
    return out, _check(n, "oracle_bfs_csr")


def _coo_args(n_vertices, src, dst):
    s = np.ascontiguousarray(src, dtype=np.int32)
    d = np.ascontiguousarray(dst, dtype=np.int32)
    if s.shape != d.shape:
        raise ValueError("src and dst differ in length")
    return int(n_vertices), s, d


def labels_uf_coo(n_vertices, src, dst, lib=None):
    lib = lib or _load()
    V, s, d = _coo_args(n_vertices, src, dst)
    out = np.empty(V, np.int32)
    n = lib.oracle_uf_coo(V, s.shape[0], _p32(s), _p32(d), _p32(out))
    return out, _check(n, "oracle_uf_coo")


def labels_bfs_coo(n_vertices, src, dst, lib=None):
    lib = lib or _load()
    V, s, d = _coo_args(n_vertices, src, dst)
    out = np.empty(V, np.int32)
    n = lib.oracle_bfs_coo(V, s.shape[0], _p32(s), _p32(d), _p32(out))
    return out, _check(n, "oracle_bfs_coo")


class SampledLabels:
    """Label of single vertices of a large symmetric CSR graph, one search at a time."""

    def __init__(self, row_ptr, col, lib=None):
        self._lib = lib or _load()
        self.V, self.rp, self.col = _csr_args(row_ptr, col)
        self._seen = np.full(max(self.V, 1), -1, np.int32)
        self._queue = np.empty(max(self.V, 1), np.int32)

    def label_of(self, v: int) -> int:
        r = self._lib.oracle_label_of(self.V, _p64(self.rp), _p32(self.col), int(v), _p32(self._seen),
                                      _p32(self._queue))
        return _check(r, "oracle_label_of")


def labels(row_ptr, col):
    """The oracle's answer for a CSR graph: union-find labels (BFS agreement is tested separately)."""
    return labels_uf_csr(row_ptr, col)[0]
