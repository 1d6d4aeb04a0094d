"""Seeded synthetic graph inputs (ER, 2D grid, R-MAT) and the symmetrising CSR builder.

Input synthesis only: nothing here computes connected components. The CUDA path's
tests and benchmarks and the CPU oracle's tests both take their graphs from this
module, so the two sides always see identical arrays.

The native part (``gen.c``) is compiled with the host C compiler on first use into
``libgen.so`` beside this file.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB_PATH = os.path.join(_HERE, "libgen.so")
_lock = threading.Lock()
_lib = None

DEFAULT_THREADS = max(1, min(64, os.cpu_count() or 1))


def build(force: bool = False) -> str:
    """Compile gen.c into libgen.so (host code only; same flags on x86-64 and aarch64)."""
    stale = force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=gnu11", "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i64, i32p, i64p = ctypes.c_int64, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
            u64, dbl, cint = ctypes.c_uint64, ctypes.c_double, ctypes.c_int
            lib.gen_er_coo.argtypes = [i64, i64, u64, i32p, i32p, cint]
            lib.gen_er_coo.restype = cint
            lib.gen_rmat_coo.argtypes = [cint, i64, dbl, dbl, dbl, u64, cint, i32p, i32p, cint]
            lib.gen_rmat_coo.restype = cint
            lib.gen_permutation.argtypes = [ctypes.c_uint32, u64, i32p]
            lib.gen_permutation.restype = cint
            lib.gen_grid_row_ptr.argtypes = [i64, dbl, u64, i64p, cint]
            lib.gen_grid_row_ptr.restype = i64
            lib.gen_grid_col.argtypes = [i64, dbl, u64, i64p, i32p, cint]
            lib.gen_grid_col.restype = cint
            lib.gen_sym_csr_row_ptr.argtypes = [i64, i64, i32p, i32p, i64p, cint]
            lib.gen_sym_csr_row_ptr.restype = i64
            lib.gen_sym_csr_col.argtypes = [i64, i64, i32p, i32p, i64p, i32p, i64p, cint]
            lib.gen_sym_csr_col.restype = cint
            _lib = lib
    return _lib


def _p32(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _p64(a: np.ndarray):
    assert a.dtype == np.int64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


class CSR:
    """Symmetric CSR graph: row_ptr[V+1] (int32 or int64), col[nnz] int32, rows sorted."""

    __slots__ = ("n_vertices", "row_ptr", "col", "n_edges", "name")

    def __init__(self, n_vertices: int, row_ptr: np.ndarray, col: np.ndarray, n_edges: int, name: str = ""):
        self.n_vertices = int(n_vertices)
        self.row_ptr = row_ptr
        self.col = col
        self.n_edges = int(n_edges)  # undirected input edges (nnz / 2)
        self.name = name

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def __repr__(self) -> str:
        return f"CSR({self.name or 'graph'}: V={self.n_vertices}, nnz={self.nnz}, off={self.row_ptr.dtype})"


def er_coo(n_vertices: int, n_edges: int, seed: int, threads: int = DEFAULT_THREADS):
    """E edges with both endpoints uniform over [0, V) (self-loops, duplicates kept)."""
    src = np.empty(n_edges, np.int32)
    dst = np.empty(n_edges, np.int32)
    rc = _load().gen_er_coo(n_vertices, n_edges, seed, _p32(src), _p32(dst), threads)
    if rc != 0:
        raise ValueError("gen_er_coo: bad arguments")
    return src, dst


def rmat_coo(scale: int, n_edges: int, seed: int, a=0.57, b=0.19, c=0.19, permute=True,
             threads: int = DEFAULT_THREADS):
    """R-MAT edge list on 2^scale vertices, IDs permuted by a keyed pseudo-random permutation."""
    src = np.empty(n_edges, np.int32)
    dst = np.empty(n_edges, np.int32)
    rc = _load().gen_rmat_coo(scale, n_edges, a, b, c, seed, int(permute), _p32(src), _p32(dst), threads)
    if rc != 0:
        raise ValueError("gen_rmat_coo: bad arguments")
    return src, dst


def permutation(n: int, seed: int) -> np.ndarray:
    """The vertex-ID permutation R-MAT applies (exposed for tests)."""
    out = np.empty(n, np.int32)
    _load().gen_permutation(n, seed, _p32(out))
    return out


def sym_csr_from_coo(n_vertices: int, src: np.ndarray, dst: np.ndarray, offsets64: bool = False,
                     threads: int = DEFAULT_THREADS, name: str = "") -> CSR:
    """Symmetrised CSR: each edge (u,v) gives arcs (u,v) and (v,u); nnz = 2E exactly."""
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    E = int(src.shape[0])
    assert dst.shape[0] == E
    lib = _load()
    row_ptr = np.empty(n_vertices + 1, np.int64)
    nnz = lib.gen_sym_csr_row_ptr(n_vertices, E, _p32(src), _p32(dst), _p64(row_ptr), threads)
    if nnz < 0:
        raise ValueError("edge endpoint outside [0, V)")
    col = np.empty(nnz, np.int32)
    scratch = np.empty(max(n_vertices, 1), np.int64)
    lib.gen_sym_csr_col(n_vertices, E, _p32(src), _p32(dst), _p64(row_ptr), _p32(col), _p64(scratch), threads)
    del scratch
    if not offsets64:
        if nnz > np.iinfo(np.int32).max:
            raise ValueError("nnz exceeds int32 row offsets; use offsets64=True")
        row_ptr = row_ptr.astype(np.int32)
    return CSR(n_vertices, row_ptr, col, E, name)


def grid_csr(side: int, p: float, seed: int, offsets64: bool = False, threads: int = DEFAULT_THREADS) -> CSR:
    """side x side 4-neighbour lattice, row-major IDs, each lattice edge kept with probability p."""
    lib = _load()
    V = side * side
    row_ptr = np.empty(V + 1, np.int64)
    nnz = lib.gen_grid_row_ptr(side, p, seed, _p64(row_ptr), threads)
    if nnz < 0:
        raise ValueError("bad grid arguments")
    col = np.empty(nnz, np.int32)
    lib.gen_grid_col(side, p, seed, _p64(row_ptr), _p32(col), threads)
    if not offsets64:
        row_ptr = row_ptr.astype(np.int32)
    return CSR(V, row_ptr, col, nnz // 2, f"grid{side}_p{p}")


def er_csr(n_vertices: int, n_edges: int, seed: int, offsets64: bool = False,
           threads: int = DEFAULT_THREADS) -> CSR:
    src, dst = er_coo(n_vertices, n_edges, seed, threads)
    return sym_csr_from_coo(n_vertices, src, dst, offsets64, threads, f"er{n_vertices}_{n_edges}")


def rmat_csr(scale: int, edge_factor: int, seed: int, a=0.57, b=0.19, c=0.19, offsets64: bool = False,
             threads: int = DEFAULT_THREADS) -> CSR:
    """R-MAT with E = edge_factor * 2^scale drawn edges, symmetrised (nnz = 2E)."""
    V = 1 << scale
    E = edge_factor * V
    src, dst = rmat_coo(scale, E, seed, a, b, c, True, threads)
    g = sym_csr_from_coo(V, src, dst, offsets64, threads, f"rmat{scale}_ef{edge_factor}")
    return g


# ----------------------------------------------------------------------------------------------
# Named workloads (sizes of the five evaluation configurations).

ER_100K = dict(n_vertices=100_000, n_edges=1_000_000)
GRID_4096 = dict(side=4096, p=0.9)
RMAT_26 = dict(scale=26, edge_factor=16)


def workload_er_100k(seed: int = 1) -> CSR:
    """Erdos-Renyi, V=100,000, 1,000,000 drawn edges, int32 CSR (nnz = 2,000,000)."""
    return er_csr(seed=seed, **ER_100K)


def workload_grid_4096(seed: int = 1) -> CSR:
    """Road-like 4096 x 4096 grid, p = 0.9, int32 CSR."""
    return grid_csr(seed=seed, **GRID_4096)


def workload_rmat_26(seed: int = 1) -> CSR:
    """R-MAT scale 26, edge factor 16 (2^30 drawn edges, nnz = 2^31), int64 row offsets."""
    return rmat_csr(seed=seed, offsets64=True, **RMAT_26)


def loguniform_int(rng: np.random.Generator, lo: float, hi: float) -> int:
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


# ----------------------------------------------------------------------------------------------
# Batches of independent graphs over a graph-offset table.

class Batch:
    """Concatenated CSR of independent graphs.

    Graph g owns vertices [v_off[g], v_off[g+1]) of the concatenated label array, arcs
    [a_off[g], a_off[g+1]) of col_cat (graph-local IDs), and its V_g + 1 graph-local row offsets
    start at row_ptr_cat[v_off[g] + g]."""

    __slots__ = ("v_off", "a_off", "row_ptr_cat", "col_cat", "kinds")

    def __init__(self, v_off, a_off, row_ptr_cat, col_cat, kinds):
        self.v_off, self.a_off, self.row_ptr_cat, self.col_cat, self.kinds = v_off, a_off, row_ptr_cat, col_cat, kinds

    @property
    def n_graphs(self) -> int:
        return int(self.v_off.shape[0] - 1)

    @property
    def total_vertices(self) -> int:
        return int(self.v_off[-1])

    @property
    def total_arcs(self) -> int:
        return int(self.a_off[-1])

    def graph(self, g: int):
        """(row_ptr, col) views of graph g (graph-local IDs)."""
        v0, v1 = int(self.v_off[g]), int(self.v_off[g + 1])
        a0, a1 = int(self.a_off[g]), int(self.a_off[g + 1])
        return self.row_ptr_cat[v0 + g: v1 + g + 1], self.col_cat[a0:a1]

    def __repr__(self):
        return f"Batch(n={self.n_graphs}, V={self.total_vertices}, arcs={self.total_arcs})"


def batch_from_graphs(graphs, kinds=None) -> Batch:
    """Concatenate CSR graphs (int32 row offsets) into a Batch."""
    n = len(graphs)
    v_off = np.zeros(n + 1, np.int64)
    a_off = np.zeros(n + 1, np.int64)
    for g, h in enumerate(graphs):
        v_off[g + 1] = v_off[g] + h.n_vertices
        a_off[g + 1] = a_off[g] + h.nnz
    row_ptr_cat = np.empty(int(v_off[-1]) + n, np.int32)
    col_cat = np.empty(int(a_off[-1]), np.int32)
    for g, h in enumerate(graphs):
        v0 = int(v_off[g]) + g
        row_ptr_cat[v0: v0 + h.n_vertices + 1] = h.row_ptr
        col_cat[int(a_off[g]): int(a_off[g + 1])] = h.col
    return Batch(v_off, a_off, row_ptr_cat, col_cat, kinds or [h.name for h in graphs])


def mixed_spec(kind: str, v_target: int, seed: int, rng: np.random.Generator) -> dict:
    """Parameters of one graph of the batched/served mixes, sized for about v_target vertices:
    'er'   Erdos-Renyi, average degree d ~ U{4..32} (E = d V / 2 drawn edges);
    'grid' square 2D grid, side round(sqrt(V)), p = 0.9;
    'rmat' R-MAT, scale round(log2 V), edge factor 8."""
    if kind == "er":
        d = int(rng.integers(4, 33))
        V = max(1, v_target)
        return dict(kind="er", n_vertices=V, n_edges=d * V // 2, seed=seed)
    if kind == "grid":
        return dict(kind="grid", side=max(1, int(round(math.sqrt(v_target)))), p=0.9, seed=seed)
    if kind == "rmat":
        return dict(kind="rmat", scale=max(1, int(round(math.log2(max(2, v_target))))), edge_factor=8, seed=seed)
    raise ValueError(kind)


def make_graph(spec: dict) -> CSR:
    if spec["kind"] == "er":
        return er_csr(spec["n_vertices"], spec["n_edges"], spec["seed"])
    if spec["kind"] == "grid":
        return grid_csr(spec["side"], spec["p"], spec["seed"])
    return rmat_csr(spec["scale"], spec["edge_factor"], spec["seed"])


def batched_specs(n_graphs: int = 4096, seed: int = 1, vmin: float = 1e3, vmax: float = 1e6,
                  kinds=("er", "grid", "rmat")) -> list:
    """Specs of the batched workload: |V| log-uniform in [vmin, vmax], family drawn uniformly per
    graph from `kinds`; graph g is generated with seed 1000 + g."""
    rng = np.random.default_rng(seed)
    specs = []
    for g in range(n_graphs):
        kind = kinds[int(rng.integers(0, len(kinds)))]
        v_target = loguniform_int(rng, vmin, vmax)
        specs.append(mixed_spec(kind, v_target, 1000 + g, rng))
    return specs


def workload_batched(n_graphs: int = 4096, seed: int = 1, vmin: float = 1e3, vmax: float = 1e6,
                     kinds=("er", "grid", "rmat")) -> Batch:
    """The batched workload as one Batch (see batched_specs)."""
    specs = batched_specs(n_graphs, seed, vmin, vmax, kinds)
    return batch_from_graphs([make_graph(s) for s in specs], [s["kind"] for s in specs])
