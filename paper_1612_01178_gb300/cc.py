"""Python binding of libcc.so (include/cc.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; this module only turns
torch CUDA tensors into device pointers and sizes. There is no CPU fallback: if the
library is missing or no GPU is present, the calls raise.

The function names follow the C ABI: ``cc_create``, ``cc_labels_csr``,
``cc_labels_coo``, ``cc_labels_csr_host``, ``cc_labels_batched``, ``cc_sync``,
``cc_destroy``. ``ConnectedComponents`` wraps a context for convenient use.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

# status codes (cc_status)
CC_OK = 0
CC_ERR_INVALID_ARG = 1
CC_ERR_OUT_OF_RANGE = 2
CC_ERR_OOM = 3
CC_ERR_CUDA = 4
CC_ERR_TIMEOUT = 5
CC_ERR_INTERNAL = 6

# flags
CC_FLAG_SYMMETRIC = 1
CC_FLAG_VALIDATE = 2
CC_FLAG_SYNC = 4
CC_FLAG_PHASE_TIMES = 8

# modes
CC_MODE_AUTO = 0
CC_MODE_PERSISTENT = 1
CC_MODE_MULTI_LAUNCH = 2
CC_MODE_SOMAN = 3
CC_MODE_SOMAN_MULTIJUMP = 4
CC_MODE_FILTERED = 5
CC_MODE_CLUSTER = 6

CC_INDEX_I32 = 4
CC_INDEX_I64 = 8


class cc_options(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_int32),
        ("segments", ctypes.c_int32),
        ("block", ctypes.c_int32),
        ("grid_blocks", ctypes.c_int32),
        ("flags", ctypes.c_int32),
        ("chunk_arcs", ctypes.c_int32),
        ("tile_vertices", ctypes.c_int32),
        ("sm_limit", ctypes.c_int32),
        ("timeout_ns", ctypes.c_int64),
        ("stream_arcs", ctypes.c_int64),
        ("hook_k", ctypes.c_int32),
        ("auto_min_vertices", ctypes.c_int32),
        ("auto_local_permille", ctypes.c_int32),
        ("auto_lowdeg_permille", ctypes.c_int32),
        ("cluster_max_vertices", ctypes.c_int32),
        ("auto_dense_degree", ctypes.c_int32),
    ]


class cc_run_info(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_int32),
        ("segments", ctypes.c_int32),
        ("grid_blocks", ctypes.c_int32),
        ("block", ctypes.c_int32),
        ("launches", ctypes.c_int32),
        ("tile_vertices", ctypes.c_int32),
        ("worklist_capacity", ctypes.c_int64),
        ("host_round_trips", ctypes.c_int32),
        ("hook_rounds", ctypes.c_int32),
        ("streamed_segments", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


class CCError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = f"{where}: {status_string(status)}"
        if detail:
            msg += f" ({detail})"
        super().__init__(msg)


_lib = None
_lib_lock = threading.Lock()

# Every exported symbol with its ctypes signature (restype, argtypes).
_vp, _i32, _i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
SIGNATURES = {
    "cc_default_options": (None, [ctypes.POINTER(cc_options)]),
    "cc_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _vp, ctypes.POINTER(cc_options)]),
    "cc_set_stream": (ctypes.c_int, [_vp, _vp]),
    "cc_set_options": (ctypes.c_int, [_vp, ctypes.POINTER(cc_options)]),
    "cc_set_launch_status": (ctypes.c_int, [_vp, _vp]),
    "cc_labels_csr": (ctypes.c_int, [_vp, _i64, _i64, _vp, ctypes.c_int, _vp, _vp]),
    "cc_labels_coo": (ctypes.c_int, [_vp, _i64, _i64, _vp, _vp, _vp]),
    "cc_labels_csr64": (ctypes.c_int, [_vp, _i64, _i64, _vp, _vp, _vp]),
    "cc_labels_csr_host": (ctypes.c_int, [_vp, _i64, _i64, _vp, ctypes.c_int, _vp, _vp]),
    "cc_labels_batched": (ctypes.c_int, [_vp, _i32, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp]),
    "cc_labels_batched_desc": (ctypes.c_int, [_vp, _i32, _vp, _vp, _i64, _vp, _i64, _vp, _i64, _vp]),
    "cc_sync": (ctypes.c_int, [_vp]),
    "cc_last_run_info": (ctypes.c_int, [_vp, ctypes.POINTER(cc_run_info)]),
    "cc_last_error_message": (ctypes.c_char_p, [_vp]),
    "cc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "cc_destroy": (None, [_vp]),
    "cc_debug_skip_barrier_arrival": (ctypes.c_int, [_vp, _i32]),
    "cc_labels_csr_noalloc": (ctypes.c_int, [_i64, _i64, _vp, ctypes.c_int, _vp, _vp, _vp, _i32]),
    "cc_last_phase_times": (ctypes.c_int, [_vp, ctypes.POINTER(_i64), _i32, ctypes.POINTER(_i32)]),
    "cc_last_worklist": (ctypes.c_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i32)]),
}


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Load libcc.so (building it first if it is missing or stale and nvcc is present)."""
    global _lib
    with _lib_lock:
        if _lib is None:
            path = _build.LIB_PATH
            if build_if_missing and (not os.path.exists(path) or _build.is_stale()):
                _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"libcc.so not found at {path}; run paper_1612_01178_gb300.build.build()")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def status_string(status: int) -> str:
    try:
        return load().cc_status_string(int(status)).decode()
    except Exception:  # the library itself failed to load
        return f"status {status}"


def _check(status: int, where: str, ctx=None):
    if status != CC_OK:
        detail = ""
        if ctx is not None:
            detail = load().cc_last_error_message(ctx).decode()
        raise CCError(status, where, detail)


def default_options(**kw) -> cc_options:
    o = cc_options()
    load().cc_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, int(v))
    return o


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


def cc_create(device: int = 0, stream=None, options: cc_options | None = None):
    """Create a context on `device` issuing work on `stream` (a torch.cuda.Stream or handle)."""
    lib = load()
    h = ctypes.c_void_p()
    opt = options if options is not None else default_options()
    st = lib.cc_create(ctypes.byref(h), int(device), ctypes.c_void_p(_stream_handle(stream)), ctypes.byref(opt))
    _check(st, "cc_create")
    return h


def cc_destroy(ctx) -> None:
    if ctx:
        load().cc_destroy(ctx)


def cc_set_options(ctx, options: cc_options) -> None:
    _check(load().cc_set_options(ctx, ctypes.byref(options)), "cc_set_options", ctx)


def cc_set_stream(ctx, stream) -> None:
    _check(load().cc_set_stream(ctx, ctypes.c_void_p(_stream_handle(stream))), "cc_set_stream", ctx)


def cc_sync(ctx, raise_input_errors: bool = True) -> int:
    """Wait for the context's stream; raise on a pending device error. With
    raise_input_errors=False a malformed-input report (CC_ERR_OUT_OF_RANGE) is returned instead
    of raised (a caller that reads per-graph or per-call statuses); fatal errors still raise."""
    st = load().cc_sync(ctx)
    if st == CC_ERR_OUT_OF_RANGE and not raise_input_errors:
        return st
    _check(st, "cc_sync", ctx)
    return st


def cc_set_launch_status(ctx, device_status=None) -> None:
    """Per-call input status output: a one-element int32 CUDA tensor (or a device pointer), or
    None to turn it off. Each following call zeroes it and its kernels set CC_ERR_OUT_OF_RANGE
    on malformed input."""
    ptr = None
    if device_status is not None:
        ptr = device_status.data_ptr() if hasattr(device_status, "data_ptr") else int(device_status)
    _check(load().cc_set_launch_status(ctx, ptr), "cc_set_launch_status", ctx)


def cc_last_run_info(ctx) -> dict:
    info = cc_run_info()
    _check(load().cc_last_run_info(ctx, ctypes.byref(info)), "cc_last_run_info")
    return {k: getattr(info, k) for k, _ in cc_run_info._fields_}


def cc_last_phase_times(ctx) -> list:
    """Relative device timestamps (ns) of the last persistent launch made with CC_FLAG_PHASE_TIMES."""
    buf = (_i64 * 64)()
    n = _i32()
    _check(load().cc_last_phase_times(ctx, buf, 64, ctypes.byref(n)), "cc_last_phase_times", ctx)
    return [int(buf[i]) for i in range(n.value)]


def cc_last_worklist(ctx) -> tuple:
    """(pairs left for the global phase, segments it used) of the last hierarchical-hook launch."""
    pairs, segs = _i64(), _i32()
    _check(load().cc_last_worklist(ctx, ctypes.byref(pairs), ctypes.byref(segs)), "cc_last_worklist", ctx)
    return pairs.value, segs.value


def _dev_tensor(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def cc_labels_csr(ctx, row_ptr, col_idx, labels=None):
    """Min-ID component labels of a CSR graph held in CUDA tensors (int32/int64 row_ptr, int32 col_idx).

    Returns the int32 labels tensor (allocated with torch if not given). Asynchronous on the
    context's stream unless the context has CC_FLAG_SYNC."""
    import torch
    if row_ptr.dtype not in (torch.int32, torch.int64):
        raise TypeError("row_ptr must be int32 or int64")
    _dev_tensor(row_ptr, row_ptr.dtype, "row_ptr")
    _dev_tensor(col_idx, torch.int32, "col_idx")
    V = row_ptr.numel() - 1
    if V < 0:
        raise ValueError("row_ptr must hold V+1 offsets")
    if labels is None:
        labels = torch.empty(V, dtype=torch.int32, device=row_ptr.device)
    _dev_tensor(labels, torch.int32, "labels")
    if labels.numel() != V:
        raise ValueError("labels must hold V entries")
    itype = CC_INDEX_I64 if row_ptr.dtype == torch.int64 else CC_INDEX_I32
    st = load().cc_labels_csr(ctx, V, col_idx.numel(), row_ptr.data_ptr(), itype,
                              col_idx.data_ptr() if col_idx.numel() else None,
                              labels.data_ptr() if V else None)
    _check(st, "cc_labels_csr", ctx)
    return labels


def cc_labels_csr64(ctx, row_ptr, col_idx, labels=None):
    """Min-ID labels of a CSR graph with 64-bit vertex IDs (int64 CUDA tensors row_ptr, col_idx;
    int64 labels), for graphs of more than 2^31 - 1 vertices."""
    import torch
    _dev_tensor(row_ptr, torch.int64, "row_ptr")
    _dev_tensor(col_idx, torch.int64, "col_idx")
    V = row_ptr.numel() - 1
    if V < 0:
        raise ValueError("row_ptr must hold V+1 offsets")
    if labels is None:
        labels = torch.empty(V, dtype=torch.int64, device=row_ptr.device)
    _dev_tensor(labels, torch.int64, "labels")
    if labels.numel() != V:
        raise ValueError("labels must hold V entries")
    st = load().cc_labels_csr64(ctx, V, col_idx.numel(), row_ptr.data_ptr(),
                                col_idx.data_ptr() if col_idx.numel() else None, labels.data_ptr() if V else None)
    _check(st, "cc_labels_csr64", ctx)
    return labels


def cc_labels_coo(ctx, n_vertices: int, src, dst, labels=None):
    """Min-ID component labels of an undirected edge list (int32 CUDA tensors src, dst)."""
    import torch
    _dev_tensor(src, torch.int32, "src")
    _dev_tensor(dst, torch.int32, "dst")
    if src.numel() != dst.numel():
        raise ValueError("src and dst differ in length")
    if labels is None:
        labels = torch.empty(n_vertices, dtype=torch.int32, device=src.device)
    _dev_tensor(labels, torch.int32, "labels")
    if labels.numel() != n_vertices:
        raise ValueError("labels must hold n_vertices entries")
    st = load().cc_labels_coo(ctx, int(n_vertices), src.numel(), src.data_ptr() if src.numel() else None,
                              dst.data_ptr() if dst.numel() else None, labels.data_ptr() if n_vertices else None)
    _check(st, "cc_labels_coo", ctx)
    return labels


def cc_labels_batched(ctx, v_off, a_off, row_ptr_cat, col_idx_cat, labels=None, graph_status=None):
    """Labels of a batch of graphs given as CUDA tensors: int64 offset tables v_off/a_off
    [n_graphs+1], per-graph int32 row offsets concatenated (graph g's at v_off[g] + g), int32
    col_idx concatenated. Returns the int32 labels tensor (graph-local minimum IDs)."""
    import torch
    _dev_tensor(v_off, torch.int64, "v_off")
    _dev_tensor(a_off, torch.int64, "a_off")
    _dev_tensor(row_ptr_cat, torch.int32, "row_ptr_cat")
    _dev_tensor(col_idx_cat, torch.int32, "col_idx_cat")
    n = v_off.numel() - 1
    if n < 0 or a_off.numel() != n + 1:
        raise ValueError("v_off and a_off must both hold n_graphs + 1 offsets")
    total_v = row_ptr_cat.numel() - n
    if labels is None:
        labels = torch.empty(max(total_v, 0), dtype=torch.int32, device=v_off.device)
    _dev_tensor(labels, torch.int32, "labels")
    if labels.numel() != total_v:
        raise ValueError("labels must hold total_vertices entries (row_ptr_cat has total_vertices + n_graphs)")
    if graph_status is not None:
        _dev_tensor(graph_status, torch.int32, "graph_status")
        if graph_status.numel() != n:
            raise ValueError("graph_status must hold n_graphs entries")
    st = load().cc_labels_batched(ctx, n, total_v, col_idx_cat.numel(), v_off.data_ptr(), a_off.data_ptr(),
                                  row_ptr_cat.data_ptr(), col_idx_cat.data_ptr() if col_idx_cat.numel() else None,
                                  labels.data_ptr() if total_v else None,
                                  graph_status.data_ptr() if graph_status is not None else None)
    _check(st, "cc_labels_batched", ctx)
    return labels


def cc_labels_csr_host(ctx, row_ptr: np.ndarray, col_idx: np.ndarray, labels: np.ndarray | None = None):
    """cc_labels_csr on host (numpy) arrays; synchronous. Pinned arrays copy fastest."""
    rp = row_ptr
    if rp.dtype not in (np.int32, np.int64) or not rp.flags.c_contiguous:
        raise TypeError("row_ptr must be a contiguous int32/int64 array")
    if col_idx.dtype != np.int32 or not col_idx.flags.c_contiguous:
        raise TypeError("col_idx must be a contiguous int32 array")
    V = rp.shape[0] - 1
    if labels is None:
        labels = np.empty(V, np.int32)
    if labels.dtype != np.int32 or labels.shape[0] != V or not labels.flags.c_contiguous:
        raise TypeError("labels must be a contiguous int32 array of V entries")
    itype = CC_INDEX_I64 if rp.dtype == np.int64 else CC_INDEX_I32
    st = load().cc_labels_csr_host(ctx, V, col_idx.shape[0], rp.ctypes.data, itype,
                                   col_idx.ctypes.data if col_idx.size else None,
                                   labels.ctypes.data if V else None)
    _check(st, "cc_labels_csr_host", ctx)
    return labels


def cc_labels_csr_noalloc(row_ptr, col_idx, labels, stream=None, symmetric: bool = False):
    """Allocation-free labelling for callers that cannot allocate device memory.

    Calls the C entry point of the same name, which uses a static scratch block inside
    the library instead of a context; `labels` must be a preallocated int32 CUDA tensor
    of V entries (this wrapper allocates nothing). Synchronous on `stream`."""
    import torch
    if row_ptr.dtype not in (torch.int32, torch.int64):
        raise TypeError("row_ptr must be int32 or int64")
    _dev_tensor(row_ptr, row_ptr.dtype, "row_ptr")
    _dev_tensor(col_idx, torch.int32, "col_idx")
    _dev_tensor(labels, torch.int32, "labels")
    V = row_ptr.numel() - 1
    if labels.numel() != V:
        raise ValueError("labels must hold V entries")
    itype = CC_INDEX_I64 if row_ptr.dtype == torch.int64 else CC_INDEX_I32
    st = load().cc_labels_csr_noalloc(V, col_idx.numel(), row_ptr.data_ptr(), itype,
                                      col_idx.data_ptr() if col_idx.numel() else None,
                                      labels.data_ptr() if V else None,
                                      ctypes.c_void_p(_stream_handle(stream)),
                                      CC_FLAG_SYMMETRIC if symmetric else 0)
    _check(st, "cc_labels_csr_noalloc")
    return labels


def cc_debug_skip_barrier_arrival(ctx, block: int) -> None:
    _check(load().cc_debug_skip_barrier_arrival(ctx, int(block)), "cc_debug_skip_barrier_arrival")


class ConnectedComponents:
    """A library context bound to one device and stream.

    >>> cc = ConnectedComponents(flags=CC_FLAG_SYMMETRIC)
    >>> labels = cc.csr(row_ptr, col_idx); cc.sync()
    """

    def __init__(self, device: int = 0, stream=None, tuner=None, **options):
        """`tuner` (a tune.Tuner) makes every call look up the tuned options of its graph's size
        bucket and run with them (the explicit `options` are the fallback for buckets without a
        tuned entry); `last_options_source` then says which applied."""
        self.device = device
        self.base_options = dict(options)
        self.options = default_options(**options)
        self.tuner = tuner
        self.last_options_source = "explicit"
        self._applied = dict(options)
        self._ctx = cc_create(device, stream, self.options)

    def _apply_tuned(self, tuned):
        want = dict(self.base_options)
        if tuned:
            want.update(tuned)
            want["flags"] = self.base_options.get("flags", 0)  # the caller's flags describe the input
        self.last_options_source = "tuner cache" if tuned else "explicit"
        if want != self._applied:
            self.options = default_options(**want)
            cc_set_options(self._ctx, self.options)
            self._applied = want

    @property
    def handle(self):
        return self._ctx

    def set_options(self, **options):
        for k, v in options.items():
            setattr(self.options, k, int(v))
        cc_set_options(self._ctx, self.options)
        self.base_options.update(options)
        self._applied.update(options)

    def set_stream(self, stream):
        cc_set_stream(self._ctx, stream)

    def csr(self, row_ptr, col_idx, labels=None):
        if self.tuner is not None:
            self._apply_tuned(self.tuner.options_for_csr(row_ptr.numel() - 1, col_idx.numel()))
        return cc_labels_csr(self._ctx, row_ptr, col_idx, labels)

    def csr64(self, row_ptr, col_idx, labels=None):
        return cc_labels_csr64(self._ctx, row_ptr, col_idx, labels)

    def coo(self, n_vertices, src, dst, labels=None):
        return cc_labels_coo(self._ctx, n_vertices, src, dst, labels)

    def batched(self, v_off, a_off, row_ptr_cat, col_idx_cat, labels=None, graph_status=None):
        if self.tuner is not None:
            n = v_off.numel() - 1
            self._apply_tuned(self.tuner.options_for_batch(n, row_ptr_cat.numel() - n, col_idx_cat.numel()))
        return cc_labels_batched(self._ctx, v_off, a_off, row_ptr_cat, col_idx_cat, labels, graph_status)

    def csr_host(self, row_ptr, col_idx, labels=None):
        return cc_labels_csr_host(self._ctx, row_ptr, col_idx, labels)

    def sync(self, raise_input_errors: bool = True):
        return cc_sync(self._ctx, raise_input_errors)

    def set_launch_status(self, device_status=None):
        cc_set_launch_status(self._ctx, device_status)

    def run_info(self):
        return cc_last_run_info(self._ctx)

    def phase_times(self):
        return cc_last_phase_times(self._ctx)

    def worklist(self):
        return cc_last_worklist(self._ctx)

    def close(self):
        if self._ctx:
            cc_destroy(self._ctx)
            self._ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
