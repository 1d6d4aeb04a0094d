"""Autotuner of the launch options (hook choice and its switch thresholds, segments s, hook
window, block size, hook work split, arcs per lane).

The best options depend on the graph family and size and on the GPU, so they are measured, not
guessed: for a graph, a coordinate search times a small set of candidate options through the
library (CUDA events around each call, after a warm-up), checks that every candidate returns the
same labels, and keeps the fastest. Results are cached per size bucket (log2 of |V|, log2 of the
average degree, whether the vertex numbering has locality) in a JSON file, so later graphs of the
same bucket start from the tuned options without measuring.
"""
from __future__ import annotations

import json
import math
import os
import statistics
import threading

from . import cc as ccapi

# Candidate values, searched one option at a time (in this order) from the current best. The mode
# and the thresholds of the automatic choice decide which hook runs (cluster, plain, two-phase,
# sampled-and-filtered); the rest shape the launches of that hook.
SEARCH = [
    ("mode", [0, 1, 5, 6]),
    ("tile_vertices", [0, -1, 8192, 16384, 32768]),
    ("auto_min_vertices", [0, 1 << 15, 1 << 20]),
    ("auto_local_permille", [0, 300, 700]),
    ("auto_lowdeg_permille", [0, 100, 500]),
    ("auto_dense_degree", [0, -1, 4, 16]),
    ("cluster_max_vertices", [0, 1 << 16, 1 << 18, 1 << 19]),
    ("segments", [0, 1, 2, 4, 8, -1]),
    ("block", [0, 256, 512, 1024]),
    ("chunk_arcs", [0, -1, 1024, 2048]),
    ("hook_k", [0, 2, 4]),
]
# The batched launch: its window (graphs up to this size stay in one CTA), segments and block.
SEARCH_BATCHED = [("tile_vertices", [0, 8192, 16384, -1]), ("segments", [0, 1, 2, 4]), ("block", [0, 512, 1024])]

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "gb300_cc_tune.json")


def bucket(kind: str, n_vertices: int, n_arcs: int, local: bool | None = None) -> str:
    """Cache key: graph kind, log2 |V| and log2 average degree rounded, numbering locality."""
    lv = int(round(math.log2(max(1, n_vertices))))
    ld = int(round(math.log2(max(1e-9, n_arcs / max(1, n_vertices))))) if n_arcs else -99
    return f"{kind}:V2^{lv}:d2^{ld}:{'local' if local else 'any' if local is None else 'random'}"


class Tuner:
    def __init__(self, cache_path: str | None = DEFAULT_CACHE):
        self.cache_path = cache_path
        self.cache = {}
        self._lock = threading.Lock()
        if cache_path and os.path.exists(cache_path):
            try:
                with open(cache_path) as f:
                    self.cache = json.load(f)
            except (OSError, ValueError):
                self.cache = {}

    def save(self):
        if not self.cache_path:
            return
        os.makedirs(os.path.dirname(self.cache_path) or ".", exist_ok=True)
        tmp = self.cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(self.cache, f, indent=1, sort_keys=True)
        os.replace(tmp, self.cache_path)

    def lookup(self, key: str):
        with self._lock:
            rec = self.cache.get(key)
        return dict(rec["options"]) if rec else None

    def options_for_csr(self, n_vertices: int, n_arcs: int):
        """Tuned options of the bucket of a CSR graph with these sizes (any numbering), or None."""
        return self.lookup(bucket("csr", n_vertices, n_arcs))

    def options_for_batch(self, n_graphs: int, total_vertices: int, total_arcs: int):
        return self.lookup(bucket(f"batch{int(round(math.log2(max(1, n_graphs))))}", total_vertices, total_arcs))

    def search(self, measure, start: dict | None = None, space=SEARCH):
        """Coordinate search: measure(options) -> (ms, labels). Returns (best options, best ms, log).
        Every candidate's labels must equal the first ones (the options only change the speed)."""
        best = dict(start or {})
        best_ms, ref = measure(best)
        log = [(dict(best), best_ms)]
        for name, values in space:
            for v in values:
                if best.get(name, 0) == v:
                    continue
                cand = dict(best)
                cand[name] = v
                try:
                    ms, labels = measure(cand)
                except ccapi.CCError:
                    continue  # e.g. a block size that cannot be co-resident, or a graph too large for one cluster
                if ref is not None and labels is not None and not _same(labels, ref):
                    raise AssertionError(f"options {cand} changed the labels")
                log.append((dict(cand), ms))
                if ms < best_ms:
                    best, best_ms = cand, ms
        return best, best_ms, log

    def tune_csr(self, row_ptr, col_idx, flags: int = ccapi.CC_FLAG_SYMMETRIC, reps: int = 3,
                 key: str | None = None, local: bool | None = None):
        """Tune cc_labels_csr for this graph (CUDA tensors); caches and returns the best options."""
        import torch
        V = row_ptr.numel() - 1
        key = key or bucket("csr", V, col_idx.numel(), local)
        labels = torch.empty(V, dtype=torch.int32, device=row_ptr.device)

        def measure(opts):
            with ccapi.ConnectedComponents(row_ptr.device.index or 0, flags=flags, **opts) as cc:
                return _time(torch, lambda: cc.csr(row_ptr, col_idx, labels), cc, reps), labels.clone()

        best, ms, log = self.search(measure, self.lookup(key))
        with self._lock:
            self.cache[key] = {"options": best, "ms": ms, "candidates": len(log)}
        self.save()
        return best

    def tune_batched(self, v_off, a_off, row_ptr_cat, col_idx_cat, flags: int = ccapi.CC_FLAG_SYMMETRIC,
                     reps: int = 3, key: str | None = None):
        import torch
        n = v_off.numel() - 1
        total_v = row_ptr_cat.numel() - n
        key = key or bucket(f"batch{int(round(math.log2(max(1, n))))}", total_v, col_idx_cat.numel())
        labels = torch.empty(total_v, dtype=torch.int32, device=v_off.device)
        space = SEARCH_BATCHED

        def measure(opts):
            with ccapi.ConnectedComponents(v_off.device.index or 0, flags=flags, **opts) as cc:
                fn = lambda: cc.batched(v_off, a_off, row_ptr_cat, col_idx_cat, labels)  # noqa: E731
                return _time(torch, fn, cc, reps), labels.clone()

        best, ms, log = self.search(measure, self.lookup(key), space)
        with self._lock:
            self.cache[key] = {"options": best, "ms": ms, "candidates": len(log)}
        self.save()
        return best


def _same(a, b) -> bool:
    try:
        import torch
        if isinstance(a, torch.Tensor):
            return bool(torch.equal(a, b))
    except ImportError:
        pass
    return a == b


def _time(torch, fn, cc, reps: int) -> float:
    fn()
    cc.sync()
    ts = []
    for _ in range(max(1, reps)):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.current_stream()
        e0.record(stream)
        fn()
        e1.record(stream)
        cc.sync()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)
