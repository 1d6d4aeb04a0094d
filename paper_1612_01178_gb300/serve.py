"""Serving loop: connected-components requests admitted by free device memory and labelled by
continuous batching.

Each request is one undirected graph (int32 CSR in pinned host memory). The server keeps three
device arenas (labels, row offsets, arcs) carved out of HBM once; a first-fit allocator places
every admitted request in them and the request's arrays stay there until its labels are back on
the host. The loop:

  1. Arrivals join a FIFO queue.
  2. Admission: the queue head is admitted as soon as its three arena slices fit (later requests
     wait behind it, so a large request cannot starve). Its row offsets and arcs are copied in on
     the copy-in stream right away, while the device may still be busy with an earlier batch.
  3. When the compute stream is idle, every admitted request not yet launched goes into ONE
     descriptor-mode batched launch (cc_labels_batched_desc) that waits on their copy-in events;
     a batch of at most `single_max` requests is launched instead as back-to-back single-graph
     launches, which cost less for few graphs. Requests arriving meanwhile are admitted and
     copied in during that launch: their copies overlap the running batch, and they form the
     next one.
  4. With the launch, each request's label copy-out is queued on the copy-out stream behind the
     batch's completion event; once a copy lands, the request is complete and its arena slices
     are freed.

Latency = completion time - arrival time (host clock). All device work is the library's CUDA
kernels and CUDA copies; this module only schedules them.
"""
from __future__ import annotations

import bisect
import ctypes
import time
from dataclasses import dataclass, field

import numpy as np

from . import cc as ccapi


class ArenaFull(Exception):
    pass


class Arena:
    """First-fit allocator over [0, capacity) elements with coalescing frees (host bookkeeping)."""

    def __init__(self, capacity: int, align: int = 32):
        self.capacity = int(capacity)
        self.align = int(align)
        self._starts = [0]            # free blocks, sorted by start
        self._sizes = {0: self.capacity}
        self.used = 0

    def _round(self, n: int) -> int:
        return max(self.align, (int(n) + self.align - 1) // self.align * self.align)

    def alloc(self, n: int):
        """Offset of a block of at least n elements, or None if no free block is large enough."""
        need = self._round(n)
        for i, s in enumerate(self._starts):
            size = self._sizes[s]
            if size >= need:
                del self._starts[i]
                del self._sizes[s]
                if size > need:
                    bisect.insort(self._starts, s + need)
                    self._sizes[s + need] = size - need
                self.used += need
                return s
        return None

    def free(self, off: int, n: int) -> None:
        size = self._round(n)
        self.used -= size
        i = bisect.bisect_left(self._starts, off)
        # merge with the next free block
        if i < len(self._starts) and self._starts[i] == off + size:
            nxt = self._starts.pop(i)
            size += self._sizes.pop(nxt)
        # merge with the previous free block
        if i > 0 and self._starts[i - 1] + self._sizes[self._starts[i - 1]] == off:
            prev = self._starts[i - 1]
            self._sizes[prev] += size
        else:
            self._starts.insert(i, off)
            self._sizes[off] = size

    def free_blocks(self):
        return [(s, self._sizes[s]) for s in self._starts]


@dataclass
class Request:
    rid: int
    arrival: float                 # seconds on the server clock
    row_ptr: np.ndarray            # int32 [V+1] (pinned host memory gives full copy bandwidth)
    col: np.ndarray                # int32 [nnz]
    labels: np.ndarray = None      # int32 [V] result (pinned host), filled on completion
    t_admit: float = None
    t_launch: float = None
    t_done: float = None
    slots: tuple = None            # (label_off, row_off, arc_off)
    ev_in: object = None
    ev_out: object = None
    status: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def n_vertices(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def n_arcs(self) -> int:
        return int(self.col.shape[0])

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


class Server:
    """Continuous-batching CC server on one GPU (see the module docstring)."""

    def __init__(self, device: int = 0, label_elems: int = 1 << 27, row_elems: int = 1 << 27,
                 arc_elems: int = 1 << 30, max_batch: int = 1024, flags: int = ccapi.CC_FLAG_SYMMETRIC,
                 pin_results: bool = True):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", device)
        if label_elems >= (1 << 31) - 1:
            raise ValueError("label arena must hold fewer than 2^31 entries")
        self.labels = torch.empty(label_elems, dtype=torch.int32, device=self.dev)
        self.rows = torch.empty(row_elems, dtype=torch.int32, device=self.dev)
        self.arcs = torch.empty(arc_elems, dtype=torch.int32, device=self.dev)
        self.arena = {"label": Arena(label_elems), "row": Arena(row_elems), "arc": Arena(arc_elems)}
        self.max_batch = int(max_batch)
        self.desc_np = torch.empty((max_batch, 5), dtype=torch.int64).pin_memory().numpy()
        self.desc_dev = torch.empty((max_batch, 5), dtype=torch.int64, device=self.dev)
        self.status_dev = torch.empty(max_batch, dtype=torch.int32, device=self.dev)
        self.s_in = torch.cuda.Stream(self.dev)
        self.s_out = torch.cuda.Stream(self.dev)
        self.s_cc = torch.cuda.Stream(self.dev)
        self.cc = ccapi.ConnectedComponents(device, stream=self.s_cc, flags=flags)
        # a batch of at most `single_max` requests goes through the single-graph entry point, one
        # launch per request back to back on the compute stream (lower fixed cost than one
        # batched launch); the plain hook avoids the one-off locality sample, which would
        # synchronise the loop
        self.cc_one = ccapi.ConnectedComponents(device, stream=self.s_cc, flags=flags, tile_vertices=-1)
        self.single_fast_path = True
        self.single_max = 4
        self.pin_results = pin_results
        self.batches = []  # (n_requests, n_arcs) per launch, for reporting

    @staticmethod
    def budget_from_free_memory(fraction: float = 0.5, device: int = 0, avg_degree: float = 16.0):
        """Arena sizes (elements) splitting `fraction` of the currently free HBM between the
        label, row-offset and arc arenas in proportion to a graph of the given average degree."""
        import torch
        free, _ = torch.cuda.mem_get_info(device)
        elems = int(free * fraction) // 4
        per_vertex = 2 + avg_degree  # label + row offset + arcs
        v = min(int(elems / per_vertex), (1 << 31) - 2)
        return dict(label_elems=v, row_elems=v + v // 16 + 4096, arc_elems=int(v * avg_degree))

    # -------------------------------------------------------------------- admission and copies

    def fits(self, req: Request) -> bool:
        V, E = req.n_vertices, req.n_arcs
        return (V <= self.arena["label"].capacity and V + 1 <= self.arena["row"].capacity and
                E <= self.arena["arc"].capacity)

    def try_admit(self, req: Request, now: float) -> bool:
        V, E = req.n_vertices, req.n_arcs
        lo = self.arena["label"].alloc(max(V, 1))
        if lo is None:
            return False
        ro = self.arena["row"].alloc(V + 1)
        if ro is None:
            self.arena["label"].free(lo, max(V, 1))
            return False
        ao = self.arena["arc"].alloc(max(E, 1))
        if ao is None:
            self.arena["label"].free(lo, max(V, 1))
            self.arena["row"].free(ro, V + 1)
            return False
        req.slots = (lo, ro, ao)
        req.t_admit = now
        torch = self.torch
        with torch.cuda.stream(self.s_in):
            self.rows[ro: ro + V + 1].copy_(torch.from_numpy(req.row_ptr), non_blocking=True)
            if E:
                self.arcs[ao: ao + E].copy_(torch.from_numpy(req.col), non_blocking=True)
            req.ev_in = torch.cuda.Event()
            req.ev_in.record(self.s_in)
        return True

    def release(self, req: Request) -> None:
        lo, ro, ao = req.slots
        self.arena["label"].free(lo, max(req.n_vertices, 1))
        self.arena["row"].free(ro, req.n_vertices + 1)
        self.arena["arc"].free(ao, max(req.n_arcs, 1))
        req.slots = None

    def launch(self, batch, now: float):
        torch = self.torch
        n = len(batch)
        if n <= self.single_max and self.single_fast_path:
            for r in batch:
                lo, ro, ao = r.slots
                r.t_launch = now
                self.s_cc.wait_event(r.ev_in)
                V, E = r.n_vertices, r.n_arcs
                ccapi.cc_labels_csr(self.cc_one.handle, self.rows[ro: ro + V + 1], self.arcs[ao: ao + E],
                                    self.labels[lo: lo + V])
            with torch.cuda.stream(self.s_cc):
                self.status_dev[:n].zero_()
            ev = torch.cuda.Event()
            ev.record(self.s_cc)
            self.batches.append((n, sum(r.n_arcs for r in batch)))
            return ev
        for i, r in enumerate(batch):
            lo, ro, ao = r.slots
            self.desc_np[i] = (lo, ro, ao, r.n_arcs, r.n_vertices)  # last word: n_vertices | reserved << 32
            r.t_launch = now
            self.s_cc.wait_event(r.ev_in)
        with torch.cuda.stream(self.s_cc):
            self.desc_dev[:n].copy_(torch.from_numpy(self.desc_np[:n]), non_blocking=True)
        lib = ccapi.load()
        st = lib.cc_labels_batched_desc(self.cc.handle, n, self.desc_dev.data_ptr(), self.rows.data_ptr(),
                                        self.rows.numel(), self.arcs.data_ptr(), self.arcs.numel(),
                                        self.labels.data_ptr(), self.labels.numel(), self.status_dev.data_ptr())
        ccapi._check(st, "cc_labels_batched_desc", self.cc.handle)
        ev = torch.cuda.Event()
        ev.record(self.s_cc)
        self.batches.append((n, sum(r.n_arcs for r in batch)))
        return ev

    def copy_out(self, batch, ev_batch):
        torch = self.torch
        self.s_out.wait_event(ev_batch)
        status = torch.empty(len(batch), dtype=torch.int32).pin_memory() if self.pin_results else None
        with torch.cuda.stream(self.s_out):
            for r in batch:
                lo = r.slots[0]
                if r.labels is None:
                    buf = torch.empty(r.n_vertices, dtype=torch.int32)
                    r.labels = (buf.pin_memory() if self.pin_results else buf).numpy()
                if r.n_vertices:
                    torch.from_numpy(r.labels).copy_(self.labels[lo: lo + r.n_vertices], non_blocking=True)
            if status is not None:
                status.copy_(self.status_dev[:len(batch)], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.s_out)
        for i, r in enumerate(batch):
            r.ev_out = ev
            r.extra["status_buf"] = (status, i)

    # --------------------------------------------------------------------------------- run loop

    def run(self, requests, clock=None, time_limit: float = 600.0):
        """Serve `requests` (sorted by arrival, arrival times relative to the start of the run).
        Returns them with t_admit/t_launch/t_done/labels filled."""
        clock = clock or time.perf_counter
        t0 = clock()
        requests = sorted(requests, key=lambda r: r.arrival)
        for r in requests:
            if not self.fits(r):
                raise ValueError(f"request {r.rid} (V={r.n_vertices}, arcs={r.n_arcs}) exceeds the arenas")
        nxt = 0
        queue, admitted, finishing = [], [], []
        running = None  # (batch, event)
        done = 0
        while done < len(requests):
            now = clock() - t0
            if now > time_limit:
                raise TimeoutError("serving loop exceeded its time limit")
            while nxt < len(requests) and requests[nxt].arrival <= now:
                queue.append(requests[nxt])
                nxt += 1
            while queue and self.try_admit(queue[0], now):
                admitted.append(queue.pop(0))
            if running is not None and running[1].query():
                finishing.extend(running[0])
                running = None
            if running is None and admitted:
                batch, admitted = admitted[:self.max_batch], admitted[self.max_batch:]
                ev = self.launch(batch, now)
                self.copy_out(batch, ev)  # the copy-out stream waits for the batch on the device
                running = (batch, ev)
            still = []
            for r in finishing:
                if r.ev_out.query():
                    r.t_done = clock() - t0
                    sbuf, i = r.extra.pop("status_buf")
                    r.status = int(sbuf[i]) if sbuf is not None else 0
                    self.release(r)
                    done += 1
                else:
                    still.append(r)
            finishing = still
            if not queue and not admitted and running is None and not finishing and nxt < len(requests):
                wait = requests[nxt].arrival - (clock() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.001))
        self.cc.sync()
        self.cc_one.sync()  # raises if a single-request launch reported a device error
        return requests

    def close(self):
        self.cc.close()
        self.cc_one.close()


def latency_summary(requests) -> dict:
    lat = np.array([r.latency for r in requests]) * 1000.0
    dev = np.array([r.t_done - r.t_launch for r in requests]) * 1000.0
    span = max(r.t_done for r in requests) - min(r.arrival for r in requests)
    arcs = sum(r.n_arcs for r in requests)
    return {"requests": len(requests), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "device_p50_ms": float(np.percentile(dev, 50)),
            "device_p99_ms": float(np.percentile(dev, 99)), "throughput_req_s": len(requests) / span,
            "edges_per_s": (arcs / 2) / span}


class SequentialServer:
    """Baseline for the serving loop: one request at a time through the single-graph entry point
    (copy in, cc_labels_csr, copy out, wait), in arrival order, with no batching or overlap."""

    def __init__(self, device: int = 0, flags: int = ccapi.CC_FLAG_SYMMETRIC):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.stream = torch.cuda.Stream(self.dev)
        self.cc = ccapi.ConnectedComponents(device, stream=self.stream, flags=flags)

    def run(self, requests, clock=None, time_limit: float = 600.0):
        torch = self.torch
        clock = clock or time.perf_counter
        t0 = clock()
        for r in sorted(requests, key=lambda q: q.arrival):
            while clock() - t0 < r.arrival:
                time.sleep(min(0.0005, max(0.0, r.arrival - (clock() - t0))))
            if clock() - t0 > time_limit:
                raise TimeoutError("sequential baseline exceeded its time limit")
            r.t_admit = r.t_launch = clock() - t0
            with torch.cuda.stream(self.stream):
                rp = torch.from_numpy(r.row_ptr).to(self.dev, non_blocking=True)
                col = torch.from_numpy(r.col).to(self.dev, non_blocking=True)
                out = self.cc.csr(rp, col)
                if r.labels is None:
                    r.labels = torch.empty(r.n_vertices, dtype=torch.int32).pin_memory().numpy()
                torch.from_numpy(r.labels).copy_(out, non_blocking=True)
            self.stream.synchronize()
            r.t_done = clock() - t0
        self.cc.sync()
        return requests

    def close(self):
        self.cc.close()
