"""Serving loop: connected-components requests admitted by free device memory and labelled by
continuous batching.

Each request is one undirected graph (int32 CSR in pinned host memory). The server keeps three
device arenas (labels, row offsets, arcs) carved out of HBM once; a first-fit allocator places
every admitted request in them and the request's arrays stay there until its labels are back on
the host. The loop:

  1. Arrivals join a FIFO queue.
  2. Admission: the queue head is admitted as soon as its three arena slices fit (later requests
     wait behind it, so a large request cannot starve). While every lane is busy, its row offsets
     and arcs are copied in on the copy-in stream right away, overlapping the batches on the
     device; when a lane is idle (the request is launched at once) the copy goes on that lane's
     stream instead, ahead of the launch. A request that can never fit, or whose admission or
     copy-in fails, is rejected with a status (CC_ERR_OOM, CC_ERR_CUDA) and the loop goes on
     serving the others.
  3. The server has `lanes` compute lanes (a stream with its own library contexts each). When a
     lane is idle, every admitted request not yet launched goes into ONE launch on that lane (on the
     lane's share of the SMs): a
     descriptor-mode batched launch (cc_labels_batched_desc) that waits on the requests' copy-in
     events, or, for a batch of at most `single_max` requests, back-to-back single-graph launches
     (cheaper for few graphs), each with the hook its graph calls for (chosen on the host from a
     small sample of the request's degrees and arcs). Requests arriving meanwhile are admitted and
     copied in during those launches and form the next batch, on the other lane if it is idle:
     batches of two lanes run on the device at the same time.
  4. With the launch, each request's labels and status are queued for copy-out on the lane's
     stream behind the kernels, into host buffers the request brought (or that the server pins
     for it); once the lane's work is done its requests are complete and their arena slices
     are freed.

Every request carries its own status: CC_OK, CC_ERR_OUT_OF_RANGE when its graph is malformed
(an endpoint outside [0, V), offsets inconsistent with its arcs; reported by the kernels for
that graph alone, the others of the batch are labelled normally), or the admission error.
Latency = completion time - arrival time (host clock). All device work is the library's CUDA
kernels and CUDA copies; this module only schedules them.
"""
from __future__ import annotations

import bisect
import time
from dataclasses import dataclass, field

import numpy as np

from . import cc as ccapi


class AdmissionError(Exception):
    """Raised by an admission step (arena allocation, copy-in) that failed for one request."""


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
    labels: np.ndarray = None      # int32 [V] result (pinned host); bring one to avoid pinning per request
    t_admit: float = None
    t_launch: float = None
    t_done: float = None
    slots: tuple = None            # (label_off, row_off, arc_off)
    ev_in: object = None
    status: int = 0
    error: str = ""
    hook: str = ""                 # single-graph launches: the hook chosen for this graph
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


# The library's automatic choice of a hook needs a sampling kernel and a synchronisation per new
# graph; a serving loop decides on the host from the request's own arrays instead, with the same
# rules: a symmetric graph of mean degree n_arcs / V >= 8 below 2^17 vertices takes the
# sampled-and-filtered hook, any other graph that small the plain hook; from 2^17 vertices on, if
# most sampled arcs join two vertices of one 16384-vertex window, the two-phase hook; else, if the
# graph is symmetric and a quarter of the sampled rows have a degree below a quarter of the mean
# (a skewed, power-law-like graph) or its mean degree is >= 8, the sampled-and-filtered hook.
HOOK_MIN_VERTICES = 1 << 17
HOOK_DENSE_DEGREE = 8
HOOK_WINDOW = 16384
HOOK_SAMPLES = 256


def choose_hook(row_ptr: np.ndarray, col: np.ndarray, symmetric: bool = True) -> str:
    V = row_ptr.shape[0] - 1
    nnz = col.shape[0]
    dense = symmetric and nnz >= HOOK_DENSE_DEGREE * V
    if nnz == 0:
        return "plain"
    if V < HOOK_MIN_VERTICES:
        return "filtered" if dense else "plain"
    u = np.linspace(0, V - 1, HOOK_SAMPLES).astype(np.int64)
    a0 = row_ptr[u].astype(np.int64)
    a1 = row_ptr[u + 1].astype(np.int64)
    ok = (a0 >= 0) & (a0 < a1) & (a1 <= nnz)
    if not ok.any():
        return "plain"
    mid = np.where(ok, (a0 + a1) // 2, 0)
    v = col[mid].astype(np.int64)
    sampled = ok & (v >= 0) & (v < V) & (v != u)
    local = sampled & (u // HOOK_WINDOW == v // HOOK_WINDOW)
    if sampled.sum() and local.sum() >= 0.5 * sampled.sum():
        return "tiled"
    low = (4.0 * (a1 - a0) * V < nnz) & (a0 <= a1)
    if symmetric and (low.mean() >= 0.25 or dense):
        return "filtered"
    return "plain"


class Server:
    """Continuous-batching CC server on one GPU (see the module docstring).

    `inject`, if given, is called as inject(stage, request) at the admission steps "admit"
    (before the arena slices are taken) and "copy_in" (before the copies are issued); an
    exception it raises rejects that request the way a failing allocator or copy would."""

    STATUS_BUFFERS = 4

    def __init__(self, device: int = 0, label_elems: int = 1 << 27, row_elems: int = 1 << 27,
                 arc_elems: int = 1 << 30, max_batch: int = 1024, flags: int = ccapi.CC_FLAG_SYMMETRIC,
                 lanes: int = 2, single_max: int = 4, inject=None):
        if label_elems >= (1 << 31) - 1:
            raise ValueError("label arena must hold fewer than 2^31 entries")
        self.device = device
        self.caps = {"label": int(label_elems), "row": int(row_elems), "arc": int(arc_elems)}
        self.arena = {k: Arena(v) for k, v in self.caps.items()}
        self.max_batch = int(max_batch)
        self.flags = flags
        self.n_lanes = max(1, int(lanes))
        self.single_max = int(single_max)
        self.single_fast_path = True
        self.inject = inject
        self.batches = []  # (n_requests, n_arcs, lane) per launch, for reporting
        self._setup_device()

    # ------------------------------------------------------------------ device side (CUDA)

    def _setup_device(self):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda", self.device)
        self.labels = torch.empty(self.caps["label"], dtype=torch.int32, device=self.dev)
        self.rows = torch.empty(self.caps["row"], dtype=torch.int32, device=self.dev)
        self.arcs = torch.empty(self.caps["arc"], dtype=torch.int32, device=self.dev)
        self.s_in = torch.cuda.Stream(self.dev)
        n_sms = torch.cuda.get_device_properties(self.dev).multi_processor_count
        # Each lane's launches fill its share of the SMs, so the lanes' cooperative launches can be
        # resident together (a lane alone on every SM measured slower under load: the other lane's
        # launch then waits for SMs, and batches serialise).
        self.share = 0 if self.n_lanes == 1 else max(1, n_sms // self.n_lanes)
        self.lanes = []
        for _ in range(self.n_lanes):
            s = torch.cuda.Stream(self.dev)
            opts = dict(flags=self.flags, sm_limit=self.share)
            lane = {
                "stream": s,
                "batched": ccapi.ConnectedComponents(self.device, stream=s, **opts),
                # single-graph launches: each hook forced, so no launch needs the one-off sample
                "plain": ccapi.ConnectedComponents(self.device, stream=s, tile_vertices=-1, **opts),
                "tiled": ccapi.ConnectedComponents(self.device, stream=s, tile_vertices=HOOK_WINDOW, **opts),
                "filtered": (ccapi.ConnectedComponents(self.device, stream=s, mode=ccapi.CC_MODE_FILTERED, **opts)
                             if self.flags & ccapi.CC_FLAG_SYMMETRIC else None),
                "desc_np": torch.empty((self.max_batch, 5), dtype=torch.int64).pin_memory().numpy(),
                "desc_dev": torch.empty((self.max_batch, 5), dtype=torch.int64, device=self.dev),
                # per-request statuses: STATUS_BUFFERS slots per lane, each reused only after every
                # request of the batch that used it was read back
                "status_dev": torch.empty((self.STATUS_BUFFERS, self.max_batch), dtype=torch.int32, device=self.dev),
                "status_host": torch.empty((self.STATUS_BUFFERS, self.max_batch), dtype=torch.int32).pin_memory(),
                "busy": [0] * self.STATUS_BUFFERS,
                "running": None,
            }
            self.lanes.append(lane)

    def _copy_in(self, req: Request, stream=None):
        """H2D of the request's arrays on `stream` (default: the copy-in stream); returns an event
        recorded after the copies (None when issued on a lane's own stream)."""
        torch = self.torch
        lo, ro, ao = req.slots
        V, E = req.n_vertices, req.n_arcs
        with torch.cuda.stream(stream or self.s_in):
            self.rows[ro: ro + V + 1].copy_(torch.from_numpy(req.row_ptr), non_blocking=True)
            if E:
                self.arcs[ao: ao + E].copy_(torch.from_numpy(req.col), non_blocking=True)
            if stream is not None:
                return None
            ev = torch.cuda.Event()
            ev.record(self.s_in)
        return ev

    def _launch(self, lane, batch, k):
        """Copies in the requests not yet on the device, labels the batch and queues the copy-out of
        labels and statuses, all on the lane's stream. Returns the event recorded after them."""
        torch = self.torch
        s = lane["stream"]
        n = len(batch)
        st = lane["status_dev"][k]
        lib = ccapi.load()
        for r in batch:
            if r.ev_in is None:
                self._copy_in(r, stream=s)
            else:
                s.wait_event(r.ev_in)
        if n <= self.single_max and self.single_fast_path:
            rows, arcs, labels, st0 = self.rows.data_ptr(), self.arcs.data_ptr(), self.labels.data_ptr(), st.data_ptr()
            for i, r in enumerate(batch):
                lo, ro, ao = r.slots
                ctx = lane[r.hook] if lane.get(r.hook) is not None else lane["plain"]
                ccapi._check(lib.cc_set_launch_status(ctx.handle, st0 + 4 * i), "cc_set_launch_status")
                rc = lib.cc_labels_csr(ctx.handle, r.n_vertices, r.n_arcs, rows + 4 * ro, ccapi.CC_INDEX_I32,
                                       arcs + 4 * ao if r.n_arcs else None, labels + 4 * lo if r.n_vertices else None)
                ccapi._check(rc, "cc_labels_csr", ctx.handle)
        else:
            dnp = lane["desc_np"]
            for i, r in enumerate(batch):
                lo, ro, ao = r.slots
                dnp[i] = (lo, ro, ao, r.n_arcs, r.n_vertices)  # last word: n_vertices | reserved << 32
            with torch.cuda.stream(s):
                lane["desc_dev"][:n].copy_(torch.from_numpy(dnp[:n]), non_blocking=True)
            rc = lib.cc_labels_batched_desc(lane["batched"].handle, n, lane["desc_dev"].data_ptr(),
                                            self.rows.data_ptr(), self.rows.numel(), self.arcs.data_ptr(),
                                            self.arcs.numel(), self.labels.data_ptr(), self.labels.numel(),
                                            st.data_ptr())
            ccapi._check(rc, "cc_labels_batched_desc", lane["batched"].handle)
        with torch.cuda.stream(s):
            for r in batch:
                lo = r.slots[0]
                if r.labels is None:  # the request brought no output buffer
                    r.labels = torch.empty(r.n_vertices, dtype=torch.int32).pin_memory().numpy()
                if r.n_vertices:
                    torch.from_numpy(r.labels).copy_(self.labels[lo: lo + r.n_vertices], non_blocking=True)
            lane["status_host"][k, :n].copy_(st[:n], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        return ev

    def _read_status(self, lane, k: int, i: int) -> int:
        return int(lane["status_host"][k, i])

    def _sync_lanes(self):
        for lane in self.lanes:
            for k in ("batched", "plain", "tiled", "filtered"):
                if lane[k] is not None:
                    lane[k].sync(raise_input_errors=False)  # input errors are per request

    def close(self):
        for lane in self.lanes:
            for k in ("batched", "plain", "tiled", "filtered"):
                if lane[k] is not None:
                    lane[k].close()

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
        return V <= self.caps["label"] and V + 1 <= self.caps["row"] and E <= self.caps["arc"]

    def try_admit(self, req: Request, now: float, defer_copy: bool = False) -> bool:
        """Admit `req` if its slices fit (True), or leave it queued (False). With defer_copy the
        copy-in waits for the launch (issued on the lane's stream). Raises AdmissionError when
        admitting it failed (it is then rejected)."""
        if self.inject is not None:
            try:
                self.inject("admit", req)
            except Exception as e:  # an allocation failure as the allocator would report it
                raise AdmissionError(f"admission failed: {e!r}") from e
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
        try:
            if self.inject is not None:
                self.inject("copy_in", req)
            req.ev_in = None if defer_copy else self._copy_in(req)
        except Exception as e:
            self.release(req)
            req.extra["copy_failed"] = True
            raise AdmissionError(f"copy-in failed: {e!r}") from e
        req.hook = choose_hook(req.row_ptr, req.col, bool(self.flags & ccapi.CC_FLAG_SYMMETRIC))
        return True

    def release(self, req: Request) -> None:
        lo, ro, ao = req.slots
        self.arena["label"].free(lo, max(req.n_vertices, 1))
        self.arena["row"].free(ro, req.n_vertices + 1)
        self.arena["arc"].free(ao, max(req.n_arcs, 1))
        req.slots = None

    # --------------------------------------------------------------------------------- run loop

    def run(self, requests, clock=None, time_limit: float = 600.0):
        """Serve `requests` (sorted by arrival, arrival times relative to the start of the run).
        Returns them with t_admit/t_launch/t_done/labels/status filled; rejected requests have a
        non-zero status and no labels."""
        clock = clock or time.perf_counter
        t0 = clock()
        requests = sorted(requests, key=lambda r: r.arrival)
        for r in requests:
            r.status, r.error, r.t_done, r.ev_in = 0, "", None, None
        nxt = 0
        queue, admitted = [], []
        done = 0

        def reject(r, status, why, now):
            r.status, r.error = status, why
            r.t_done = now
            r.labels = None

        while done < len(requests):
            now = clock() - t0
            if now > time_limit:
                raise TimeoutError("serving loop exceeded its time limit")
            while nxt < len(requests) and requests[nxt].arrival <= now:
                queue.append(requests[nxt])
                nxt += 1
            while queue:
                r = queue[0]
                if not self.fits(r):  # can never fit the arenas
                    queue.pop(0)
                    reject(r, ccapi.CC_ERR_OOM, "request larger than the arenas", now)
                    done += 1
                    continue
                idle = any(lane["running"] is None for lane in self.lanes)
                try:
                    if not self.try_admit(r, now, defer_copy=idle):
                        break
                except AdmissionError as e:
                    queue.pop(0)
                    reject(r, ccapi.CC_ERR_CUDA if r.extra.pop("copy_failed", False) else ccapi.CC_ERR_OOM,
                           str(e), now)
                    done += 1
                    continue
                admitted.append(queue.pop(0))
            for lane in self.lanes:
                run = lane["running"]
                if run is not None and run[1].query():  # kernels and copy-out of the batch are done
                    t_done = clock() - t0
                    for i, r in enumerate(run[0]):
                        r.t_done = t_done
                        r.status = self._read_status(lane, run[2], i)
                        self.release(r)
                        done += 1
                    lane["busy"][run[2]] = 0
                    lane["running"] = None
            for lane in self.lanes:
                if lane["running"] is None and admitted:
                    k = next((j for j, b in enumerate(lane["busy"]) if b == 0), None)
                    if k is None:  # every status slot of this lane still has results to read
                        continue
                    batch, admitted = admitted[:self.max_batch], admitted[self.max_batch:]
                    for r in batch:
                        r.t_launch = now
                    ev = self._launch(lane, batch, k)
                    lane["busy"][k] = len(batch)
                    lane["running"] = (batch, ev, k)
                    self.batches.append((len(batch), sum(r.n_arcs for r in batch), self.lanes.index(lane)))
            busy = any(lane["running"] is not None for lane in self.lanes)
            if not queue and not admitted and not busy and nxt < len(requests):
                wait = requests[nxt].arrival - (clock() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.001))
        self._sync_lanes()  # raises on a fatal device error
        return requests


def latency_summary(requests) -> dict:
    served = [r for r in requests if r.status == 0]
    lat = np.array([r.latency for r in served]) * 1000.0
    dev = np.array([r.t_done - r.t_launch for r in served]) * 1000.0
    span = max(r.t_done for r in requests) - min(r.arrival for r in requests)
    arcs = sum(r.n_arcs for r in served)
    return {"requests": len(requests), "failed": len(requests) - len(served),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "device_p50_ms": float(np.percentile(dev, 50)),
            "device_p99_ms": float(np.percentile(dev, 99)), "throughput_req_s": len(served) / span,
            "edges_per_s": (arcs / 2) / span}


class SequentialServer:
    """Baseline for the serving loop: one request at a time through the single-graph entry point
    (copy in, cc_labels_csr with the library's automatic hook, copy out, wait), in arrival order,
    with no batching or overlap."""

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
