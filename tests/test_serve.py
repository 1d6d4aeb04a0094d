"""Host-side logic of the serving loop (no GPU): the first-fit arena allocator behind admission by
free device memory, and the run loop itself over a stand-in device whose "kernels" are the oracle:
FIFO admission, batching over several lanes, per-request status, and failures injected on the host
(an allocation or a copy-in that fails, a request that can never fit, a malformed request), each of
which must reject that request alone while every other request is still served correctly."""
import numpy as np
import pytest

import gen
import oracle
from paper_1612_01178_gb300 import cc as ccapi
from paper_1612_01178_gb300.serve import Arena, Request, Server, choose_hook, latency_summary


def test_alloc_free_coalesce():
    a = Arena(1024, align=32)
    x = a.alloc(100)   # 128
    y = a.alloc(200)   # 224
    z = a.alloc(300)   # 320
    assert (x, y, z) == (0, 128, 352)
    assert a.used == 128 + 224 + 320
    assert a.alloc(500) is None            # only 352 left at the end
    a.free(y, 200)
    assert a.alloc(224) == 128             # first fit reuses the hole
    a.free(128, 224)
    a.free(x, 100)
    a.free(z, 300)
    assert a.used == 0 and a.free_blocks() == [(0, 1024)]


def test_random_alloc_free_never_overlaps():
    rng = np.random.default_rng(0)
    a = Arena(1 << 16, align=32)
    live = {}
    for _ in range(3000):
        if live and rng.random() < 0.45:
            off = list(live)[int(rng.integers(0, len(live)))]
            a.free(off, live.pop(off))
        else:
            n = int(rng.integers(1, 3000))
            off = a.alloc(n)
            if off is not None:
                live[off] = n
        spans = sorted((o, o + ((n + 31) // 32) * 32) for o, n in live.items())
        assert all(s1[1] <= s2[0] for s1, s2 in zip(spans, spans[1:]))
        assert all(0 <= s[0] and s[1] <= a.capacity for s in spans)
        assert a.used == sum(e - s for s, e in spans)
    for off, n in list(live.items()):
        a.free(off, n)
    assert a.free_blocks() == [(0, 1 << 16)]


class _Event:
    """Completes after a fixed number of polls (a stand-in for a CUDA event)."""

    def __init__(self, polls):
        self.polls = polls

    def query(self):
        self.polls -= 1
        return self.polls <= 0


class FakeServer(Server):
    """The serving loop over a stand-in device: launches compute the oracle's labels at once and
    report CC_ERR_OUT_OF_RANGE for a malformed graph, as the kernels do; events complete after a
    few polls so that batches stay "on the device" for a while and overlap across lanes."""

    polls = 3

    def _setup_device(self):
        self.lanes = [{"running": None, "busy": [0] * self.STATUS_BUFFERS,
                       "status": [[0] * self.max_batch for _ in range(self.STATUS_BUFFERS)]}
                      for _ in range(self.n_lanes)]
        self.in_flight_max = 0
        self.copies_in = 0

    def _copy_in(self, req, stream=None):
        self.copies_in += 1
        return None if stream is not None else _Event(1)

    def _launch(self, lane, batch, k):
        for i, r in enumerate(batch):
            if r.ev_in is None:
                self._copy_in(r, stream=lane)
            V = r.n_vertices
            bad = r.n_arcs and (r.col.min() < 0 or r.col.max() >= V or r.row_ptr[-1] != r.n_arcs)
            lane["status"][k][i] = ccapi.CC_ERR_OUT_OF_RANGE if bad else 0
            if r.labels is None:
                r.labels = np.empty(r.n_vertices, np.int32)
            if not bad:
                r.labels[:] = oracle.labels_uf_csr(r.row_ptr, r.col)[0]
        running = sum(1 for ln in self.lanes if ln["running"] is not None) + 1
        self.in_flight_max = max(self.in_flight_max, running)
        return _Event(self.polls)

    def _read_status(self, lane, k, i):
        return lane["status"][k][i]

    def _sync_lanes(self):
        pass

    def close(self):
        pass


def graphs(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        if i % 2:
            out.append(gen.er_csr(int(rng.integers(10, 400)), int(rng.integers(5, 900)), seed=seed * 100 + i))
        else:
            out.append(gen.rmat_csr(int(rng.integers(4, 9)), 4, seed=seed * 100 + i))
    return out


def requests(gs, arrivals):
    return [Request(i, float(t), g.row_ptr, g.col) for i, (g, t) in enumerate(zip(gs, arrivals))]


def check_served(out, gs, failed=()):
    for r in out:
        if r.rid in failed:
            continue
        assert r.status == 0, (r.rid, r.status, r.error)
        assert np.array_equal(r.labels, oracle.labels_uf_csr(gs[r.rid].row_ptr, gs[r.rid].col)[0]), r.rid


def test_run_loop_serves_every_request_over_two_lanes():
    gs = graphs(40, 1)
    srv = FakeServer(0, label_elems=1 << 12, row_elems=1 << 12, arc_elems=1 << 14, max_batch=8, lanes=2)
    out = srv.run(requests(gs, np.zeros(len(gs))))
    check_served(out, gs)
    assert srv.in_flight_max == 2                     # both lanes had a batch on the device at once
    assert max(n for n, _, _ in srv.batches) > 1      # requests were batched together
    assert {lane for _, _, lane in srv.batches} == {0, 1}
    assert all(a.used == 0 for a in srv.arena.values())
    assert srv.copies_in == len(gs)                   # every request copied in exactly once
    s = latency_summary(out)
    assert s["failed"] == 0 and s["p99_ms"] >= s["p50_ms"] >= 0


@pytest.mark.parametrize("stage,status", [("admit", ccapi.CC_ERR_OOM), ("copy_in", ccapi.CC_ERR_CUDA)])
def test_injected_admission_failure_rejects_only_that_request(stage, status):
    gs = graphs(30, 2)
    victims = {3, 11, 12, 29}

    def inject(where, req):
        if where == stage and req.rid in victims:
            raise RuntimeError(f"injected {where} failure")

    srv = FakeServer(0, label_elems=1 << 12, row_elems=1 << 12, arc_elems=1 << 14, max_batch=6, inject=inject)
    out = srv.run(requests(gs, np.linspace(0, 0.002, len(gs))))
    for r in out:
        if r.rid in victims:
            assert r.status == status and r.labels is None and "injected" in r.error
    check_served(out, gs, failed=victims)
    assert all(a.used == 0 for a in srv.arena.values())  # a failed copy-in gave its slices back
    assert latency_summary(out)["failed"] == len(victims)


def test_malformed_and_oversized_requests_fail_alone():
    gs = graphs(20, 3)
    bad = gs[5]
    col = bad.col.copy()
    col[0] = bad.n_vertices + 3
    gs[5] = gen.CSR(bad.n_vertices, bad.row_ptr, col, bad.n_edges, "bad")
    huge = gen.er_csr(5000, 100, seed=1)  # more vertices than the label arena holds
    gs.append(huge)
    srv = FakeServer(0, label_elems=4096, row_elems=1 << 13, arc_elems=1 << 14, max_batch=4)
    out = srv.run(requests(gs, np.zeros(len(gs))))
    by_id = {r.rid: r for r in out}
    assert by_id[5].status == ccapi.CC_ERR_OUT_OF_RANGE
    assert by_id[len(gs) - 1].status == ccapi.CC_ERR_OOM
    check_served(out, gs, failed={5, len(gs) - 1})


def test_admission_waits_for_memory_in_fifo_order():
    gs = [gen.er_csr(1500, 3000, seed=i) for i in range(10)]
    srv = FakeServer(0, label_elems=3200, row_elems=3300, arc_elems=13000, max_batch=16, lanes=1)
    out = srv.run(requests(gs, np.zeros(len(gs))))
    check_served(out, gs)
    assert max(n for n, _, _ in srv.batches) <= 2      # at most two requests fit at once
    admits = [r.t_admit for r in sorted(out, key=lambda r: r.rid)]
    assert admits == sorted(admits)                     # FIFO: nobody overtakes the queue head


def test_host_hook_choice():
    assert choose_hook(*(lambda g: (g.row_ptr, g.col))(gen.er_csr(1000, 2000, seed=1))) == "plain"  # small, sparse
    grid = gen.grid_csr(600, 0.9, seed=1)
    assert choose_hook(grid.row_ptr, grid.col) == "tiled"
    rm = gen.rmat_csr(18, 8, seed=1)
    assert choose_hook(rm.row_ptr, rm.col) == "filtered"
    assert choose_hook(rm.row_ptr, rm.col, symmetric=False) == "plain"
    er = gen.er_csr(1 << 18, 1 << 21, seed=2)                      # mean degree 16
    assert choose_hook(er.row_ptr, er.col) == "filtered"
    assert choose_hook(er.row_ptr, er.col, symmetric=False) == "plain"
    sparse = gen.er_csr(1 << 18, 1 << 19, seed=3)                  # mean degree 4
    assert choose_hook(sparse.row_ptr, sparse.col) == "plain"
    small = gen.er_csr(20_000, 200_000, seed=4)                     # small, mean degree 20
    assert choose_hook(small.row_ptr, small.col) == "filtered"
