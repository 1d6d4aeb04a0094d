"""Serving loop on the GPU: every request's labels are the same when it is served alone and
when it is served in a mix of concurrent arrivals (continuous batching over two lanes), and equal
the oracle's; a malformed request and requests whose admission fails are rejected alone."""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
import paper_1612_01178_gb300 as ccl  # noqa: E402
from paper_1612_01178_gb300 import cc as ccapi  # noqa: E402
from paper_1612_01178_gb300.serve import Request, Server, latency_summary  # noqa: E402

pytestmark = pytest.mark.gpu


def pool(n, seed):
    rng = np.random.default_rng(seed)
    graphs = []
    for i in range(n):
        E = gen.loguniform_int(rng, 1e3, 3e5)
        if rng.random() < 0.5:
            d = int(rng.integers(4, 33))
            g = gen.er_csr(max(2, 2 * E // d), E, seed=100 + i)
        else:
            scale = max(4, int(round(np.log2(max(16, E / 8)))))
            g = gen.rmat_csr(scale, 8, seed=100 + i)
        graphs.append(g)
    graphs.append(gen.grid_csr(300, 0.9, seed=99))  # local numbering: multi-window path
    graphs.append(gen.rmat_csr(18, 8, seed=98))     # large enough for the filtered single-graph hook
    graphs.append(gen.grid_csr(600, 0.9, seed=97))  # large enough for the two-phase single-graph hook
    graphs.append(gen.CSR(1, np.array([0, 0], np.int32), np.zeros(0, np.int32), 0, "single"))
    return graphs


def make_requests(graphs, arrivals):
    return [Request(i, float(t), g.row_ptr, g.col) for i, (g, t) in enumerate(zip(graphs, arrivals))]


@pytest.mark.parametrize("lanes", [1, 2])
def test_alone_equals_in_the_mix(lanes):
    assert torch.cuda.is_available()
    graphs = pool(24, seed=3)
    want = [oracle.labels_uf_csr(g.row_ptr, g.col)[0] for g in graphs]
    srv = Server(0, label_elems=1 << 21, row_elems=1 << 21, arc_elems=1 << 23, max_batch=8, lanes=lanes)
    try:
        alone = []
        for i, g in enumerate(graphs):
            r = srv.run(make_requests([g], [0.0]))[0]
            assert r.status == 0
            alone.append(r.labels.copy())
            assert np.array_equal(alone[-1], want[i]), i
        # a burst and a Poisson stream: requests arrive while others are on the GPU
        rng = np.random.default_rng(1)
        for arrivals in (np.zeros(len(graphs)), np.cumsum(rng.exponential(1 / 2000.0, len(graphs)))):
            order = rng.permutation(len(graphs))
            reqs = make_requests([graphs[i] for i in order], arrivals)
            out = srv.run(reqs)
            for r, i in zip(out, order):
                assert r.status == 0
                assert np.array_equal(r.labels, alone[i]), f"request {r.rid} (graph {i}) differs in the mix"
            s = latency_summary(out)
            assert s["p99_ms"] >= s["p50_ms"] > 0
        assert max(n for n, _, _ in srv.batches) > 1  # requests really were batched together
        assert len({lane for _, _, lane in srv.batches}) == lanes
        assert srv.arena["label"].used == 0 and srv.arena["arc"].used == 0
    finally:
        srv.close()


def test_admission_waits_for_memory():
    """Arenas that hold only a few requests at a time: later arrivals wait for memory to free up."""
    graphs = [gen.er_csr(20_000, 60_000, seed=i) for i in range(12)]
    want = [oracle.labels_uf_csr(g.row_ptr, g.col)[0] for g in graphs]
    srv = Server(0, label_elems=50_000, row_elems=50_000, arc_elems=300_000, max_batch=16)
    try:
        out = srv.run(make_requests(graphs, np.zeros(len(graphs))))
        for r in out:
            assert np.array_equal(r.labels, want[r.rid])
        assert max(n for n, _, _ in srv.batches) <= 2  # at most two requests fit at once
        r = srv.run(make_requests([gen.er_csr(60_000, 10, seed=1)], [0.0]))[0]  # larger than the arenas
        assert r.status == ccapi.CC_ERR_OOM and r.labels is None
    finally:
        srv.close()


def test_bad_requests_fail_alone_in_a_poisson_mix():
    """One malformed request (an endpoint outside [0, V)) and two whose admission fails (injected
    on the host) in a Poisson stream: those three come back with their error, every other request
    equals the oracle, in the same batch and in later ones."""
    graphs = pool(30, seed=5)
    bad_id = 7
    g = graphs[bad_id]
    col = g.col.copy()
    col[int(g.row_ptr[np.flatnonzero(np.diff(g.row_ptr))[0]])] = g.n_vertices + 11
    graphs[bad_id] = gen.CSR(g.n_vertices, g.row_ptr, col, g.n_edges, "bad")
    victims = {3, 20}

    def inject(stage, req):
        if stage == "admit" and req.rid in victims:
            raise MemoryError("injected allocation failure")

    want = {i: oracle.labels_uf_csr(h.row_ptr, h.col)[0] for i, h in enumerate(graphs) if i != bad_id}
    srv = Server(0, label_elems=1 << 21, row_elems=1 << 21, arc_elems=1 << 23, max_batch=8, inject=inject)
    try:
        rng = np.random.default_rng(2)
        for arrivals in (np.zeros(len(graphs)), np.cumsum(rng.exponential(1 / 3000.0, len(graphs)))):
            out = srv.run(make_requests(graphs, arrivals))
            for r in out:
                if r.rid == bad_id:
                    assert r.status == ccapi.CC_ERR_OUT_OF_RANGE
                elif r.rid in victims:
                    assert r.status == ccapi.CC_ERR_OOM and "injected" in r.error
                else:
                    assert r.status == 0, (r.rid, r.status)
                    assert np.array_equal(r.labels, want[r.rid]), f"request {r.rid} differs"
        assert all(a.used == 0 for a in srv.arena.values())
    finally:
        srv.close()


def test_large_request():
    """A request of 5 * 10^6 edges (the top of the serving mix's size range is 2 * 10^7) with small
    ones around it."""
    big = gen.rmat_csr(20, 5, seed=31)  # 2^20 vertices, 5.2M drawn edges
    small = [gen.er_csr(5000, 20_000, seed=40 + i) for i in range(6)]
    graphs = small[:3] + [big] + small[3:]
    want = [oracle.labels_uf_csr(h.row_ptr, h.col)[0] for h in graphs]
    srv = Server(0, label_elems=1 << 22, row_elems=1 << 22, arc_elems=1 << 25, max_batch=8)
    try:
        out = srv.run(make_requests(graphs, np.linspace(0, 0.001, len(graphs))))
        for r in out:
            assert r.status == 0
            assert np.array_equal(r.labels, want[r.rid]), r.rid
    finally:
        srv.close()
