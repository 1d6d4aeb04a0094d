"""Batched labelling (cc_labels_batched) through the C ABI: every graph's labels must equal
the oracle's for that graph alone (bit-exact), and the single-graph entry point run graph by
graph must give the same answer."""
import numpy as np
import pytest

import gen
import oracle
from graphs import path_edges, symmetric_csr

torch = pytest.importorskip("torch")
import paper_1612_01178_gb300 as ccl  # noqa: E402
from paper_1612_01178_gb300 import cc as ccapi  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    ccl.load()
    return torch.device("cuda:0")


def to_dev(dev, b):
    return (torch.from_numpy(b.v_off).to(dev), torch.from_numpy(b.a_off).to(dev),
            torch.from_numpy(b.row_ptr_cat).to(dev), torch.from_numpy(b.col_cat).to(dev))


def run_batched(dev, b, status=False, **opts):
    o = dict(flags=ccl.CC_FLAG_SYNC)
    o.update(opts)
    with ccl.ConnectedComponents(0, **o) as cc:
        v_off, a_off, rp, col = to_dev(dev, b)
        st = torch.full((b.n_graphs,), -7, dtype=torch.int32, device=dev) if status else None
        out = cc.batched(v_off, a_off, rp, col, graph_status=st)
        torch.cuda.synchronize()
        return out.cpu().numpy(), (st.cpu().numpy() if status else None)


def expected(b):
    out = np.empty(b.total_vertices, np.int32)
    for g in range(b.n_graphs):
        rp, col = b.graph(g)
        v0, v1 = int(b.v_off[g]), int(b.v_off[g + 1])
        if v1 > v0:
            out[v0:v1] = oracle.labels_uf_csr(rp, col)[0]
    return out


def assert_batch(got, b, want=None, what=""):
    want = expected(b) if want is None else want
    if not np.array_equal(got, want):
        for g in range(b.n_graphs):
            v0, v1 = int(b.v_off[g]), int(b.v_off[g + 1])
            if not np.array_equal(got[v0:v1], want[v0:v1]):
                raise AssertionError(f"{what}: graph {g} ({b.kinds[g]}, V={v1 - v0}) differs")
    return want


def edge_case_graphs():
    """Empty graph, single vertex, edgeless graph, graphs at and across the window size."""
    gs = []
    gs.append(gen.CSR(0, np.zeros(1, np.int32), np.zeros(0, np.int32), 0, "empty"))
    gs.append(gen.CSR(1, np.array([0, 0], np.int32), np.zeros(0, np.int32), 0, "single"))
    gs.append(gen.CSR(50, np.zeros(51, np.int32), np.zeros(0, np.int32), 0, "edgeless"))
    rp, col = symmetric_csr(3, [2, 1], [1, 0], np.int32)
    gs.append(gen.CSR(3, rp, col, 2, "tiny_path"))
    for V in (256, 257, 1024, 1025):
        rp, col = symmetric_csr(V, *path_edges(range(V - 1, -1, -1)), np.int32)
        gs.append(gen.CSR(V, rp, col, V - 1, f"descending_path{V}"))
    return gs


@pytest.mark.parametrize("tile", [0, -1, 256, 1024])
@pytest.mark.parametrize("sym", [True, False])
def test_mixed_small_batch(dev, tile, sym):
    b = gen.workload_batched(120, seed=2, vmin=50, vmax=3e4)
    got, _ = run_batched(dev, b, tile_vertices=tile, flags=ccl.CC_FLAG_SYNC | (ccl.CC_FLAG_SYMMETRIC if sym else 0))
    assert_batch(got, b, what=f"tile={tile} sym={sym}")


@pytest.mark.parametrize("tile", [0, -1, 4096])
def test_batch_with_multi_window_graphs(dev, tile):
    graphs = edge_case_graphs()
    graphs.append(gen.grid_csr(600, 0.9, seed=5))       # local numbering: phase A windows
    graphs.append(gen.er_csr(150_000, 600_000, seed=6))  # random numbering: windows hooked arc by arc
    graphs.append(gen.rmat_csr(17, 8, seed=7))
    graphs.append(gen.grid_csr(300, 0.55, seed=8))
    graphs += edge_case_graphs()
    b = gen.batch_from_graphs(graphs)
    got, _ = run_batched(dev, b, tile_vertices=tile, flags=ccl.CC_FLAG_SYNC | ccl.CC_FLAG_SYMMETRIC)
    assert_batch(got, b, what=f"tile={tile}")
    for segments in (1, 3):
        got, _ = run_batched(dev, b, tile_vertices=tile, segments=segments,
                             flags=ccl.CC_FLAG_SYNC | ccl.CC_FLAG_SYMMETRIC)
        assert_batch(got, b, what=f"tile={tile} s={segments}")


def test_batch_equals_graph_by_graph(dev):
    b = gen.workload_batched(40, seed=9, vmin=1e3, vmax=2e5)
    got, _ = run_batched(dev, b, flags=ccl.CC_FLAG_SYNC | ccl.CC_FLAG_SYMMETRIC)
    want = assert_batch(got, b)
    # the single-graph entry point on each graph in place (pointers into the same arrays)
    v_off, a_off, rp, col = to_dev(dev, b)
    labels = torch.empty(b.total_vertices, dtype=torch.int32, device=dev)
    with ccl.ConnectedComponents(0, flags=ccl.CC_FLAG_SYMMETRIC) as cc:
        for g in range(b.n_graphs):
            v0, v1, a0, a1 = int(b.v_off[g]), int(b.v_off[g + 1]), int(b.a_off[g]), int(b.a_off[g + 1])
            cc.csr(rp[v0 + g: v1 + g + 1], col[a0:a1], labels[v0:v1])
        cc.sync()
    assert np.array_equal(labels.cpu().numpy(), want)


def test_batch_repeat_and_phase_times(dev):
    b = gen.workload_batched(60, seed=4, vmin=1e3, vmax=1e5)
    want = expected(b)
    with ccl.ConnectedComponents(0, flags=ccl.CC_FLAG_SYMMETRIC | ccapi.CC_FLAG_PHASE_TIMES) as cc:
        v_off, a_off, rp, col = to_dev(dev, b)
        out = torch.empty(b.total_vertices, dtype=torch.int32, device=dev)
        for _ in range(5):
            cc.batched(v_off, a_off, rp, col, out)
            cc.sync()
            assert np.array_equal(out.cpu().numpy(), want)
        assert len(cc.phase_times()) >= 3


def test_per_graph_status(dev):
    graphs = [gen.er_csr(500, 1000, seed=1), gen.er_csr(400, 800, seed=2), gen.grid_csr(300, 0.9, seed=3)]
    bad = graphs[1]
    col = bad.col.copy()
    col[7] = 400  # endpoint outside graph 1's [0, 400)
    graphs[1] = gen.CSR(bad.n_vertices, bad.row_ptr, col, bad.n_edges, "bad")
    b = gen.batch_from_graphs(graphs)
    with ccl.ConnectedComponents(0, flags=ccl.CC_FLAG_SYMMETRIC) as cc:
        v_off, a_off, rp, colt = to_dev(dev, b)
        st = torch.full((3,), -7, dtype=torch.int32, device=dev)
        out = cc.batched(v_off, a_off, rp, colt, graph_status=st)
        with pytest.raises(ccl.CCError) as ei:
            cc.sync()
        assert ei.value.status == ccapi.CC_ERR_OUT_OF_RANGE
        assert list(st.cpu().numpy()) == [0, ccapi.CC_ERR_OUT_OF_RANGE, 0]
        # a malformed graph is reported but does not stop the launch: the other graphs are labelled
        got = out.cpu().numpy()
        for g in (0, 2):
            v0, v1 = int(b.v_off[g]), int(b.v_off[g + 1])
            grp, gcol = b.graph(g)
            assert np.array_equal(got[v0:v1], oracle.labels_uf_csr(grp, gcol)[0]), f"graph {g}"
        b2 = gen.batch_from_graphs([graphs[0], graphs[2]])
        v_off, a_off, rp, colt = to_dev(dev, b2)
        out = cc.batched(v_off, a_off, rp, colt)
        cc.sync()
        assert_batch(out.cpu().numpy(), b2)


@pytest.mark.parametrize("n_good", [3, 600])
def test_bad_graphs_do_not_stop_the_batch(dev, n_good):
    """Malformed graphs (an endpoint outside [0, V_g), offsets past the graph's arcs) spread over a
    batch of windows of every kind: each is reported in graph_status and every other graph still
    equals the oracle, and the next call on the same context is unaffected."""
    rng = np.random.default_rng(40 + n_good)
    graphs, bad = [], set()
    for i in range(n_good):
        kind = i % 3
        if kind == 0:
            g = gen.er_csr(int(rng.integers(50, 3000)), int(rng.integers(50, 9000)), seed=1000 + i)
        elif kind == 1:
            g = gen.grid_csr(int(rng.integers(10, 250)), 0.9, seed=1000 + i)
        else:
            g = gen.rmat_csr(int(rng.integers(8, 16)), 8, seed=1000 + i)
        graphs.append(g)
    graphs.append(gen.grid_csr(700, 0.9, seed=7))   # several windows (phase A)
    graphs.append(gen.rmat_csr(17, 8, seed=8))      # several windows without locality
    for j in sorted(rng.choice(len(graphs), size=min(5, len(graphs)), replace=False).tolist()):
        g = graphs[j]
        if g.nnz == 0:
            continue
        col = g.col.copy()
        rp = g.row_ptr.copy()
        if j % 2 == 0:  # the first arc of a row: every hook variant reads it
            rows = np.flatnonzero(np.diff(g.row_ptr) > 0)
            col[int(g.row_ptr[int(rng.choice(rows))])] = g.n_vertices + int(rng.integers(0, 50))
        else:
            rp[g.n_vertices // 2 + 1:] = rp[g.n_vertices // 2 + 1:] + 3  # offsets past the arc range
            rp[-1] = g.nnz
        graphs[j] = gen.CSR(g.n_vertices, rp, col, g.n_edges, "bad")
        bad.add(j)
    b = gen.batch_from_graphs(graphs)
    good_want = {}
    for g in range(b.n_graphs):
        if g not in bad:
            grp, gcol = b.graph(g)
            good_want[g] = oracle.labels_uf_csr(grp, gcol)[0]
    with ccl.ConnectedComponents(0, flags=ccl.CC_FLAG_SYMMETRIC) as cc:
        v_off, a_off, rp, colt = to_dev(dev, b)
        st = torch.full((b.n_graphs,), -7, dtype=torch.int32, device=dev)
        out = cc.batched(v_off, a_off, rp, colt, graph_status=st)
        assert cc.sync(raise_input_errors=False) == ccapi.CC_ERR_OUT_OF_RANGE
        status = st.cpu().numpy()
        got = out.cpu().numpy()
        for g in range(b.n_graphs):
            if g in bad:
                continue
            assert status[g] == 0, f"graph {g} flagged"
            v0, v1 = int(b.v_off[g]), int(b.v_off[g + 1])
            assert np.array_equal(got[v0:v1], good_want[g]), f"graph {g} ({b.kinds[g]}) differs"
        # bad offsets that stay inside the graph's own arc range may go unnoticed (its labels are
        # unspecified); an endpoint out of range in the first arc of a row is always seen
        for j in bad:
            if j % 2 == 0:
                assert status[j] == ccapi.CC_ERR_OUT_OF_RANGE, f"bad graph {j} not flagged"
        # the next call on the same context: the good graphs alone, nothing left over
        good = [graphs[g] for g in range(len(graphs)) if g not in bad]
        b2 = gen.batch_from_graphs(good)
        v_off, a_off, rp, colt = to_dev(dev, b2)
        out2 = cc.batched(v_off, a_off, rp, colt)
        assert cc.sync() == ccapi.CC_OK
        assert_batch(out2.cpu().numpy(), b2, what="after a batch with bad graphs")


def test_batched_argument_errors(dev):
    lib = ccapi.load()
    with ccl.ConnectedComponents(0) as cc:
        x = torch.zeros(8, dtype=torch.int64, device=dev)
        assert lib.cc_labels_batched(cc.handle, -1, 0, 0, None, None, None, None, None, None) == \
            ccapi.CC_ERR_INVALID_ARG
        assert lib.cc_labels_batched(cc.handle, 2, 10, 0, None, x.data_ptr(), x.data_ptr(), None, x.data_ptr(),
                                     None) == ccapi.CC_ERR_INVALID_ARG
        assert lib.cc_labels_batched(cc.handle, 1, 1 << 31, 0, x.data_ptr(), x.data_ptr(), x.data_ptr(), None,
                                     x.data_ptr(), None) == ccapi.CC_ERR_INVALID_ARG


def test_graph_mixing_local_and_random_windows(dev):
    """One graph whose first half is a grid (windows with locality: phase A, which leaves arcs
    with v < u to their reverse arcs) and whose second half is random (windows hooked arc by arc),
    joined by a few edges, in a batch with more windows than CTAs: the filter must not skip rows
    of such a graph. Also the random half alone (every window without locality: filtered)."""
    side = 200
    grid = gen.grid_csr(side, 0.9, seed=21)
    n_grid = side * side
    er = gen.er_csr(40_000, 160_000, seed=22)
    src = [np.repeat(np.arange(n_grid), np.diff(grid.row_ptr)), n_grid + np.repeat(np.arange(40_000), np.diff(er.row_ptr))]
    dst = [grid.col.astype(np.int64), n_grid + er.col.astype(np.int64)]
    links = np.random.default_rng(23).integers(0, n_grid, 50)
    src.append(links)
    dst.append(n_grid + links % 40_000)
    s = np.concatenate(src)
    d = np.concatenate(dst)
    rp, col = symmetric_csr(n_grid + 40_000, s, d, np.int32)
    mixed = gen.CSR(n_grid + 40_000, rp, col, len(col) // 2, "grid+er")
    b = gen.batch_from_graphs([mixed, er] + edge_case_graphs())
    for tile in (256, 1024):
        got, _ = run_batched(dev, b, tile_vertices=tile, flags=ccl.CC_FLAG_SYNC | ccl.CC_FLAG_SYMMETRIC)
        assert_batch(got, b, what=f"mixed windows tile={tile}")


def test_million_vertex_graphs_among_small_ones(dev):
    """The batched workload draws graphs of up to 10^6 vertices: a 1000 x 1000 grid (windows with
    locality) and an R-MAT graph of 2^20 vertices (windows without) among a few hundred small ones,
    every graph checked against the oracle, symmetric and not."""
    rng = np.random.default_rng(61)
    graphs = [gen.grid_csr(1000, 0.9, seed=62), gen.rmat_csr(20, 8, seed=63)]
    for i in range(300):
        V = int(rng.integers(1000, 40_000))
        graphs.append(gen.er_csr(V, int(V * rng.integers(2, 16)), seed=700 + i) if i % 2 else
                      gen.grid_csr(int(np.sqrt(V)), 0.9, seed=700 + i))
    order = rng.permutation(len(graphs))
    b = gen.batch_from_graphs([graphs[i] for i in order])
    want = expected(b)
    for flags in (ccl.CC_FLAG_SYNC | ccl.CC_FLAG_SYMMETRIC, ccl.CC_FLAG_SYNC):
        got, st = run_batched(dev, b, status=True, flags=flags)
        assert (st == 0).all()
        assert_batch(got, b, want, what=f"flags={flags}")


def test_window_boundary_sizes_with_many_windows(dev):
    """Graphs of W - 1, W, W + 1, W + 232, 2W - 1 and 2W + 1 vertices (W = 32768, the batch window) of
    both families, in a batch with more windows than CTAs, so each multi-window graph takes one hook
    for all its windows from its locality sample (phase A for the grids, the sampled-and-filtered hook
    for the ER graphs); every graph against the oracle, symmetric and not."""
    W = 32768
    graphs = []
    for i, V in enumerate((W - 1, W, W + 1, W + 232, 2 * W - 1, 2 * W + 1)):
        graphs.append(gen.er_csr(V, 6 * V, seed=800 + i))
        side = int(np.ceil(np.sqrt(V)))
        graphs.append(gen.grid_csr(side, 0.9, seed=820 + i))
    for i in range(100):  # filler: 200 windows of ER graphs, so the batch has more windows than CTAs
        graphs.append(gen.er_csr(40_000, 40_000 * (2 + i % 8), seed=840 + i))
    order = np.random.default_rng(71).permutation(len(graphs))
    b = gen.batch_from_graphs([graphs[i] for i in order])
    want = expected(b)
    for flags in (ccl.CC_FLAG_SYNC | ccl.CC_FLAG_SYMMETRIC, ccl.CC_FLAG_SYNC):
        got, st = run_batched(dev, b, status=True, flags=flags)
        assert (st == 0).all()
        assert_batch(got, b, want, what=f"boundary sizes flags={flags}")


def test_batched_reports_two_launches(dev):
    """A batched labelling is two launches (phase A with the window in shared memory, then the
    rest), and the run info says so."""
    b = gen.batch_from_graphs([gen.er_csr(5000, 20_000, seed=91), gen.grid_csr(100, 0.9, seed=92)])
    with ccl.ConnectedComponents(0, flags=ccl.CC_FLAG_SYNC | ccl.CC_FLAG_SYMMETRIC) as cc:
        v_off, a_off, rp, col = to_dev(dev, b)
        out = cc.batched(v_off, a_off, rp, col)
        info = cc.run_info()
    assert info["launches"] == 2, info
    assert_batch(out.cpu().numpy(), b, what="two launches")
