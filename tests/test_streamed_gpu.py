"""Graphs larger than device memory (Section III-B: the segments bound the resident working set
to the |V|-sized parent array): cc_labels_csr_host with the arcs left in host memory and streamed
in segments of stream_arcs arcs through two device buffers. Forced on graphs that do fit, with
small segments, the labels must equal the oracle's bit for bit."""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
import paper_1612_01178_gb300 as ccl  # noqa: E402
from paper_1612_01178_gb300 import cc as ccapi  # noqa: E402

pytestmark = pytest.mark.gpu


def pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


def streamed(g, seg, sym=True, **opts):
    flags = ccl.CC_FLAG_SYMMETRIC if sym else 0
    with ccl.ConnectedComponents(0, flags=flags, stream_arcs=seg, **opts) as cc:
        out = pinned(np.full(g.n_vertices, -1, np.int32))
        cc.csr_host(pinned(g.row_ptr), pinned(g.col), out)
        return out.copy(), cc.run_info()


@pytest.mark.parametrize("seg", [100_000, 12_345, 1 << 20])
def test_er_streamed_segments(seg):
    g = gen.workload_er_100k(1)
    got, info = streamed(g, seg)
    assert np.array_equal(got, oracle.labels_uf_csr(g.row_ptr, g.col)[0])
    assert info["streamed_segments"] == -(-g.nnz // seg)


def test_grid_and_rmat_streamed():
    grid = gen.grid_csr(1000, 0.9, seed=5)
    got, info = streamed(grid, 54_321)
    assert np.array_equal(got, oracle.labels_uf_csr(grid.row_ptr, grid.col)[0])
    assert info["streamed_segments"] > 50
    rm = gen.rmat_csr(20, 16, seed=3, offsets64=True)
    for sym in (True, False):
        got, info = streamed(rm, 1 << 21, sym=sym)
        assert np.array_equal(got, oracle.labels_uf_csr(rm.row_ptr, rm.col)[0]), sym
        assert info["streamed_segments"] == 16


def test_streaming_off_when_the_segment_covers_the_graph():
    g = gen.er_csr(5000, 20_000, seed=2)
    got, info = streamed(g, g.nnz)
    assert np.array_equal(got, oracle.labels_uf_csr(g.row_ptr, g.col)[0])
    assert info["streamed_segments"] == 0


def test_streamed_out_of_range_endpoint_and_reuse():
    g = gen.er_csr(50_000, 200_000, seed=4)
    col = g.col.copy()
    col[len(col) // 2 + 7] = g.n_vertices + 1
    with ccl.ConnectedComponents(0, flags=ccl.CC_FLAG_SYMMETRIC, stream_arcs=30_000) as cc:
        out = pinned(np.zeros(g.n_vertices, np.int32))
        with pytest.raises(ccl.CCError) as ei:
            cc.csr_host(pinned(g.row_ptr), pinned(col), out)
        assert ei.value.status == ccapi.CC_ERR_OUT_OF_RANGE
        cc.csr_host(pinned(g.row_ptr), pinned(g.col), out)  # the same context afterwards
        assert np.array_equal(out, oracle.labels_uf_csr(g.row_ptr, g.col)[0])


def test_graphs_that_fit_are_not_streamed_by_default():
    """With the default options a graph that fits on the device is copied whole (no streaming), and
    stream_arcs = -1 never streams; both give the oracle's labels."""
    g = gen.rmat_csr(23, 16, seed=2, offsets64=True)  # 2^28 arcs
    want = oracle.labels_uf_csr(g.row_ptr, g.col)[0]
    prp, pcol = pinned(g.row_ptr), pinned(g.col)
    for seg in (0, -1):
        with ccl.ConnectedComponents(0, flags=ccl.CC_FLAG_SYMMETRIC, stream_arcs=seg) as cc:
            out = pinned(np.full(g.n_vertices, -1, np.int32))
            cc.csr_host(prp, pcol, out)
            assert cc.run_info()["streamed_segments"] == 0
        assert np.array_equal(out, want), seg
