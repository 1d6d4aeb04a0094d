"""The allocation-free entry point (cc_labels_csr_noalloc) must give the oracle's labels, and
the same labels as the regular entry point (cc_labels_csr), on calls in a row.

It serves callers that cannot allocate device memory (code inside a device memory
allocator or pool, plug-ins whose host owns all device memory, real-time paths that
must not allocate). Its scratch is a static array inside the library that every call
shares and that keeps the previous call's contents: the calls in a row check that the
leftover barrier count, work counters and status of one call do not leak into the next,
including a call that ends with an error (an arc endpoint outside [0, V)), whose sticky
error word must not be seen by the valid call after it.
The file is named to be collected last."""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
import paper_1612_01178_gb300 as ccl  # noqa: E402
from paper_1612_01178_gb300 import cc as ccapi  # noqa: E402

pytestmark = pytest.mark.gpu


def regular_labels(dev, g, sym):
    flags = ccl.CC_FLAG_SYNC | (ccl.CC_FLAG_SYMMETRIC if sym else 0)
    with ccl.ConnectedComponents(0, flags=flags) as cc:
        out = cc.csr(torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev))
        return out.cpu().numpy()


def test_noalloc_matches_oracle_and_regular_entry_point_on_calls_in_a_row():
    assert torch.cuda.is_available(), "needs a CUDA device"
    dev = torch.device("cuda:0")
    graphs = [(gen.grid_csr(1500, 0.8, seed=4), True), (gen.rmat_csr(18, 8, seed=6, offsets64=True), False),
              (gen.er_csr(100_000, 1_000_000, seed=3), True)]
    oracle_labels = [oracle.labels_uf_csr(g.row_ptr, g.col)[0] for g, _ in graphs]
    regular = [regular_labels(dev, g, sym) for g, sym in graphs]
    for want, reg in zip(oracle_labels, regular):
        assert np.array_equal(reg, want)
    stream = torch.cuda.Stream(device=dev)
    inputs = []
    for g, sym in graphs:  # device buffers allocated up front by the caller
        rp = torch.from_numpy(g.row_ptr).to(dev)
        col = torch.from_numpy(g.col).to(dev)
        lab = torch.full((g.n_vertices,), -1, dtype=torch.int32, device=dev)
        inputs.append((rp, col, lab, sym))
    torch.cuda.synchronize()
    for _ in range(2):
        for (rp, col, lab, sym), want in zip(inputs, oracle_labels):
            lab.fill_(-1)
            ccapi.cc_labels_csr_noalloc(rp, col, lab, stream=stream, symmetric=sym)
            got = lab.cpu().numpy()
            assert np.array_equal(got, want), f"{(got != want).sum()} labels differ from the oracle"


def test_noalloc_error_does_not_leak_into_the_next_call():
    dev = torch.device("cuda:0")
    g = gen.er_csr(20_000, 60_000, seed=9)
    want = oracle.labels_uf_csr(g.row_ptr, g.col)[0]
    bad_col = g.col.copy()
    bad_col[len(bad_col) // 2] = g.n_vertices + 5  # an endpoint outside [0, V): the hook reports it
    rp = torch.from_numpy(g.row_ptr).to(dev)
    col_bad = torch.from_numpy(bad_col).to(dev)
    col_ok = torch.from_numpy(g.col).to(dev)
    lab = torch.empty(g.n_vertices, dtype=torch.int32, device=dev)
    with pytest.raises(ccl.CCError) as ei:
        ccapi.cc_labels_csr_noalloc(rp, col_bad, lab)
    assert ei.value.status == ccapi.CC_ERR_OUT_OF_RANGE
    ccapi.cc_labels_csr_noalloc(rp, col_ok, lab)
    assert np.array_equal(lab.cpu().numpy(), want)


def test_noalloc_rejects_a_capturing_stream():
    dev = torch.device("cuda:0")
    g = gen.er_csr(1000, 3000, seed=2)
    rp = torch.from_numpy(g.row_ptr).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    lab = torch.empty(g.n_vertices, dtype=torch.int32, device=dev)
    want = oracle.labels_uf_csr(g.row_ptr, g.col)[0]
    ccapi.cc_labels_csr_noalloc(rp, col, lab)  # the per-device set-up happens outside the capture
    assert np.array_equal(lab.cpu().numpy(), want)
    s = torch.cuda.Stream(device=dev)
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        graph.capture_begin()
        try:
            st = ccapi.load().cc_labels_csr_noalloc(g.n_vertices, g.nnz, rp.data_ptr(), ccapi.CC_INDEX_I32,
                                                    col.data_ptr(), lab.data_ptr(), s.cuda_stream, 0)
        finally:
            graph.capture_end()  # the capture must still be valid (nothing was issued on it)
    assert st == ccapi.CC_ERR_INVALID_ARG
    lab.fill_(-1)
    ccapi.cc_labels_csr_noalloc(rp, col, lab)  # and the entry point still works afterwards
    assert np.array_equal(lab.cpu().numpy(), want)


def test_noalloc_rejects_bad_arguments():
    lib = ccapi.load()
    assert lib.cc_labels_csr_noalloc(-1, 0, None, 4, None, None, None, 0) == ccapi.CC_ERR_INVALID_ARG
    assert lib.cc_labels_csr_noalloc(4, 1 << 31, 1, 4, 1, 1, None, 0) == ccapi.CC_ERR_INVALID_ARG
    assert lib.cc_labels_csr_noalloc(4, 8, 1, 4, 1, 1, None, ccl.CC_FLAG_SYNC) == ccapi.CC_ERR_INVALID_ARG
