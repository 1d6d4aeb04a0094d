"""The thread-block-cluster kernel (CC_MODE_CLUSTER: pi in the distributed shared memory of one
cluster) through the C ABI: bit-exact against the oracle on the small-graph cases, both hooks it
runs (the filtered hook with CC_FLAG_SYMMETRIC, every arc without), every part size up to the
largest graph one cluster holds, and its error paths."""
import numpy as np
import pytest

import gen
import oracle
from graphs import clique_edges, directed_csr, path_edges, symmetric_csr

torch = pytest.importorskip("torch")
import paper_1612_01178_gb300 as ccl  # noqa: E402
from paper_1612_01178_gb300 import cc as ccapi  # noqa: E402

from test_cc_gpu import assert_labels, expect, union_of_all_small_graphs  # noqa: E402

pytestmark = pytest.mark.gpu


def cluster_csr(row_ptr, col, sym, mode=ccapi.CC_MODE_CLUSTER, expect_status=0, **opts):
    dev = torch.device("cuda:0")
    flags = ccl.CC_FLAG_SYNC | (ccl.CC_FLAG_SYMMETRIC if sym else 0)
    with ccl.ConnectedComponents(0, mode=mode, flags=flags, **opts) as cc:
        rp = torch.from_numpy(np.ascontiguousarray(row_ptr)).to(dev)
        cl = torch.from_numpy(np.ascontiguousarray(col, np.int32)).to(dev)
        if expect_status:
            with pytest.raises(ccl.CCError) as ei:
                cc.csr(rp, cl)
            assert ei.value.status == expect_status
            return None, None
        out = cc.csr(rp, cl)
        return out.cpu().numpy(), cc.run_info()


def test_union_of_all_small_graphs_and_multigraphs():
    V, s, d = union_of_all_small_graphs()
    for sym in (False, True):
        rp, col = symmetric_csr(V, s, d, np.int32)
        got, info = cluster_csr(rp, col, sym)
        assert_labels(got, expect(rp, col), f"sym={sym}")
        assert info["mode"] == ccapi.CC_MODE_CLUSTER
    rp, col = directed_csr(V, d, s, np.int64)
    assert_labels(cluster_csr(rp, col, False)[0], expect(rp, col), "directed, int64 offsets")
    rng = np.random.default_rng(5)
    for _ in range(30):
        n = int(rng.integers(1, 300))
        m = int(rng.integers(0, 5 * n))
        rp, col = symmetric_csr(n, rng.integers(0, n, m), rng.integers(0, n, m), np.int32)
        for sym in (False, True):
            assert_labels(cluster_csr(rp, col, sym)[0], expect(rp, col), f"n={n} m={m} sym={sym}")


@pytest.mark.parametrize("V", [2, 3, 1000, 32768, 65537, 131072, 262144])
def test_every_part_size(V):
    rng = np.random.default_rng(V)
    g = gen.er_csr(V, 3 * V, seed=V)
    for sym in (False, True):
        assert_labels(cluster_csr(g.row_ptr, g.col, sym)[0], expect(g.row_ptr, g.col), f"V={V} sym={sym}")
    rm = gen.rmat_csr(int(np.log2(max(4, V))), 8, seed=int(rng.integers(1 << 30)))
    assert_labels(cluster_csr(rm.row_ptr, rm.col, True)[0], expect(rm.row_ptr, rm.col), f"rmat V={rm.n_vertices}")


def test_er_100k_1m_and_automatic_choice():
    g = gen.workload_er_100k(1)
    want = expect(g.row_ptr, g.col)
    for sym in (False, True):
        got, info = cluster_csr(g.row_ptr, g.col, sym)
        assert_labels(got, want, f"sym={sym}")
    got, info = cluster_csr(g.row_ptr, g.col, True, mode=ccapi.CC_MODE_AUTO)
    assert_labels(got, want, "automatic")
    assert info["mode"] != ccapi.CC_MODE_CLUSTER  # off unless cluster_max_vertices enables it
    got, info = cluster_csr(g.row_ptr, g.col, True, mode=ccapi.CC_MODE_AUTO, cluster_max_vertices=1 << 18)
    assert_labels(got, want, "automatic, enabled")
    assert info["mode"] == ccapi.CC_MODE_CLUSTER


def test_adversarial_shapes():
    n = 200_000
    rng = np.random.default_rng(8)
    cases = [("descending_path", n, *path_edges(range(n - 1, -1, -1))),
             ("random_path", n, *path_edges(rng.permutation(n))),
             ("star_hub_high", 150_001, np.full(150_000, 150_000), np.arange(150_000)),
             ("star_hub_zero", 150_001, np.zeros(150_000, np.int64), np.arange(1, 150_001)),
             ("clique", 400, *clique_edges(range(0, 400, 2))),
             ("grid", 250_000, *gen_grid(500))]
    for name, V, s, d in cases:
        rp, col = symmetric_csr(V, s, d, np.int32)
        want = expect(rp, col)
        for sym in (False, True):
            assert_labels(cluster_csr(rp, col, sym)[0], want, f"{name} sym={sym}")


def gen_grid(side):
    g = gen.grid_csr(side, 0.85, seed=side)
    src = np.repeat(np.arange(g.n_vertices), np.diff(g.row_ptr))
    keep = src < g.col
    return src[keep], g.col[keep].astype(np.int64)


def test_errors():
    rp = np.array([0, 2, 3, 4], np.int32)
    col = np.array([1, 7, 0, 1], np.int32)  # 7 >= V = 3
    cluster_csr(rp, col, False, expect_status=ccapi.CC_ERR_OUT_OF_RANGE)
    cluster_csr(rp, col, True, expect_status=ccapi.CC_ERR_OUT_OF_RANGE)
    big = np.zeros((1 << 20) + 1, np.int32)  # more vertices than one cluster holds
    cluster_csr(big, np.zeros(0, np.int32), False, expect_status=ccapi.CC_ERR_INVALID_ARG)
    # the context still works after an input error (malformed input is not fatal)
    dev = torch.device("cuda:0")
    with ccl.ConnectedComponents(0, mode=ccapi.CC_MODE_CLUSTER) as cc:
        cc.csr(torch.from_numpy(rp).to(dev), torch.from_numpy(col).to(dev))
        with pytest.raises(ccl.CCError):
            cc.sync()
        ok = cc.csr(torch.tensor([0, 1, 2, 2], dtype=torch.int32, device=dev), torch.tensor([1, 0], dtype=torch.int32, device=dev))
        cc.sync()
        assert list(ok.cpu().numpy()) == [0, 0, 2]
