"""Autotuner on the GPU: every candidate gives the oracle's labels, and the tuned options do too."""
import numpy as np
import pytest

import gen
import oracle

torch = pytest.importorskip("torch")
import paper_1612_01178_gb300 as ccl  # noqa: E402
from paper_1612_01178_gb300.tune import Tuner  # noqa: E402

pytestmark = pytest.mark.gpu


def test_tune_csr_and_batched(tmp_path):
    assert torch.cuda.is_available()
    dev = torch.device("cuda:0")
    t = Tuner(str(tmp_path / "tune.json"))
    for g in (gen.grid_csr(700, 0.9, seed=2), gen.er_csr(200_000, 800_000, seed=3)):
        rp = torch.from_numpy(g.row_ptr).to(dev)
        col = torch.from_numpy(g.col).to(dev)
        best = t.tune_csr(rp, col, reps=2)
        with ccl.ConnectedComponents(0, flags=ccl.CC_FLAG_SYMMETRIC | ccl.CC_FLAG_SYNC, **best) as cc:
            got = cc.csr(rp, col).cpu().numpy()
        assert np.array_equal(got, oracle.labels_uf_csr(g.row_ptr, g.col)[0])
    b = gen.workload_batched(24, seed=5, vmin=200, vmax=6e4)
    best = t.tune_batched(torch.from_numpy(b.v_off).to(dev), torch.from_numpy(b.a_off).to(dev),
                          torch.from_numpy(b.row_ptr_cat).to(dev), torch.from_numpy(b.col_cat).to(dev), reps=2)
    assert isinstance(best, dict)
    assert len(Tuner(str(tmp_path / "tune.json")).cache) == 3


def test_context_uses_the_tuned_options_of_the_bucket(tmp_path):
    """A context given the tuner runs every call with the tuned options of the graph's size bucket;
    tuned and default options give the oracle's labels."""
    dev = torch.device("cuda:0")
    t = Tuner(str(tmp_path / "tune.json"))
    g = gen.workload_er_100k(3)
    rp = torch.from_numpy(g.row_ptr).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    want = oracle.labels_uf_csr(g.row_ptr, g.col)[0]
    best = t.tune_csr(rp, col, reps=2)
    assert t.options_for_csr(g.n_vertices, g.nnz) == best
    with ccl.ConnectedComponents(0, flags=ccl.CC_FLAG_SYMMETRIC | ccl.CC_FLAG_SYNC, tuner=t) as cc:
        got = cc.csr(rp, col).cpu().numpy()
        assert cc.last_options_source == "tuner cache"
        assert np.array_equal(got, want)
        other = gen.grid_csr(300, 0.9, seed=4)  # a bucket without a tuned entry: the explicit options
        got2 = cc.csr(torch.from_numpy(other.row_ptr).to(dev), torch.from_numpy(other.col).to(dev)).cpu().numpy()
        assert cc.last_options_source == "explicit"
        assert np.array_equal(got2, oracle.labels_uf_csr(other.row_ptr, other.col)[0])
    with ccl.ConnectedComponents(0, flags=ccl.CC_FLAG_SYMMETRIC | ccl.CC_FLAG_SYNC) as cc:
        assert np.array_equal(cc.csr(rp, col).cpu().numpy(), want)
