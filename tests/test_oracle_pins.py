"""Pins for the CPU oracle: it must equal the Section II definition of connected
components (min-ID representative) on inputs whose answer is fixed independently of
the oracle: brute force, hand-derived fixtures, closed forms, SciPy, invariants."""
import itertools
import os

import numpy as np
import pytest

import gen
import oracle
from graphs import (check_min_label_invariants, clique_edges, closure_labels, directed_csr, grid_edges,
                    min_id_from_component_ids, path_edges, symmetric_csr)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "handworked_labels.txt")


def all_oracles(V, src, dst, lib=None):
    """Every oracle entry point on every input form of one undirected edge list."""
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    out = {}
    out["uf_coo"] = oracle.labels_uf_coo(V, src, dst, lib)
    out["bfs_coo"] = oracle.labels_bfs_coo(V, src, dst, lib)
    rp, col = symmetric_csr(V, src, dst)
    out["uf_csr_sym"] = oracle.labels_uf_csr(rp, col, lib)
    out["bfs_csr_sym"] = oracle.labels_bfs_csr(rp, col, lib)
    rp, col = directed_csr(V, src, dst)  # one direction only: still undirected edges
    out["uf_csr_dir"] = oracle.labels_uf_csr(rp, col, lib)
    out["bfs_csr_dir"] = oracle.labels_bfs_csr(rp, col, lib)
    rp, col = directed_csr(V, dst, src)
    out["uf_csr_rev"] = oracle.labels_uf_csr(rp, col, lib)
    out["bfs_csr_rev"] = oracle.labels_bfs_csr(rp, col, lib)
    return out


def assert_all_equal(V, src, dst, expected, lib=None):
    expected = np.asarray(expected, np.int32)
    n_comp = int((expected == np.arange(V)).sum())
    for name, (lab, n) in all_oracles(V, src, dst, lib).items():
        assert np.array_equal(lab, expected), (name, lab, expected)
        assert n == n_comp, (name, n, n_comp)


def load_golden():
    cases, cur = [], {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, rest = line.partition(" ")
            if key == "graph":
                cur = {"name": rest}
                cases.append(cur)
            elif key == "V":
                cur["V"] = int(rest)
            elif key == "edges":
                pairs = [tuple(map(int, e.split("-"))) for e in rest.split()]
                cur["src"] = [p[0] for p in pairs]
                cur["dst"] = [p[1] for p in pairs]
            elif key == "labels":
                cur["labels"] = [int(x) for x in rest.split()]
    return cases


def pins(lib=None):
    """Run the whole fast pin set against one oracle build; raises AssertionError on a mismatch."""
    # hand-derived fixtures
    for c in load_golden():
        assert_all_equal(c["V"], c["src"], c["dst"], c["labels"], lib)
    # brute force over every simple graph on up to 4 vertices
    for n in range(0, 5):
        pairs = list(itertools.combinations(range(n), 2))
        for mask in range(1 << len(pairs)):
            chosen = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
            s = [p[0] for p in chosen]
            d = [p[1] for p in chosen]
            assert_all_equal(n, s, d, closure_labels(n, s, d), lib)
    # closed forms
    for V in (2, 7, 33):
        assert_all_equal(V, *path_edges(range(V)), np.zeros(V), lib)
        assert_all_equal(V, *path_edges(range(V - 1, -1, -1)), np.zeros(V), lib)
    assert_all_equal(9, [], [], np.arange(9), lib)


def test_golden_fixtures():
    cases = load_golden()
    assert len(cases) >= 5
    for c in cases:
        assert len(c["labels"]) == c["V"]
        assert_all_equal(c["V"], c["src"], c["dst"], c["labels"])


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5])
def test_brute_force_every_simple_graph(n):
    pairs = list(itertools.combinations(range(n), 2))
    for mask in range(1 << len(pairs)):
        chosen = [pairs[i] for i in range(len(pairs)) if mask >> i & 1]
        s = [p[0] for p in chosen]
        d = [p[1] for p in chosen]
        assert_all_equal(n, s, d, closure_labels(n, s, d))


def test_brute_force_random_multigraphs():
    rng = np.random.default_rng(7)
    for _ in range(1500):
        n = int(rng.integers(1, 9))
        m = int(rng.integers(0, 3 * n))
        s = rng.integers(0, n, m)
        d = rng.integers(0, n, m)  # self-loops and duplicates included
        assert_all_equal(n, s, d, closure_labels(n, s, d))


@pytest.mark.parametrize("V", [1, 2, 5, 100, 10_000])
def test_closed_form_paths(V):
    rng = np.random.default_rng(V)
    assert_all_equal(V, *path_edges(range(V)), np.zeros(V))
    assert_all_equal(V, *path_edges(range(V - 1, -1, -1)), np.zeros(V))
    assert_all_equal(V, *path_edges(rng.permutation(V)), np.zeros(V))


@pytest.mark.parametrize("V", [0, 1, 17, 5000])
def test_closed_form_edgeless(V):
    assert_all_equal(V, [], [], np.arange(V))


@pytest.mark.parametrize("k,size", [(1, 5), (3, 4), (10, 7), (50, 3)])
def test_closed_form_disjoint_cliques(k, size):
    V = k * size
    # contiguous blocks: clique j = {j*size, ..., j*size+size-1} -> label j*size
    s, d = zip(*[clique_edges(range(j * size, (j + 1) * size)) for j in range(k)])
    expected = (np.arange(V) // size) * size
    assert_all_equal(V, np.concatenate(s), np.concatenate(d), expected)
    # interleaved: clique j = {j, j+k, j+2k, ...} -> label j
    s, d = zip(*[clique_edges(range(j, V, k)) for j in range(k)])
    expected = np.arange(V) % k
    assert_all_equal(V, np.concatenate(s), np.concatenate(d), expected)


@pytest.mark.parametrize("V", [2, 10, 1000])
def test_closed_form_stars(V):
    hub = V - 1
    assert_all_equal(V, np.full(V - 1, hub), np.arange(V - 1), np.zeros(V))
    assert_all_equal(V, np.zeros(V - 1, np.int64), np.arange(1, V), np.zeros(V))


@pytest.mark.parametrize("side", [1, 2, 8, 40])
def test_closed_form_full_and_empty_grid(side):
    V = side * side
    s, d = grid_edges(side)
    assert_all_equal(V, s, d, np.zeros(V))
    g = gen.grid_csr(side, 1.0, seed=3, offsets64=True)
    assert g.nnz == 2 * 2 * side * (side - 1)
    lab, n = oracle.labels_uf_csr(g.row_ptr, g.col)
    assert n == 1 and not lab.any()
    g = gen.grid_csr(side, 0.0, seed=3, offsets64=True)
    assert g.nnz == 0
    lab, n = oracle.labels_bfs_csr(g.row_ptr, g.col)
    assert n == V and np.array_equal(lab, np.arange(V))


def _scipy_min_labels(V, row_ptr, col):
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    m = sp.csr_matrix((np.ones(len(col), np.int8), np.asarray(col), np.asarray(row_ptr, np.int64)), shape=(V, V))
    n, comp = csg.connected_components(m, directed=False)
    return n, min_id_from_component_ids(comp)


@pytest.mark.parametrize("kind", ["er_sparse", "er_dense", "grid_half", "grid_road", "rmat"])
def test_against_scipy(kind):
    if kind == "er_sparse":
        g = gen.er_csr(50_000, 20_000, seed=11)
    elif kind == "er_dense":
        g = gen.er_csr(20_000, 200_000, seed=12)
    elif kind == "grid_half":
        g = gen.grid_csr(300, 0.5, seed=13)
    elif kind == "grid_road":
        g = gen.grid_csr(300, 0.9, seed=14)
    else:
        g = gen.rmat_csr(16, 4, seed=15)
    n_sp, expect = _scipy_min_labels(g.n_vertices, g.row_ptr, g.col)
    lab_uf, n_uf = oracle.labels_uf_csr(g.row_ptr, g.col)
    lab_bfs, n_bfs = oracle.labels_bfs_csr(g.row_ptr, g.col)
    assert n_uf == n_bfs == n_sp
    assert np.array_equal(lab_uf, expect)
    assert np.array_equal(lab_bfs, expect)
    assert check_min_label_invariants(g.row_ptr, g.col, lab_uf) == []


def test_coo_and_csr_agree_on_er():
    src, dst = gen.er_coo(30_000, 40_000, seed=21)
    g = gen.sym_csr_from_coo(30_000, src, dst)
    a, na = oracle.labels_uf_coo(30_000, src, dst)
    b, nb = oracle.labels_bfs_coo(30_000, src, dst)
    c, nc = oracle.labels_uf_csr(g.row_ptr, g.col)
    assert na == nb == nc
    assert np.array_equal(a, b) and np.array_equal(a, c)


def test_sampled_labels_match_full():
    g = gen.grid_csr(120, 0.55, seed=31)
    full, _ = oracle.labels_bfs_csr(g.row_ptr, g.col)
    s = oracle.SampledLabels(g.row_ptr, g.col)
    rng = np.random.default_rng(0)
    for v in rng.integers(0, g.n_vertices, 200):
        assert s.label_of(int(v)) == full[v]


def test_malformed_inputs_rejected():
    with pytest.raises(ValueError):
        oracle.labels_uf_coo(3, [0, 3], [1, 1])
    with pytest.raises(ValueError):
        oracle.labels_bfs_coo(3, [-1], [1])
    with pytest.raises(ValueError):
        oracle.labels_uf_csr(np.array([0, 2, 1, 3]), np.array([1, 2, 0], np.int32))  # non-monotone
    with pytest.raises(ValueError):
        oracle.labels_bfs_csr(np.array([0, 1, 2]), np.array([1, 5], np.int32))  # endpoint out of range


def test_pin_set_passes_on_the_real_oracle():
    pins()
