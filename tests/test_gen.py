"""Seeded input generators: determinism, thread-count independence and the
statistics each family is defined by."""
import numpy as np
import pytest

import gen


def test_er_deterministic_and_thread_independent():
    a = gen.er_coo(1000, 200_000, seed=5, threads=1)
    b = gen.er_coo(1000, 200_000, seed=5, threads=8)
    c = gen.er_coo(1000, 200_000, seed=6, threads=8)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0])
    # uniform endpoints: every vertex near E*2/V = 400 endpoint hits
    hits = np.bincount(np.concatenate(a), minlength=1000)
    assert hits.min() > 300 and hits.max() < 500


def test_symmetric_csr_properties():
    src, dst = gen.er_coo(5000, 30_000, seed=9)
    g = gen.sym_csr_from_coo(5000, src, dst, threads=4)
    g1 = gen.sym_csr_from_coo(5000, src, dst, threads=1)
    assert np.array_equal(g.row_ptr, g1.row_ptr) and np.array_equal(g.col, g1.col)
    assert g.nnz == 2 * 30_000 and g.row_ptr.dtype == np.int32
    rows = np.repeat(np.arange(5000), np.diff(g.row_ptr))
    fwd = np.sort(rows.astype(np.int64) * 5000 + g.col)
    rev = np.sort(g.col.astype(np.int64) * 5000 + rows)
    assert np.array_equal(fwd, rev)  # the reverse of every arc is present (with multiplicity)
    for v in range(0, 5000, 97):
        seg = g.col[g.row_ptr[v]:g.row_ptr[v + 1]]
        assert np.all(seg[:-1] <= seg[1:])


def test_self_loop_emits_two_arcs():
    g = gen.sym_csr_from_coo(3, np.array([1, 0], np.int32), np.array([1, 2], np.int32))
    assert list(g.row_ptr) == [0, 1, 3, 4]
    assert list(g.col) == [2, 1, 1, 0]


def test_grid_counts_and_structure():
    side, p = 64, 0.9
    g = gen.grid_csr(side, p, seed=1)
    g8 = gen.grid_csr(side, p, seed=1, threads=1)
    assert np.array_equal(g.col, g8.col)
    lattice = 2 * side * (side - 1)
    kept = g.nnz // 2
    assert abs(kept - p * lattice) < 5 * np.sqrt(lattice * p * (1 - p))
    rows = np.repeat(np.arange(side * side), np.diff(g.row_ptr))
    diff = np.abs(g.col - rows)
    assert set(np.unique(diff)) <= {1, side}
    full = gen.grid_csr(side, 1.0, seed=1)
    assert full.nnz == 2 * lattice


def test_permutation_is_bijection():
    for n in (1, 2, 5, 1000, 1 << 12, (1 << 11) + 3):
        perm = gen.permutation(n, seed=4)
        assert np.array_equal(np.sort(perm), np.arange(n))
    p = gen.permutation(1 << 12, seed=4)
    assert (p != np.arange(1 << 12)).mean() > 0.99


def test_rmat_quadrant_statistics():
    scale, E = 10, 400_000
    src, dst = gen.rmat_coo(scale, E, seed=2, permute=False)
    # top bit of (u, v) follows the first quadrant choice: P(u<half, v<half) = a, etc.
    half = 1 << (scale - 1)
    q = (src >= half).astype(int) * 2 + (dst >= half).astype(int)
    freq = np.bincount(q, minlength=4) / E
    assert np.allclose(freq, [0.57, 0.19, 0.19, 0.05], atol=0.005)
    s2, d2 = gen.rmat_coo(scale, E, seed=2, permute=True)
    perm = gen.permutation(1 << scale, seed=2)
    assert np.array_equal(s2, perm[src]) and np.array_equal(d2, perm[dst])
    s3, _ = gen.rmat_coo(scale, E, seed=2, permute=True, threads=1)
    assert np.array_equal(s2, s3)


def test_named_small_workload_sizes():
    g = gen.workload_er_100k()
    assert g.n_vertices == 100_000 and g.nnz == 2_000_000 and g.n_edges == 1_000_000


def test_bad_arguments():
    with pytest.raises(ValueError):
        gen.sym_csr_from_coo(3, np.array([0], np.int32), np.array([3], np.int32))
    with pytest.raises(ValueError):
        gen.er_coo(0, 5, seed=1)
