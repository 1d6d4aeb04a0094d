"""Sampled-and-filtered hook (CC_MODE_FILTERED): bit-exact parity with the oracle on graphs with
and without a giant component, with the skipped rows' reverse arcs as the only path between
components, and across launch shapes; argument and input errors."""
import itertools

import numpy as np
import pytest

import gen
import oracle
from graphs import clique_edges, directed_csr, path_edges, symmetric_csr

torch = pytest.importorskip("torch")
import paper_1612_01178_gb300 as ccl  # noqa: E402
from paper_1612_01178_gb300 import cc as ccapi  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    ccl.load()
    return torch.device("cuda:0")


def expect(row_ptr, col):
    return oracle.labels_uf_csr(row_ptr, col)[0]


def filtered(dev, row_ptr, col, block=0, grid_blocks=0, sym=True, expect_status=ccapi.CC_OK):
    flags = ccl.CC_FLAG_SYNC | (ccl.CC_FLAG_SYMMETRIC if sym else 0)
    with ccl.ConnectedComponents(0, mode=ccl.CC_MODE_FILTERED, flags=flags, block=block,
                                 grid_blocks=grid_blocks) as cc:
        rp = torch.from_numpy(np.ascontiguousarray(row_ptr)).to(dev)
        cl = torch.from_numpy(np.ascontiguousarray(col, np.int32)).to(dev)
        if expect_status != ccapi.CC_OK:
            with pytest.raises(ccl.CCError) as ei:
                cc.csr(rp, cl)
            assert ei.value.status == expect_status
            return None, None
        out = cc.csr(rp, cl)
        torch.cuda.synchronize()
        return out.cpu().numpy(), cc.run_info()


def check(dev, row_ptr, col, what, **kw):
    got, info = filtered(dev, row_ptr, col, **kw)
    want = expect(row_ptr, col)
    if not np.array_equal(got, want):
        bad = np.flatnonzero(got != want)
        raise AssertionError(f"{what}: {bad.size} labels differ, first at v={bad[0]}: got {got[bad[0]]}, "
                             f"want {want[bad[0]]}")
    assert info["mode"] == ccl.CC_MODE_FILTERED and info["launches"] == 1, info


def test_small_graphs_every_shape(dev):
    src, dst, base = [], [], 0
    for n in range(1, 6):
        pairs = list(itertools.combinations(range(n), 2))
        for mask in range(1 << len(pairs)):
            for i, (a, b) in enumerate(pairs):
                if mask >> i & 1:
                    src.append(base + a)
                    dst.append(base + b)
            base += n
    perm = np.random.default_rng(3).permutation(base)
    rp, col = symmetric_csr(base, perm[np.array(src)], perm[np.array(dst)], np.int32)
    for block in (0, 64, 1024):
        check(dev, rp, col, f"all graphs <= 5 vertices, block {block}", block=block)


def test_giant_component_families(dev):
    for g in (gen.workload_er_100k(), gen.grid_csr(1200, 0.9, seed=2), gen.rmat_csr(18, 8, seed=3),
              gen.rmat_csr(20, 16, seed=4), gen.rmat_csr(16, 8, seed=5, offsets64=True)):
        check(dev, g.row_ptr, g.col, str(g))


def test_no_giant_component(dev):
    # many small components: no root holds an eighth of the sample, so every arc is hooked
    for p in (0.3, 0.45):
        g = gen.grid_csr(800, p, seed=6)
        check(dev, g.row_ptr, g.col, f"grid p={p}")
    n = 400_000  # 2000 disjoint 4-cliques in interleaved numbering, the rest isolated
    members = np.arange(n).reshape(4, -1).T[:2000]
    parts = [clique_edges(m) for m in members]
    src = np.concatenate([p[0] for p in parts])
    dst = np.concatenate([p[1] for p in parts])
    rp, col = symmetric_csr(n, src, dst, np.int32)
    check(dev, rp, col, "cliques + isolated vertices")


def test_components_joined_only_through_skipped_rows(dev):
    # A giant star (hub 0) plus two-vertex paths, some of them linked to star vertices: the
    # star's rows are skipped in the second slice, so those links are hooked from the path side.
    n = 300_000
    src, dst = [], []
    src += [0] * (n // 2 - 1)
    dst += list(range(1, n // 2))
    rest = np.arange(n // 2, n)
    for a, b in zip(rest[:-1:3], rest[1::3]):
        src.append(int(a))
        dst.append(int(b))
    for x in rest[::97]:  # some path vertices hang on late arcs of star vertices 5..
        src.append(int(5 + x % 1000))
        dst.append(int(x))
    rp, col = symmetric_csr(n, np.array(src), np.array(dst), np.int32)
    check(dev, rp, col, "star + paths")
    # the same with the hub at the top ID (the star's root is then not the hub)
    perm = np.arange(n)[::-1]
    rp, col = symmetric_csr(n, perm[np.array(src)], perm[np.array(dst)], np.int32)
    check(dev, rp, col, "star + paths, reversed IDs")


def test_paths_and_two_giants(dev):
    n = 200_000
    for order in (range(n - 1, -1, -1), np.random.default_rng(7).permutation(n)):
        rp, col = symmetric_csr(n, *path_edges(order), np.int32)
        check(dev, rp, col, "path")
    # two equal halves: the sample picks one of them; the other is hooked arc by arc
    half = n // 2
    a = gen.er_csr(half, 4 * half, seed=8)
    s1 = np.repeat(np.arange(half), np.diff(a.row_ptr))
    src = np.concatenate([s1, s1 + half])
    dst = np.concatenate([a.col, a.col + half])
    rp, col = directed_csr(n, src, dst, np.int32)
    check(dev, rp, col, "two ER halves")


def test_launch_shapes(dev):
    g = gen.rmat_csr(17, 8, seed=9)
    for block, grid in ((32, 1), (256, 7), (1024, 0), (128, 0)):
        check(dev, g.row_ptr, g.col, f"block {block} grid {grid}", block=block, grid_blocks=grid)


def test_degenerate_inputs(dev):
    for V in (1, 2, 1000):
        rp = np.zeros(V + 1, np.int32)
        check(dev, rp, np.zeros(0, np.int32), f"edgeless V={V}")
    rp, col = symmetric_csr(5, np.array([0, 1, 2]), np.array([0, 1, 2]), np.int32)  # self-loops only
    check(dev, rp, col, "self-loops")


def test_errors(dev):
    g = gen.er_csr(1000, 4000, seed=10)
    filtered(dev, g.row_ptr, g.col, sym=False, expect_status=ccapi.CC_ERR_INVALID_ARG)
    col = g.col.copy()
    col[int(g.row_ptr[17])] = 5000  # first arc of row 17: read by the first slice
    filtered(dev, g.row_ptr, col, expect_status=ccapi.CC_ERR_OUT_OF_RANGE)
    with ccl.ConnectedComponents(0, mode=ccl.CC_MODE_FILTERED, flags=ccl.CC_FLAG_SYNC) as cc:
        s = torch.zeros(4, dtype=torch.int32, device=dev)
        with pytest.raises(ccl.CCError) as ei:
            cc.coo(8, s, s)
        assert ei.value.status == ccapi.CC_ERR_INVALID_ARG
