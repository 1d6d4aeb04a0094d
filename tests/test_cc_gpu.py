"""Parity of the CUDA path (through the C ABI) with the CPU oracle: bit-exact labels.

Every case runs on the GPU through ``paper_1612_01178_gb300.cc`` (ctypes -> libcc.so);
expected labels come from the pinned oracle on the same seeded inputs."""
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

MODES = {"persistent": ccl.CC_MODE_PERSISTENT, "multi": ccl.CC_MODE_MULTI_LAUNCH}


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    ccl.load()
    return torch.device("cuda:0")


# hierarchical hook windows exercised by the tests: default (8192), off, smallest, largest
TILES = [0, -1, 256, 32768]


def gpu_csr(dev, row_ptr, col, *, mode="persistent", segments=0, sym=False, grid_blocks=0, block=256,
            validate=False, expect_status=ccl.cc.CC_OK, tile=0, chunk=0):
    flags = ccl.CC_FLAG_SYNC | (ccl.CC_FLAG_SYMMETRIC if sym else 0) | (ccl.CC_FLAG_VALIDATE if validate else 0)
    with ccl.ConnectedComponents(0, mode=MODES[mode], segments=segments, flags=flags, grid_blocks=grid_blocks,
                                 block=block, tile_vertices=tile, chunk_arcs=chunk) as cc:
        rp = torch.from_numpy(np.ascontiguousarray(row_ptr)).to(dev)
        cl = torch.from_numpy(np.ascontiguousarray(col, np.int32)).to(dev)
        if expect_status != ccl.cc.CC_OK:
            with pytest.raises(ccl.CCError) as ei:
                cc.csr(rp, cl)
            assert ei.value.status == expect_status
            return None
        out = cc.csr(rp, cl)
        torch.cuda.synchronize()
        return out.cpu().numpy()


def gpu_coo(dev, V, src, dst, *, mode="persistent", segments=0):
    with ccl.ConnectedComponents(0, mode=MODES[mode], segments=segments, flags=ccl.CC_FLAG_SYNC) as cc:
        s = torch.from_numpy(np.ascontiguousarray(src, np.int32)).to(dev)
        d = torch.from_numpy(np.ascontiguousarray(dst, np.int32)).to(dev)
        out = cc.coo(V, s, d)
        torch.cuda.synchronize()
        return out.cpu().numpy()


def expect(row_ptr, col):
    lab, _ = oracle.labels_uf_csr(row_ptr, col)
    return lab


def assert_labels(got, want, what=""):
    assert got.shape == want.shape, what
    if not np.array_equal(got, want):
        bad = np.flatnonzero(got != want)
        raise AssertionError(f"{what}: {bad.size} labels differ, first at v={bad[0]}: got {got[bad[0]]}, "
                             f"want {want[bad[0]]}")


# ------------------------------------------------------------------------------------------- small

def union_of_all_small_graphs(max_n=5, seed=0):
    """Disjoint union of every simple graph on <= max_n vertices, vertex IDs shuffled."""
    src, dst, base = [], [], 0
    for n in range(1, max_n + 1):
        pairs = list(itertools.combinations(range(n), 2))
        for mask in range(1 << len(pairs)):
            for i, (a, b) in enumerate(pairs):
                if mask >> i & 1:
                    src.append(base + a)
                    dst.append(base + b)
            base += n
    if seed is None:
        return base, np.array(src, np.int64), np.array(dst, np.int64)
    perm = np.random.default_rng(seed).permutation(base)
    return base, perm[np.array(src, np.int64)], perm[np.array(dst, np.int64)]


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("segments", [0, 1, 3, 64])
@pytest.mark.parametrize("tile", TILES)
def test_union_of_all_small_graphs(dev, mode, segments, tile):
    V, s, d = union_of_all_small_graphs()
    for sym in (False, True):
        rp, col = symmetric_csr(V, s, d, np.int32)
        want = expect(rp, col)
        assert_labels(gpu_csr(dev, rp, col, mode=mode, segments=segments, sym=sym, tile=tile), want, f"sym={sym}")
    rp, col = directed_csr(V, d, s, np.int64)  # one direction only, int64 offsets
    assert_labels(gpu_csr(dev, rp, col, mode=mode, segments=segments, tile=tile), expect(rp, col), "directed")
    # ordered (unshuffled) IDs keep most arcs inside one window
    Vo, so, do_ = union_of_all_small_graphs(seed=None)
    rp, col = symmetric_csr(Vo, so, do_, np.int32)
    assert_labels(gpu_csr(dev, rp, col, mode=mode, segments=segments, sym=True, tile=tile),
                  expect(rp, col), "ordered")
    assert_labels(gpu_coo(dev, V, s, d, mode=mode, segments=segments), oracle.labels_uf_coo(V, s, d)[0], "coo")


@pytest.mark.parametrize("mode", sorted(MODES))
def test_random_multigraphs_individually(dev, mode):
    rng = np.random.default_rng(3)
    for _ in range(40):
        n = int(rng.integers(1, 40))
        m = int(rng.integers(0, 4 * n))
        s, d = rng.integers(0, n, m), rng.integers(0, n, m)
        rp, col = symmetric_csr(n, s, d, np.int32)
        want = expect(rp, col)
        assert_labels(gpu_csr(dev, rp, col, mode=mode, sym=True), want, "sym")
        assert_labels(gpu_csr(dev, rp, col, mode=mode, sym=True, tile=-1), want, "sym plain hook")
        assert_labels(gpu_csr(dev, rp, col, mode=mode, segments=int(rng.integers(1, 9))), want, "segments")
        assert_labels(gpu_coo(dev, n, s, d, mode=mode), want, "coo")


def test_degenerate_sizes(dev):
    # V = 0
    assert gpu_csr(dev, np.zeros(1, np.int32), np.zeros(0, np.int32)).shape == (0,)
    # V = 1, no arcs; V = 1 with a self-loop
    assert list(gpu_csr(dev, np.array([0, 0], np.int32), np.zeros(0, np.int32))) == [0]
    assert list(gpu_csr(dev, np.array([0, 2], np.int32), np.array([0, 0], np.int32))) == [0]
    # edgeless graph of many vertices: identity
    V = 1 << 20
    lab = gpu_csr(dev, np.zeros(V + 1, np.int32), np.zeros(0, np.int32))
    assert np.array_equal(lab, np.arange(V))
    # only self-loops and duplicates
    s = np.repeat(np.arange(1000), 3)
    rp, col = symmetric_csr(1000, s, s, np.int32)
    assert np.array_equal(gpu_csr(dev, rp, col, sym=True), np.arange(1000))
    assert np.array_equal(gpu_coo(dev, 5, np.zeros(0, np.int32), np.zeros(0, np.int32)), np.arange(5))


@pytest.mark.parametrize("mode", sorted(MODES))
def test_adversarial_shapes(dev, mode):
    rng = np.random.default_rng(11)
    cases = []
    n = 300_000
    cases.append(("ascending_path", n, *path_edges(range(n))))
    cases.append(("descending_path", n, *path_edges(range(n - 1, -1, -1))))
    cases.append(("random_path", n, *path_edges(rng.permutation(n))))
    hub = 1 << 20
    cases.append(("star_hub_high", hub + 1, np.full(hub, hub), np.arange(hub)))
    cases.append(("star_hub_zero", hub + 1, np.zeros(hub, np.int64), np.arange(1, hub + 1)))
    s, d = clique_edges(range(0, 600, 2))
    cases.append(("clique_even_ids", 600, s, d))
    k = 500
    s, d = zip(*[clique_edges(range(j, 5000, k)) for j in range(k)])
    cases.append(("interleaved_cliques", 5000, np.concatenate(s), np.concatenate(d)))
    # two long paths interleaved with isolated vertices (runs of empty rows)
    m = 200_000
    ids = np.arange(0, 4 * m, 4)
    cases.append(("sparse_rows", 4 * m + 7, ids[:-1], ids[1:]))
    for name, V, s, d in cases:
        rp, col = symmetric_csr(V, s, d, np.int32)
        want = expect(rp, col)
        for sym in (False, True):
            for segments in (1, 0, 7):
                for tile in (0, -1, 1024):
                    got = gpu_csr(dev, rp, col, mode=mode, sym=sym, segments=segments, tile=tile)
                    assert_labels(got, want, f"{name} sym={sym} s={segments} tile={tile}")


def test_launch_shapes(dev):
    g = gen.er_csr(50_000, 200_000, seed=41)
    want = expect(g.row_ptr, g.col)
    for grid, block in ((1, 32), (1, 256), (3, 64), (7, 96), (152, 256), (0, 128), (0, 512), (0, 1024), (5, 1024)):
        for mode in sorted(MODES):
            for tile in (0, -1):
                got = gpu_csr(dev, g.row_ptr, g.col, mode=mode, grid_blocks=grid, block=block, sym=True, tile=tile)
                assert_labels(got, want, f"grid={grid} block={block} {mode} tile={tile}")
    for chunk in (32, 1024):  # dynamically scheduled plain hook
        got = gpu_csr(dev, g.row_ptr, g.col, sym=True, tile=-1, chunk=chunk)
        assert_labels(got, want, f"chunk={chunk}")


# ----------------------------------------------------------------------------------- workloads

@pytest.mark.parametrize("mode", sorted(MODES))
def test_er_100k_1m(dev, mode):
    """Erdos-Renyi V=100,000 with 1,000,000 drawn edges (the small single-graph workload)."""
    g = gen.workload_er_100k()
    want = expect(g.row_ptr, g.col)
    for sym in (False, True):
        for segments in (0, 1, 5, 40):
            for tile in TILES:
                assert_labels(gpu_csr(dev, g.row_ptr, g.col, mode=mode, sym=sym, segments=segments, tile=tile), want,
                              f"sym={sym} s={segments} tile={tile}")
    rp64 = g.row_ptr.astype(np.int64)
    assert_labels(gpu_csr(dev, rp64, g.col, mode=mode, sym=True), want, "int64 offsets")
    src, dst = gen.er_coo(100_000, 1_000_000, seed=1)
    assert_labels(gpu_coo(dev, 100_000, src, dst, mode=mode), want, "coo")


def test_er_varied_density(dev):
    for V, E, seed in ((10_000, 2_000, 1), (10_000, 5_000, 2), (200_000, 100_000, 3), (50_000, 2_000_000, 4)):
        g = gen.er_csr(V, E, seed=seed)
        want = expect(g.row_ptr, g.col)
        assert_labels(gpu_csr(dev, g.row_ptr, g.col, sym=True), want, f"V={V} E={E}")


def test_grid_4096_road(dev):
    """Road-like 4096 x 4096 grid, p = 0.9 (the benchmark workload), full size."""
    g = gen.workload_grid_4096()
    want = expect(g.row_ptr, g.col)
    for mode in sorted(MODES):
        for sym in (True, False):
            for tile in TILES:
                for segments in (0, 1):
                    assert_labels(gpu_csr(dev, g.row_ptr, g.col, mode=mode, sym=sym, tile=tile, segments=segments),
                                  want, f"{mode} sym={sym} tile={tile} s={segments}")


def test_automatic_window_choice(dev):
    """Automatic hook choice: the grid (ID locality) gets the two-phase hook (two launches) with a
    balanced window, a multiple of 256 in [2048, 18432]; a randomly numbered R-MAT graph (skewed
    degrees) and an ER graph of mean degree 20 get the sampled-and-filtered hook, a sparse ER graph
    (mean degree 4) and a small sparse one the plain hook (one launch each)."""
    cases = ((gen.grid_csr(1500, 0.9, seed=11), True, ccl.CC_MODE_PERSISTENT),
             (gen.rmat_csr(18, 8, seed=12), False, ccl.CC_MODE_FILTERED),
             (gen.er_csr(300_000, 3_000_000, seed=13), False, ccl.CC_MODE_FILTERED),
             (gen.er_csr(300_000, 600_000, seed=14), False, ccl.CC_MODE_PERSISTENT),
             (gen.er_csr(20_000, 30_000, seed=15), False, ccl.CC_MODE_PERSISTENT),
             (gen.er_csr(50_000, 500_000, seed=16), False, ccl.CC_MODE_FILTERED))
    for g, tiled, mode in cases:
        want = expect(g.row_ptr, g.col)
        with ccl.ConnectedComponents(0, flags=ccl.CC_FLAG_SYNC | ccl.CC_FLAG_SYMMETRIC) as cc:
            out = cc.csr(torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev))
            info = cc.run_info()
        assert_labels(out.cpu().numpy(), want, f"auto {g}")
        W = info["tile_vertices"]
        if tiled:
            assert W % 256 == 0 and 2048 <= W <= 18432, info
            assert info["launches"] == 2, info
        else:
            assert W == 0 and info["launches"] == 1, info
        assert info["mode"] == mode, info


def test_dense_degree_threshold(dev):
    """auto_dense_degree sets the mean degree n_arcs / V from which a symmetric graph without ID
    locality takes the sampled-and-filtered hook: -1 keeps the plain hook for a dense ER graph, a
    threshold above its mean degree too, the default (8) and a lower one take the filter; the labels
    are the oracle's every time. A value below -1 is refused."""
    g = gen.er_csr(150_000, 1_500_000, seed=17)  # mean degree 20
    want = expect(g.row_ptr, g.col)
    rp, col = torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev)
    for dense, mode in ((0, ccl.CC_MODE_FILTERED), (4, ccl.CC_MODE_FILTERED), (-1, ccl.CC_MODE_PERSISTENT),
                        (32, ccl.CC_MODE_PERSISTENT)):
        with ccl.ConnectedComponents(0, flags=ccl.CC_FLAG_SYNC | ccl.CC_FLAG_SYMMETRIC,
                                     auto_dense_degree=dense) as cc:
            out = cc.csr(rp, col)
            info = cc.run_info()
        assert_labels(out.cpu().numpy(), want, f"auto_dense_degree={dense}")
        assert info["mode"] == mode and info["tile_vertices"] == 0, (dense, info)
    with pytest.raises(ccl.CCError):
        ccl.ConnectedComponents(0, auto_dense_degree=-2)


def test_grid_small_percolation(dev):
    for p in (0.3, 0.5, 0.7, 1.0):
        g = gen.grid_csr(700, p, seed=9)
        want = expect(g.row_ptr, g.col)
        for tile in TILES:
            assert_labels(gpu_csr(dev, g.row_ptr, g.col, sym=True, tile=tile), want, f"p={p} tile={tile}")


def test_rmat_mid(dev):
    g = gen.rmat_csr(20, 16, seed=1)
    want = expect(g.row_ptr, g.col)
    for mode in sorted(MODES):
        for tile in TILES:
            assert_labels(gpu_csr(dev, g.row_ptr, g.col, mode=mode, sym=True, tile=tile), want, f"{mode} {tile}")
    g64 = gen.rmat_csr(18, 8, seed=2, offsets64=True)
    for tile in TILES:
        assert_labels(gpu_csr(dev, g64.row_ptr, g64.col, sym=True, tile=tile), expect(g64.row_ptr, g64.col),
                      f"int64 tile={tile}")


def test_deterministic_repeats(dev):
    g = gen.rmat_csr(17, 16, seed=5)
    want = expect(g.row_ptr, g.col)
    with ccl.ConnectedComponents(0, flags=ccl.CC_FLAG_SYMMETRIC) as cc:
        rp = torch.from_numpy(g.row_ptr).to(dev)
        cl = torch.from_numpy(g.col).to(dev)
        out = torch.empty(g.n_vertices, dtype=torch.int32, device=dev)
        for _ in range(20):
            cc.csr(rp, cl, out)
            cc.sync()
            assert_labels(out.cpu().numpy(), want, "repeat")


def test_host_buffer_entry_point(dev):
    g = gen.grid_csr(1000, 0.6, seed=8)
    want = expect(g.row_ptr, g.col)
    with ccl.ConnectedComponents(0, flags=ccl.CC_FLAG_SYMMETRIC) as cc:
        assert_labels(cc.csr_host(g.row_ptr, g.col), want, "host")
        g2 = gen.er_csr(3000, 9000, seed=3)
        assert_labels(cc.csr_host(g2.row_ptr.astype(np.int64), g2.col), expect(g2.row_ptr, g2.col), "host 2")


# -------------------------------------------------------------------------------------- errors

def test_host_argument_errors(dev):
    lib = ccapi.load()
    with ccl.ConnectedComponents(0) as cc:
        h = cc.handle
        x = torch.zeros(16, dtype=torch.int32, device=dev)
        assert lib.cc_labels_csr(h, -1, 0, x.data_ptr(), 4, None, x.data_ptr()) == ccapi.CC_ERR_INVALID_ARG
        assert lib.cc_labels_csr(h, 4, 4, x.data_ptr(), 3, x.data_ptr(), x.data_ptr()) == ccapi.CC_ERR_INVALID_ARG
        assert lib.cc_labels_csr(h, 4, 4, None, 4, x.data_ptr(), x.data_ptr()) == ccapi.CC_ERR_INVALID_ARG
        # labels overlapping col_idx
        assert lib.cc_labels_csr(h, 4, 8, x.data_ptr(), 4, x[4:].data_ptr(), x[6:].data_ptr()) == \
            ccapi.CC_ERR_INVALID_ARG
        assert lib.cc_labels_coo(h, 4, 2, None, None, x.data_ptr()) == ccapi.CC_ERR_INVALID_ARG
    bad = ccapi.default_options(block=48)
    with pytest.raises(ccl.CCError):
        ccapi.cc_create(0, None, bad)


@pytest.mark.parametrize("mode", sorted(MODES))
def test_out_of_range_endpoint_reported(dev, mode):
    rp = np.array([0, 2, 3, 4], np.int32)
    col = np.array([1, 7, 0, 1], np.int32)  # 7 >= V = 3: caught by the hook's range check
    gpu_csr(dev, rp, col, mode=mode, expect_status=ccapi.CC_ERR_OUT_OF_RANGE)
    # endpoints checked by the COO hook too
    with ccl.ConnectedComponents(0, mode=MODES[mode]) as cc:
        s = torch.tensor([0, 1], dtype=torch.int32, device=dev)
        d = torch.tensor([1, 9], dtype=torch.int32, device=dev)
        cc.coo(3, s, d)
        with pytest.raises(ccl.CCError) as ei:
            cc.sync()
        assert ei.value.status == ccapi.CC_ERR_OUT_OF_RANGE
        # the context stays usable after the error was read
        out = cc.coo(3, s[:1], d[:1])
        cc.sync()
        assert list(out.cpu().numpy()) == [0, 0, 2]


def test_validate_flags_bad_offsets(dev):
    # non-monotone offsets whose arcs all stay inside the arrays: only validation reports it
    rp = np.array([0, 3, 1, 4], np.int32)
    col = np.array([1, 2, 0, 1], np.int32)
    gpu_csr(dev, rp, col, validate=True, expect_status=ccapi.CC_ERR_OUT_OF_RANGE)
    ok = gpu_csr(dev, np.array([0, 1, 2, 2], np.int32), np.array([1, 0], np.int32), validate=True)
    assert list(ok) == [0, 0, 2]


def test_barrier_wait_times_out_and_context_survives(dev):
    g = gen.er_csr(20_000, 40_000, seed=2)
    want = expect(g.row_ptr, g.col)
    with ccl.ConnectedComponents(0, mode=ccl.CC_MODE_PERSISTENT, timeout_ns=50_000_000, grid_blocks=8) as cc:
        rp = torch.from_numpy(g.row_ptr).to(dev)
        cl = torch.from_numpy(g.col).to(dev)
        ccapi.cc_debug_skip_barrier_arrival(cc.handle, 0)
        cc.csr(rp, cl)
        with pytest.raises(ccl.CCError) as ei:
            cc.sync()
        assert ei.value.status == ccapi.CC_ERR_TIMEOUT
        out = cc.csr(rp, cl)  # hook disarmed itself; status cleared
        cc.sync()
        assert_labels(out.cpu().numpy(), want, "after timeout")


# ------------------------------------------------------------------ the paper's baselines (Fig. 1/2)

SOMAN = {"soman": ccapi.CC_MODE_SOMAN, "soman_multijump": ccapi.CC_MODE_SOMAN_MULTIJUMP}


def gpu_csr_mode(dev, row_ptr, col, mode, sym=True):
    flags = ccl.CC_FLAG_SYNC | (ccl.CC_FLAG_SYMMETRIC if sym else 0)
    with ccl.ConnectedComponents(0, mode=mode, flags=flags) as cc:
        out = cc.csr(torch.from_numpy(np.ascontiguousarray(row_ptr)).to(dev),
                     torch.from_numpy(np.ascontiguousarray(col, np.int32)).to(dev))
        torch.cuda.synchronize()
        return out.cpu().numpy(), cc.run_info()


@pytest.mark.parametrize("name", sorted(SOMAN))
def test_host_driven_baselines(dev, name):
    mode = SOMAN[name]
    V, s, d = union_of_all_small_graphs()
    for sym in (True, False):
        rp, col = symmetric_csr(V, s, d, np.int32)
        got, _ = gpu_csr_mode(dev, rp, col, mode, sym)
        assert_labels(got, expect(rp, col), f"{name} small sym={sym}")
    n = 100_000
    for shape in (path_edges(range(n - 1, -1, -1)), path_edges(np.random.default_rng(1).permutation(n)),
                  (np.full(n - 1, n - 1), np.arange(n - 1))):
        rp, col = symmetric_csr(n, *shape, np.int32)
        got, info = gpu_csr_mode(dev, rp, col, mode)
        assert_labels(got, expect(rp, col), f"{name} adversarial")
        assert info["host_round_trips"] >= info["hook_rounds"] >= 1
    for g in (gen.workload_er_100k(), gen.grid_csr(1000, 0.6, seed=3), gen.rmat_csr(16, 8, seed=4)):
        got, info = gpu_csr_mode(dev, g.row_ptr, g.col, mode)
        assert_labels(got, expect(g.row_ptr, g.col), f"{name} {g}")
    with ccl.ConnectedComponents(0, mode=mode, flags=ccl.CC_FLAG_SYNC) as cc:
        s_ = torch.tensor([0], dtype=torch.int32, device=dev)
        with pytest.raises(ccl.CCError):
            cc.coo(2, s_, s_)  # the host-driven baselines take CSR input only


@pytest.mark.slow
def test_rmat26_full_size(dev):
    """R-MAT scale 26, edge factor 16 (2^31 arcs, int64 row offsets): full-size labels against the
    oracle, in the launch configuration the benchmark uses (automatic choice, CC_FLAG_SYMMETRIC)."""
    g = gen.workload_rmat_26()
    assert g.row_ptr.dtype == np.int64 and g.nnz == 1 << 31
    want = expect(g.row_ptr, g.col)
    rp = torch.from_numpy(g.row_ptr).to(dev)
    col = torch.from_numpy(g.col).to(dev)
    for opts in (dict(), dict(mode=ccl.CC_MODE_PERSISTENT, segments=4)):  # filtered (automatic), plain
        with ccl.ConnectedComponents(0, flags=ccl.CC_FLAG_SYMMETRIC | ccl.CC_FLAG_SYNC, **opts) as cc:
            got = cc.csr(rp, col).cpu().numpy()
            info = cc.run_info()
        assert_labels(got, want, f"rmat26 {opts}")
        assert info["mode"] == (ccl.CC_MODE_FILTERED if not opts else ccl.CC_MODE_PERSISTENT), info
    n_comp = int((want == np.arange(g.n_vertices)).sum())
    sizes = np.bincount(want)
    assert sizes.max() > g.n_vertices // 4 and n_comp > 1000  # one giant component plus many singletons
