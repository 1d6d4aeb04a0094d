"""Host-side logic of the serving loop (no GPU): the first-fit arena allocator behind
admission by free device memory."""
import numpy as np

from paper_1612_01178_gb300.serve import Arena


def test_alloc_free_coalesce():
    a = Arena(1024, align=32)
    x = a.alloc(100)   # 128
    y = a.alloc(200)   # 224
    z = a.alloc(300)   # 320
    assert (x, y, z) == (0, 128, 352)
    assert a.used == 128 + 224 + 320
    assert a.alloc(500) is None            # only 352 left at the end
    a.free(y, 200)
    assert a.alloc(224) == 128             # first fit reuses the hole
    a.free(128, 224)
    a.free(x, 100)
    a.free(z, 300)
    assert a.used == 0 and a.free_blocks() == [(0, 1024)]


def test_random_alloc_free_never_overlaps():
    rng = np.random.default_rng(0)
    a = Arena(1 << 16, align=32)
    live = {}
    for _ in range(3000):
        if live and rng.random() < 0.45:
            off = list(live)[int(rng.integers(0, len(live)))]
            a.free(off, live.pop(off))
        else:
            n = int(rng.integers(1, 3000))
            off = a.alloc(n)
            if off is not None:
                live[off] = n
        spans = sorted((o, o + ((n + 31) // 32) * 32) for o, n in live.items())
        assert all(s1[1] <= s2[0] for s1, s2 in zip(spans, spans[1:]))
        assert all(0 <= s[0] and s[1] <= a.capacity for s in spans)
        assert a.used == sum(e - s for s, e in spans)
    for off, n in list(live.items()):
        a.free(off, n)
    assert a.free_blocks() == [(0, 1 << 16)]
