"""Autotuner host logic (no GPU): size buckets, the coordinate search over candidate options,
the labels-must-not-change check and the JSON cache."""
import pytest

from paper_1612_01178_gb300.tune import Tuner, bucket


def test_bucket_keys():
    assert bucket("csr", 16_777_216, 60_384_074, True) == "csr:V2^24:d2^2:local"
    assert bucket("csr", 100_000, 2_000_000) == "csr:V2^17:d2^4:any"
    assert bucket("csr", 5, 0, False) == "csr:V2^2:d2^-99:random"


def test_search_picks_fastest_and_caches(tmp_path):
    cost = {("tile_vertices", -1): 5.0, ("segments", 4): 2.0, ("block", 512): 1.0}

    def measure(opts):
        ms = 10.0 - sum(v for (k, val), v in cost.items() if opts.get(k) == val)
        return ms, "same-labels"

    t = Tuner(str(tmp_path / "tune.json"))
    best, ms, log = t.search(measure)
    assert best == {"tile_vertices": -1, "segments": 4, "block": 512}
    assert ms == 2.0 and len(log) > 5
    t.cache["k"] = {"options": best, "ms": ms}
    t.save()
    t2 = Tuner(str(tmp_path / "tune.json"))
    assert t2.lookup("k") == best
    assert t2.lookup("missing") is None


def test_search_rejects_options_that_change_labels():
    def measure(opts):
        return 1.0, ("different" if opts.get("segments") == 2 else "labels")

    with pytest.raises(AssertionError):
        Tuner(None).search(measure)


def test_search_space_names_real_options():
    from paper_1612_01178_gb300 import cc
    from paper_1612_01178_gb300.tune import SEARCH, SEARCH_BATCHED
    fields = {f for f, _ in cc.cc_options._fields_}
    for name, values in SEARCH + SEARCH_BATCHED:
        assert name in fields, name
        assert values and values[0] == 0 or name == "mode"
    names = [n for n, _ in SEARCH]
    for knob in ("hook_k", "auto_min_vertices", "auto_local_permille", "auto_lowdeg_permille", "cluster_max_vertices"):
        assert knob in names


def test_bucket_lookup_helpers(tmp_path):
    t = Tuner(str(tmp_path / "t.json"))
    t.cache[bucket("csr", 100_000, 2_000_000)] = {"options": {"mode": 6}, "ms": 0.02}
    assert t.options_for_csr(100_000, 2_000_000) == {"mode": 6}
    assert t.options_for_csr(100_000, 200) is None
    t.cache[bucket("batch12", 5_000_000, 60_000_000)] = {"options": {"block": 512}, "ms": 9.0}
    assert t.options_for_batch(4096, 5_000_000, 60_000_000) == {"block": 512}
