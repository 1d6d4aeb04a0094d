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
