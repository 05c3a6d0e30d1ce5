"""The autotuner's cache of tile shapes (paper_1901_08766_gb300.tuning) on the host:
workload classes, the JSON file, and tuning through the cache."""
import json
import os

from paper_1901_08766_gb300 import tuning


def _key(domains, storage="f16s", deform=False, device="dev", sms=152):
    return tuning.workload_key(device, sms, storage, deform, domains)


def test_workload_classes():
    base = _key([(1024, 512)] * 4)
    # cells rounded to half octaves: a few percent more cells is the same class, twice as
    # many is another; the width class is the octave of nx
    assert _key([(1024, 512)] * 4 + [(64, 32)]) == base
    assert _key([(1024, 512)] * 8) != base
    assert _key([(1100, 476)] * 4) == base                        # same octave, ~same cells
    assert _key([(2048, 256)] * 4) != base                        # same cells, wider
    assert _key([(1024, 512)] * 4, storage="f32") != base
    assert _key([(1024, 512)] * 4, deform=True) != base
    assert _key([(1024, 512)] * 4, device="other") != base
    assert _key([(1024, 512)] * 4, sms=148) != base
    # widths holding at least a quarter of the cells: one narrow domain among wide ones
    # does not change the class, a quarter of the cells in narrow domains does
    assert _key([(1024, 512)] * 3 + [(256, 128)]) == _key([(1024, 512)] * 3)
    mixed = _key([(1024, 512)] * 3 + [(256, 4096)])
    assert mixed.endswith("|w8.10")
    assert _key([]).endswith("|empty")
    # the order of the domains does not matter
    assert _key([(300, 100), (2000, 900)]) == _key([(2000, 900), (300, 100)])


def test_cache_round_trip_and_atomic_file(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    c = tuning.TuneCache(path)
    assert c.get("k1") is None and c.misses == 1
    c.put("k1", (8, 12, 4, 4), 376.5)
    c.put("k2", [4, 8, 2, 0], 50.0)
    assert c.get("k1") == ((8, 12, 4, 4), 376.5) and c.hits == 1
    with open(path) as f:
        data = json.load(f)
    assert data["k1"] == {"tile": [8, 12, 4, 4], "us": 376.5}
    assert sorted(os.listdir(os.path.dirname(path))) == ["tune.json"]  # no temporary left
    d = tuning.TuneCache(path)
    assert d.entries == c.entries
    # malformed entries are skipped, the rest kept
    data["bad"] = {"tile": [1, 2]}
    data["worse"] = {"us": 3.0}
    with open(path, "w") as f:
        json.dump(data, f)
    assert set(tuning.TuneCache(path).entries) == {"k1", "k2"}
    # a cache without a path lives in memory only
    m = tuning.TuneCache()
    m.put("k", (8, 8, 1, 0), 1.0)
    assert m.get("k") == ((8, 8, 1, 0), 1.0)


def test_cached_autotune_times_once_per_class():
    cache = tuning.TuneCache()
    state = {"tile": (0, 0, 0, 0), "timed": 0}

    def tune():
        state["timed"] += 1
        state["tile"] = (8, 12, 4, 4)
        return 42.0

    def set_tile(*t):
        state["tile"] = t

    get_tile = lambda: state["tile"]  # noqa: E731
    assert tuning.cached_autotune(cache, "a", tune, set_tile, get_tile) == 42.0
    state["tile"] = (4, 4, 1, 0)  # changed by hand since
    assert tuning.cached_autotune(cache, "a", tune, set_tile, get_tile) == 42.0
    assert state == {"tile": (8, 12, 4, 4), "timed": 1}
    tuning.cached_autotune(cache, "b", tune, set_tile, get_tile)
    assert state["timed"] == 2
