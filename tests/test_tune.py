"""Host logic of the tile autotuner (no GPU): candidate set, selection, cache."""

import json

from paper_1712_07973_gb300 import tune


def test_tune_selects_fastest_and_caches(tmp_path):
    path = str(tmp_path / "tiles.json")
    fake = {2: 9.0, 4: 5.0, 6: 5.0, 8: 7.0}
    best, timings = tune.tune(96, 64, "fp32", path=path, measure=lambda t: fake[t], sm_count=152)
    assert best == 6  # ties go to the larger tile
    assert timings == fake
    d = json.load(open(path))
    assert d[tune.cache_key(96, 64, "fp32", 152)]["tile"] == 6
    # a second entry keeps the first
    tune.tune(48, 5, "fp64", path=path, measure=lambda t: 10.0 - t, sm_count=152)
    d = tune.load_cache(path)
    assert set(d) == {"n96:N64:fp32:sm152", "n48:N5:fp64:sm152"}
    # candidates are clipped to N
    assert d["n48:N5:fp64:sm152"]["tile"] == 5
    assert sorted(map(int, d["n48:N5:fp64:sm152"]["ms"])) == [2, 4, 5]


def test_cache_path_env(monkeypatch, tmp_path):
    monkeypatch.setenv("EXX_TUNE_CACHE", str(tmp_path / "x.json"))
    assert tune.cache_path() == str(tmp_path / "x.json")
    assert tune.load_cache() == {}
