"""Host side of the tile cache (no GPU): the JSON file ddsp_plan_autotune
writes and ddsp_plan_create reads, through ddsp_tile_cache_get / _put."""
import json

import pytest

from paper_2605_03531_b300 import DdspError, build, tile_cache_get, tile_cache_put


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def test_round_trip_and_replace(tmp_path):
    path = tmp_path / "tiles.json"
    assert tile_cache_get(path, "gpu/nchan=4096") is None   # no file yet
    tile_cache_put(path, "gpu/nchan=4096", (16, 4, 11, 2, 48), 37.8)
    tile_cache_put(path, "gpu/nchan=256", (8, 8, 5, 2, 16), 0.41)
    assert tile_cache_get(path, "gpu/nchan=4096") == ((16, 4, 11, 2, 48),
                                                       pytest.approx(37.8))
    tile_cache_put(path, "gpu/nchan=4096", (32, 8, 6, 2, 48), 36.5)
    t, ms = tile_cache_get(path, "gpu/nchan=4096")
    assert t == (32, 8, 6, 2, 48) and ms == pytest.approx(36.5)
    assert tile_cache_get(path, "gpu/nchan=256")[0] == (8, 8, 5, 2, 16)
    # the file is JSON with one entry per key
    doc = json.loads(path.read_text())
    assert doc["version"] == 1 and len(doc["entries"]) == 2
    assert {e["key"] for e in doc["entries"]} == {"gpu/nchan=4096",
                                                  "gpu/nchan=256"}


def test_bad_keys_and_files(tmp_path):
    path = tmp_path / "tiles.json"
    for key in ('a"b', "a\\b", "", "x\ny"):
        with pytest.raises(DdspError):
            tile_cache_put(path, key, (16, 4, 11, 2, 48), 1.0)
    bad = tmp_path / "bad.json"
    bad.write_text('{"entries": [{"key": "k", "tile": [1, 2')
    with pytest.raises(DdspError):
        tile_cache_get(bad, "k")
    assert tile_cache_get(tmp_path / "missing.json", "k") is None
