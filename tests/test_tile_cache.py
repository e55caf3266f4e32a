"""Host logic of the JSON autotune cache (no GPU): keys, storage, reuse."""

import json
from types import SimpleNamespace

from paper_1211_0780_b300 import xy


def fake_sim(L, R, mode=None):
    s = SimpleNamespace(L=list(L), R=list(R))
    if mode is not None:
        s.exec_mode = mode
    return s


def test_key_depends_on_every_field():
    base = xy.autotune_cache_key(fake_sim([64], [32]), 1, 3, device="B300", library="abc")
    assert json.loads(base) == {"L": [64], "R": [32], "nM": 1, "nOR": 3, "exec": xy.EXEC_PLAIN,
                                "device": "B300", "library": "abc"}
    others = [
        xy.autotune_cache_key(fake_sim([64], [16]), 1, 3, device="B300", library="abc"),
        xy.autotune_cache_key(fake_sim([64, 32], [32, 8]), 1, 3, device="B300", library="abc"),
        xy.autotune_cache_key(fake_sim([64], [32]), 1, 5, device="B300", library="abc"),
        xy.autotune_cache_key(fake_sim([64], [32], xy.EXEC_PERSISTENT), 1, 3, device="B300", library="abc"),
        xy.autotune_cache_key(fake_sim([64], [32]), 1, 3, device="other", library="abc"),
        xy.autotune_cache_key(fake_sim([64], [32]), 1, 3, device="B300", library="abd"),
    ]
    assert len(set(others + [base])) == len(others) + 1


def test_store_and_load_round_trip(tmp_path):
    path = str(tmp_path / "tiles.json")
    assert xy.load_tile_cache(path) == {}
    k1 = xy.autotune_cache_key(fake_sim([160], [1]), 1, 5, device="d", library="l")
    k2 = xy.autotune_cache_key(fake_sim([16, 24], [2, 3]), 1, 3, device="d", library="l")
    xy.store_tile_cache(path, k1, [(8, 8, 3)])
    xy.store_tile_cache(path, k2, [(4, 8, 0), (3, 8, 3)])
    got = xy.load_tile_cache(path)
    assert got == {k1: [(8, 8, 3)], k2: [(4, 8, 0), (3, 8, 3)]}
    xy.store_tile_cache(path, k1, [(16, 8, 3)])  # replaces the old entry only
    got = xy.load_tile_cache(path)
    assert got[k1] == [(16, 8, 3)] and got[k2] == [(4, 8, 0), (3, 8, 3)]
    assert not list(tmp_path.glob("*.tmp"))


def test_unreadable_cache_is_empty(tmp_path):
    path = tmp_path / "tiles.json"
    path.write_text("{not json")
    assert xy.load_tile_cache(str(path)) == {}
    path.write_text("[1, 2]")
    assert xy.load_tile_cache(str(path)) == {}
