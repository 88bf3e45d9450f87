"""Host logic of the autotuner cache: keys separate GPU models, rings and levels; stores merge and
round-trip; a missing file reads as empty."""
import json

import pytest

from paper_2509_03024_gb300 import capi


def test_keys_separate_device_ring_and_level():
    k = capi.tune_cache_key("GB300", 1 << 15, [97, 193], 6)
    assert k != capi.tune_cache_key("B200", 1 << 15, [97, 193], 6)
    assert k != capi.tune_cache_key("GB300", 1 << 16, [97, 193], 6)
    assert k != capi.tune_cache_key("GB300", 1 << 15, [97, 257], 6)
    assert k != capi.tune_cache_key("GB300", 1 << 15, [97, 193], 5)
    assert k == capi.tune_cache_key("GB300", 1 << 15, (97, 193), 6)


def test_store_merges_and_round_trips(tmp_path):
    path = str(tmp_path / "tune.json")
    assert capi.load_tune_cache(path) == {}
    a = capi.tune_cache_key("GB300", 1 << 15, [97], 6)
    b = capi.tune_cache_key("GB300", 1 << 16, [97], 11)
    capi.store_tune_cache(path, a, {"ntt": "r8b4", "ks_inner": "s2l"})
    capi.store_tune_cache(path, b, {"ntt": "r16b4"})
    capi.store_tune_cache(path, a, {"ntt": "r8b4", "ks_inner": "p1"})   # replaces a's choices
    got = capi.load_tune_cache(path)
    assert got == {a: {"ntt": "r8b4", "ks_inner": "p1"}, b: {"ntt": "r16b4"}}
    assert json.load(open(path)) == got
    assert list(tmp_path.iterdir()) == [tmp_path / "tune.json"]          # no temporary file left


def test_rejects_a_file_that_is_not_a_cache(tmp_path):
    path = tmp_path / "bad.json"
    path.write_text("[1, 2]")
    with pytest.raises(ValueError):
        capi.load_tune_cache(str(path))
