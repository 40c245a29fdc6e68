"""The on-disk autotune cache (host only, no GPU): key format and size
classes, round trips of every field (floats exactly, 1e30 "never"
included), replacement, several keys, names that need JSON escapes, and
files that are absent, foreign or broken (reported, never overwritten)."""
import json
import os

import pytest

from paper_2106_14402_gb300 import cb

pytest.importorskip("torch")

BOUNDS = {"sym_hash_max": 1024, "num_hash_max": 2048, "learn_max": 512, "cf_esc": 1.25,
          "cf_prereduce": 1e30}


def test_key_names_device_semiring_sizing_and_size_classes():
    k = cb.tune_key("NVIDIA GB300", "plus_times_f64", 262144, 7_700_000, 5, sizing="learned")
    assert k == f"NVIDIA GB300|sr{cb.SEMIRING['plus_times_f64'][0]}|sizing1|m2^18|a2^23|b2^2"
    # nearest power of two: 3 -> 2^2, 2 -> 2^1, 1 and 0 -> 2^0; 0.75 * 2^20 rounds up
    assert cb.tune_key("d", "min_plus_u32", 0, 1, 3).endswith("|m2^0|a2^0|b2^2")
    assert cb.tune_key("d", "min_plus_u32", 786432, 2, 2).endswith("|m2^20|a2^1|b2^1")
    with pytest.raises(cb.CBError):
        cb.tune_key("d", "min_plus_u32", -1, 1, 1)
    lib = cb.load()
    import ctypes
    small = ctypes.create_string_buffer(8)
    assert lib.cb_tune_key(b"NVIDIA GB300", 1, 0, 1, 1, 1, small, 8) == 1 and small.value == b""


def test_round_trip_replace_and_several_keys(tmp_path):
    path = str(tmp_path / "tune.json")
    assert cb.tune_cache_get(path, "k1") is None           # absent file: a miss, not an error
    cb.tune_cache_put(path, "k1", BOUNDS, 12.5)
    got, ms = cb.tune_cache_get(path, "k1")
    assert got["sym_hash_max"] == 1024 and got["num_hash_max"] == 2048 and got["learn_max"] == 512
    assert got["cf_esc"] == pytest.approx(1.25, abs=0) and got["cf_prereduce"] == pytest.approx(1e30, rel=1e-7)
    assert ms == 12.5
    other = dict(BOUNDS, sym_hash_max=512, cf_esc=0.0, cf_prereduce=4.0)
    cb.tune_cache_put(path, "k2", other, 3.25)
    cb.tune_cache_put(path, "k1", dict(BOUNDS, learn_max=64), 11.0)   # replaces k1 only
    assert cb.tune_cache_get(path, "k1")[0]["learn_max"] == 64
    assert cb.tune_cache_get(path, "k1")[1] == 11.0
    assert cb.tune_cache_get(path, "k2")[0]["cf_prereduce"] == 4.0
    assert cb.tune_cache_get(path, "k3") is None
    doc = json.load(open(path))                       # plain JSON of the documented shape
    assert doc["format"] == "cb-tune-cache-1" and sorted(doc["entries"]) == ["k1", "k2"]
    assert set(doc["entries"]["k2"]) == set(BOUNDS) | {"ms"}
    assert [f for f in os.listdir(tmp_path) if ".tmp" in f] == []


def test_keys_that_need_escapes(tmp_path):
    path = str(tmp_path / "tune.json")
    key = 'GPU "x"\\y\t|sr2'
    cb.tune_cache_put(path, key, BOUNDS, 1.0)
    assert json.load(open(path))["entries"][key]["ms"] == 1.0
    assert cb.tune_cache_get(path, key)[1] == 1.0


def test_hand_edited_file_is_read(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({"note": [1, 2, {"x": None, "y": True}], "format": "cb-tune-cache-1",
                                "entries": {"k": {"ms": 2e-1, "cf_esc": 2, "cf_prereduce": 16,
                                                  "learn_max": 0, "num_hash_max": 4096,
                                                  "sym_hash_max": 4096}}}, indent=3))
    got, ms = cb.tune_cache_get(str(path), "k")
    assert got["num_hash_max"] == 4096 and got["cf_prereduce"] == 16.0 and ms == pytest.approx(0.2)


@pytest.mark.parametrize("text", ["", "{", "[]", '{"format": "other", "entries": {}}',
                                  '{"format": "cb-tune-cache-1", "entries": {"k": {"ms": 1}}}',
                                  '{"format": "cb-tune-cache-1", "entries": {"k": 3}}',
                                  '{"format": "cb-tune-cache-1", "entries": {}} trailing',
                                  '{"format": "cb-tune-cache-1", "entries": {"k": {"ms": 1, '
                                  '"cf_esc": 1, "cf_prereduce": 1, "learn_max": 1.5, '
                                  '"num_hash_max": 1, "sym_hash_max": 1}}}'])
def test_foreign_or_broken_files_are_errors_and_left_alone(tmp_path, text):
    path = tmp_path / "tune.json"
    path.write_text(text)
    with pytest.raises(cb.CBError) as e:
        cb.tune_cache_get(str(path), "k")
    assert e.value.code == 1
    with pytest.raises(cb.CBError):
        cb.tune_cache_put(str(path), "k", BOUNDS, 1.0)
    assert path.read_text() == text


def test_unwritable_location_is_an_error(tmp_path):
    with pytest.raises(cb.CBError):
        cb.tune_cache_put(str(tmp_path / "no_such_dir" / "tune.json"), "k", BOUNDS, 1.0)
