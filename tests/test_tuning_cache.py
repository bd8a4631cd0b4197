"""The tile-shape cache file (host logic of Plan.autotune; no device)."""
import json

import pytest

from paper_2401_09961_gb300 import tuning


def test_round_trip_and_other_keys_kept(tmp_path):
    path = str(tmp_path / "sub" / "tiles.json")
    assert tuning.cache_get(path, "k") is None          # no file yet: empty cache
    k1 = tuning.tuning_key(4096, 4096, 2, 0, "NVIDIA GB300")
    k2 = tuning.tuning_key(256, 384, 2, 0, "NVIDIA GB300")
    assert k1 != k2
    tuning.cache_put(path, k1, (24, 32), [0.1] * 8)
    tuning.cache_put(path, k2, (8, 16))
    assert tuning.cache_get(path, k1) == (24, 32)
    assert tuning.cache_get(path, k2) == (8, 16)
    data = json.load(open(path))
    assert data[k1]["ms"]["direction"] == [0.1] * 4 and data[k1]["ms"]["rows"] == [8, 16, 24, 32]
    tuning.cache_put(path, k1, (16, 16))                # replaced, k2 kept
    assert tuning.cache_get(path, k1) == (16, 16) and tuning.cache_get(path, k2) == (8, 16)
    assert [p.name for p in (tmp_path / "sub").iterdir()] == ["tiles.json"]   # no temp files


def test_keys_separate_size_precision_system_and_gpu():
    keys = {tuning.tuning_key(*a) for a in [(256, 256, 2, 0, "A"), (256, 256, 2, 0, "B"),
                                            (256, 256, 1, 0, "A"), (256, 256, 2, 1, "A"),
                                            (256, 512, 2, 0, "A"), (512, 256, 2, 0, "A")]}
    assert len(keys) == 6


def test_unreadable_or_invalid_entries_are_misses(tmp_path):
    path = tmp_path / "tiles.json"
    path.write_text("{not json")
    assert tuning.cache_get(str(path), "k") is None
    path.write_text(json.dumps({"k": {"tiles": [12, 32]}, "j": {"tiles": [8]}, "i": [8, 8],
                                "h": {"tiles": [8, 32]}}))
    assert tuning.cache_get(str(path), "k") is None     # 12 rows: no such kernel
    assert tuning.cache_get(str(path), "j") is None
    assert tuning.cache_get(str(path), "i") is None
    assert tuning.cache_get(str(path), "h") == (8, 32)
    path.write_text("[1, 2]")                           # not a mapping
    assert tuning.cache_get(str(path), "h") is None
    tuning.cache_put(str(path), "h", (32, 8))           # a bad file is replaced, not appended to
    assert tuning.cache_get(str(path), "h") == (32, 8)


def test_put_rejects_rows_without_a_kernel(tmp_path):
    with pytest.raises(ValueError):
        tuning.cache_put(str(tmp_path / "t.json"), "k", (12, 32))
    with pytest.raises(ValueError):
        tuning.cache_put(str(tmp_path / "t.json"), "k", (8,))


def test_batch_key_depends_on_shapes_and_order():
    a = tuning.batch_key([(256, 384), (512, 512)], 2, 0, "G")
    assert a == tuning.batch_key([(256, 384), (512, 512)], 2, 0, "G")
    assert a != tuning.batch_key([(512, 512), (256, 384)], 2, 0, "G")
    assert a != tuning.batch_key([(256, 384)], 2, 0, "G")
    assert a != tuning.batch_key([(256, 384), (512, 512)], 1, 0, "G")
    assert a != tuning.tuning_key(256, 384, 2, 0, "G")
