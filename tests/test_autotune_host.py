"""Autotuner host logic: the result cache round-trips through its JSON file and is keyed by
device and size bucket (CPU only)."""
import json

from paper_2508_04701_gb300 import autotune


def test_cache_roundtrip(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("SIRIUS_AUTOTUNE_CACHE", str(path))
    assert autotune.cache_path() == str(path)
    assert autotune._load() == {}
    autotune._store({"k": {"rows_per_unit": 65536, "load_factor": 0.5}})
    assert json.loads(path.read_text())["k"]["rows_per_unit"] == 65536
    assert autotune._load()["k"]["load_factor"] == 0.5


def test_size_buckets():
    assert autotune._bucket(1) == 0
    assert autotune._bucket(1023) == 9
    assert autotune._bucket(1024) == 10
    assert autotune._bucket(0) == 0
