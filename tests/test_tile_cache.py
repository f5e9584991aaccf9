"""The autotuner's JSON tile cache (host code of the library, no GPU)."""
import json
import os

import pytest

from paper_1704_06258_gb300 import binding, build as _build

DEV = "NVIDIA GB300"


@pytest.fixture(scope="module", autouse=True)
def built():
    return _build.build()


def test_missing_file_is_an_empty_cache(tmp_path):
    assert binding.tile_cache_lookup(str(tmp_path / "none.json"), DEV, 1000, 20, 4096) is None


def test_store_then_lookup_by_bucket(tmp_path):
    path = str(tmp_path / "c.json")
    binding.tile_cache_store(path, DEV, 1000, 20, 4096, 128, 3, 1, 0.25)
    binding.tile_cache_store(path, DEV, 6000, 50, 2048, 256, 2, 0, 7.5)
    # same bucket: ceil(n/128) row blocks, p, population rounded up to a power of two
    got = binding.tile_cache_lookup(path, DEV, 1024, 20, 2049)
    assert got == {"ntile": 128, "stages": 3, "raster": 1, "pair": 0, "ms": 0.25}
    assert binding.tile_cache_lookup(path, DEV, 5993, 50, 1100)["stages"] == 2
    # other buckets
    assert binding.tile_cache_lookup(path, DEV, 1025, 20, 4096) is None      # 9 row blocks
    assert binding.tile_cache_lookup(path, DEV, 1000, 21, 4096) is None      # p
    assert binding.tile_cache_lookup(path, DEV, 1000, 20, 4097) is None      # 8192
    assert binding.tile_cache_lookup(path, "NVIDIA B200", 1000, 20, 4096) is None
    doc = json.load(open(path))
    assert doc["format"] == "usaphmp-tile-cache-1" and len(doc["entries"]) == 2


def test_pair_mode_round_trips(tmp_path):
    path = str(tmp_path / "c.json")
    binding.tile_cache_store(path, DEV, 6000, 20, 2048, 256, 4, 1, 1.5, pair=1)
    assert json.load(open(path))["entries"][0]["pair"] == 1
    assert binding.tile_cache_lookup(path, DEV, 6000, 20, 2048) == {"ntile": 256, "stages": 4, "raster": 1,
                                                                   "pair": 1, "ms": 1.5}


def test_store_replaces_the_bucket_entry(tmp_path):
    path = str(tmp_path / "c.json")
    binding.tile_cache_store(path, DEV, 1000, 20, 4096, 128, 3, 1, 0.25)
    binding.tile_cache_store(path, DEV, 1000, 20, 4096, 256, 3, 0, 0.2)
    assert binding.tile_cache_lookup(path, DEV, 1000, 20, 4096)["ntile"] == 256
    assert len(json.load(open(path))["entries"]) == 1
    assert not os.path.exists(path + ".tmp")


def test_quoted_device_names_round_trip(tmp_path):
    path = str(tmp_path / "c.json")
    name = 'GPU "x" \\ y'
    binding.tile_cache_store(path, name, 200, 5, 64, 64, 4, 0, 1.0)
    assert json.load(open(path))["entries"][0]["device"] == name
    assert binding.tile_cache_lookup(path, name, 200, 5, 64)["ntile"] == 64


def test_hand_written_file_with_extra_keys_and_foreign_entries(tmp_path):
    path = str(tmp_path / "c.json")
    doc = {"format": "usaphmp-tile-cache-1", "comment": ["any", {"json": True}, None, -1.5e3],
           "entries": [{"device": DEV, "note": "skipped: no tile fields"},
                       "not an object",
                       {"device": DEV, "n_blocks": 8, "p": 20, "B_pow2": 4096, "ntile": 64, "stages": 2,
                        "raster": 1, "extra": {"k": [1, 2]}}]}
    with open(path, "w") as f:
        json.dump(doc, f, indent=3)
    got = binding.tile_cache_lookup(path, DEV, 1000, 20, 4096)
    # written before pair mode: no "pair" key, read as 0
    assert got == {"ntile": 64, "stages": 2, "raster": 1, "pair": 0, "ms": 0.0}


@pytest.mark.parametrize("text", ['{"format": "usaphmp-tile-cache-1", "entries": [',
                                  '[]', '{"format": "other", "entries": []}',
                                  '{"format": "usaphmp-tile-cache-1"}',
                                  '{"format": "usaphmp-tile-cache-1", "entries": []} trailing'])
def test_malformed_files_are_errors(tmp_path, text):
    path = str(tmp_path / "c.json")
    open(path, "w").write(text)
    with pytest.raises(binding.UsaphmpError) as e:
        binding.tile_cache_lookup(path, DEV, 1000, 20, 4096)
    assert e.value.name == "EINVAL"
    with pytest.raises(binding.UsaphmpError):
        binding.tile_cache_store(path, DEV, 1000, 20, 4096, 256, 3, 0, 0.2)
    assert open(path).read() == text          # a bad file is never overwritten


def test_unwritable_location_is_eio(tmp_path):
    path = str(tmp_path / "no_such_dir" / "c.json")
    with pytest.raises(binding.UsaphmpError) as e:
        binding.tile_cache_store(path, DEV, 1000, 20, 4096, 256, 3, 0, 0.2)
    assert e.value.name == "EIO"
