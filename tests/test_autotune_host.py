"""The autotuner's decision cache file, on the CPU (no device needed): entries
round-trip, a file written for another device tag or format is ignored and
replaced, malformed files are ignored, unsafe text is never written, and the
file is always valid JSON (written through a temporary file and a rename)."""
import json
import os

import pytest

DEV = "NVIDIA GB300|sm=152|cc=10.3|spec-autotune-1"


@pytest.fixture(scope="module")
def S():
    from paper_2108_03948_gb300 import build
    build.build()
    from paper_2108_03948_gb300 import spec
    spec.lib()
    return spec


def test_store_and_lookup_round_trip(S, tmp_path):
    p = str(tmp_path / "t.json")
    assert S.spec_tune_cache_lookup(p, DEV, "czt n=1 m=1 b=1") is None          # no file yet
    assert S.spec_tune_cache_store(p, DEV, "czt n=1024 m=512 b=65536", "gemm_f16x3") == 0
    assert S.spec_tune_cache_store(p, DEV, "czt n=2048 m=1024 b=4096", "bluestein") == 0
    assert S.spec_tune_cache_lookup(p, DEV, "czt n=1024 m=512 b=65536") == "gemm_f16x3"
    assert S.spec_tune_cache_lookup(p, DEV, "czt n=2048 m=1024 b=4096") == "bluestein"
    assert S.spec_tune_cache_lookup(p, DEV, "czt n=9 m=9 b=9") is None
    # replace one entry, keep the other
    assert S.spec_tune_cache_store(p, DEV, "czt n=1024 m=512 b=65536", "bluestein") == 0
    assert S.spec_tune_cache_lookup(p, DEV, "czt n=1024 m=512 b=65536") == "bluestein"
    d = json.load(open(p))
    assert d == {"format": "spec-autotune-1", "device": DEV,
                 "entries": {"czt n=1024 m=512 b=65536": "bluestein", "czt n=2048 m=1024 b=4096": "bluestein"}}
    assert not os.path.exists(p + ".tmp")


def test_another_device_invalidates(S, tmp_path):
    p = str(tmp_path / "t.json")
    S.spec_tune_cache_store(p, DEV, "czt n=1 m=2 b=4", "gemm_f16x3")
    other = DEV.replace("sm=152", "sm=148")
    assert S.spec_tune_cache_lookup(p, other, "czt n=1 m=2 b=4") is None
    # storing for the other device replaces the file: the first device's entry is gone
    assert S.spec_tune_cache_store(p, other, "czt n=3 m=3 b=4", "bluestein") == 0
    assert S.spec_tune_cache_lookup(p, DEV, "czt n=1 m=2 b=4") is None
    assert S.spec_tune_cache_lookup(p, other, "czt n=3 m=3 b=4") == "bluestein"
    assert json.load(open(p))["device"] == other


@pytest.mark.parametrize("text", [
    "", "{", "not json", '{"format": "spec-autotune-0", "device": "%s", "entries": {"k": "v"}}' % DEV,
    '{"format": "spec-autotune-1", "device": "%s"}' % DEV,
    '{"format": "spec-autotune-1", "device": "%s", "entries": {"k": }}' % DEV])
def test_malformed_or_old_files_are_ignored_and_replaced(S, tmp_path, text):
    p = tmp_path / "t.json"
    p.write_text(text)
    assert S.spec_tune_cache_lookup(str(p), DEV, "k") is None
    assert S.spec_tune_cache_store(str(p), DEV, "czt n=5 m=5 b=8", "bluestein") == 0
    d = json.loads(p.read_text())
    assert d["entries"] == {"czt n=5 m=5 b=8": "bluestein"}


def test_unsafe_text_is_not_written(S, tmp_path):
    p = str(tmp_path / "t.json")
    assert S.spec_tune_cache_store(p, DEV, 'czt "quoted"', "bluestein") == 0
    assert S.spec_tune_cache_lookup(p, DEV, 'czt "quoted"') is None
    json.load(open(p))                                   # still valid JSON
    assert S.spec_tune_cache_store(p, 'bad"device', "k", "v") == -1
    assert S.spec_tune_cache_store(str(tmp_path / "no" / "dir" / "t.json"), DEV, "k", "v") == -1
