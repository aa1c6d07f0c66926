"""Autotuner host logic: buckets, the fallback model and table persistence."""
import json

from paper_1510_08642_gb300 import autotune


def test_bucket_and_default():
    assert autotune.bucket(2, 1024, 1000, 33) == "2:10:10:5"
    assert autotune.default_choice(2, 4096, 4096, 4096) == ("winograd", 256)
    assert autotune.default_choice(2, 8192, 8192, 8192) == ("winograd", 256)
    assert autotune.default_choice(2, 16384, 16384, 16384) == ("winograd", 512)
    assert autotune.default_choice(4, 3000, 3000, 3000) == ("winograd", 256)
    assert autotune.default_choice(2, 600, 700, 900) == ("winograd", 256)
    assert autotune.default_choice(4, 100, 2000, 2000)[0] == "block"


def test_table_roundtrip(tmp_path):
    path = str(tmp_path / "tune.json")
    t = autotune.Tuner(path)
    t.table[autotune.bucket(2, 512, 512, 512)] = {"algo": "strassen", "cutoff": 128, "seconds": 1e-3}
    t.save()
    data = json.load(open(path))
    assert t.gpu in data
    t2 = autotune.Tuner(path)
    assert t2.choose(2, 512, 500, 530) == ("strassen", 128)
    assert t2.choose(2, 64, 64, 64) == ("block", 512)


def test_candidates_split_at_least_once():
    t = autotune.Tuner("/nonexistent/x.json")
    c = t.candidates(300, 300, 300)
    assert ("block", 512) in c and ("winograd", 256) in c and ("winograd", 512) not in c
