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


def test_product_candidates_and_fallback():
    t = autotune.Tuner("/nonexistent/x.json")
    c = t.product_candidates(2, 600, 600, 600)
    algos = {(x["algo"], x["accum"]) for x in c}
    assert ("block", "fx") in algos and ("block", "fx_tile") in algos and ("winograd", "fx") in algos
    assert all(x["algo"] != "ozaki2_tc" for x in c)  # elementwise class by default
    assert t.choose_product(2, 4096, 4096, 4096) == dict(algo="winograd", cutoff=256, accum="fx", slices=0)
    t.table[t._pkey(2, 1024, 1024, 1024, True, 104)] = dict(algo="ozaki2_tc", cutoff=512, accum="fx",
                                                           slices=31, seconds=1e-3)
    assert t.choose_product(2, 1000, 1100, 1024, allow_normwise=True)["slices"] == 31
    assert t.choose_product(2, 1000, 1100, 1024)["algo"] != "ozaki2_tc"


def test_moduli_for_meets_the_precision():
    """The fewest moduli whose scaling precision P >= bits + ceil(log2 l),
    against the library's own P (the C ABI, no GPU needed)."""
    from paper_1510_08642_gb300 import capi
    for l, bits in ((64, 100), (1024, 104), (4096, 104), (65536, 100)):
        N = autotune.moduli_for(l, bits)
        need = bits + (l - 1).bit_length()
        assert N >= 2 and capi.ddg_ozaki2_precision(N, l) >= need
        assert capi.ddg_ozaki2_precision(N - 1, l) < need


def test_unreadable_table_starts_empty(tmp_path):
    bad = tmp_path / "tune.json"
    for text in ("{not json", "[1, 2]"):
        bad.write_text(text)
        t = autotune.Tuner(str(bad))
        assert t.table == {} and t.choose(2, 4096, 4096, 4096) == ("winograd", 256)
    t.table["2:9:9:9"] = {"algo": "block", "cutoff": 512, "seconds": 1e-3}
    t.save()  # replaces the unreadable file
    assert autotune.Tuner(str(bad)).choose(2, 512, 512, 512) == ("block", 512)
