"""The bench's roofline arithmetic on CPU: the dominant-kernel figures from a
launch profile and the committed ncu counts, and the source-hash check that
withholds them once the kernel's sources differ from the captured ones."""
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _prof(block_ops, busy_ms, launches, convert_launches=1, ozaki_launches=0):
    z = {"launches": 0, "sum_ms": 0.0, "busy_ms": 0.0, "ops": 0.0, "bytes": 0.0}
    return {"simple": dict(z), "pass": dict(z), "gemv": dict(z),
            "block": {"launches": launches, "sum_ms": 2.5 * busy_ms, "busy_ms": busy_ms, "ops": block_ops,
                      "bytes": 0.0},
            "convert": dict(z, launches=convert_launches),
            "ozaki": dict(z, launches=ozaki_launches), "steps": 1}


def test_counts_match_the_sources():
    b = _bench()
    for kernel in ("block_fxc_kernel<2>", "block_fxc_kernel<4>"):
        rec = b.profile_record(kernel)
        assert rec is not None, kernel
        # instructions per multiply-add = warp instructions x 32 / multiply-adds
        runs = rec["launches_read_write_ns_warpinst"]
        inst = sum(r[3] for r in runs) / len(runs)
        assert abs(inst * 32 / rec["macs_per_launch"] - rec["inst_per_mac"]) < 1e-3
        assert rec["dram_bytes_per_launch"] <= rec["algorithmic_bytes_per_launch"]


def test_roofline_of_block_kernel():
    b = _bench()
    macs = 2401.0 * 256 ** 3  # one DD n = 4096 step at cutoff 256: 2401 leaves, 343 launches
    r = b.roofline_of(_prof(macs, 100.0, 343), 2)
    rec = b.profile_record("block_fxc_kernel<2>")
    want = macs / 0.100 * rec["inst_per_mac"]
    assert r["bound"] == "alu" and r["kernel"].startswith("block_fxc_kernel<2>")
    assert abs(r["achieved"] - want / 1e12) < 1e-9 * want
    assert abs(r["frac"] - want / b.ISSUE_PEAK) < 1e-12
    assert r["traffic"] == rec["dram_bytes_per_launch"]
    assert abs(r["avg_launch_ms"] - 250.0 / 343) < 1e-12
    # tiles converted as staged: the per-tile kernel, whose counts are not committed
    r2 = b.roofline_of(_prof(macs, 100.0, 343, convert_launches=0), 2)
    assert r2["kernel"].startswith("block_fx_kernel<2>") and r2["frac"] is None


def test_stale_counts_are_withheld(tmp_path, monkeypatch):
    b = _bench()
    path = os.path.join(ROOT, "profiles", "block_fx_counts.json")
    data = json.load(open(path))
    data["block_fxc_kernel<2>"]["sources_sha256"] = "0" * 64
    fake_root = tmp_path
    os.makedirs(fake_root / "profiles")
    json.dump(data, open(fake_root / "profiles" / "block_fx_counts.json", "w"))
    for f in data["block_fxc_kernel<2>"]["sources"]:
        dst = fake_root / f
        os.makedirs(dst.parent, exist_ok=True)
        dst.write_bytes(open(os.path.join(ROOT, f), "rb").read())
    monkeypatch.setattr(b, "ROOT", str(fake_root))
    assert b.profile_record("block_fxc_kernel<2>") is None
    r = b.roofline_of(_prof(1e9, 1.0, 1), 2)
    assert r["achieved"] is None and r["frac"] is None and r["traffic"] is None


def test_roofline_of_int8_products():
    b = _bench()
    p = _prof(0.0, 0.0, 0, convert_launches=0, ozaki_launches=1)
    p["ozaki"].update(ops=2.0 * 4096 ** 3 * 32, busy_ms=30.0, sum_ms=30.0)
    r = b.roofline_of(p, 2)
    assert r["bound"] == "tensor"
    assert abs(r["frac"] - (2.0 * 4096 ** 3 * 32 / 0.030) / b.INT8_MMA_PEAK) < 1e-12
