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
    # algorithmic: 16 IMAD per DD multiply-add (the pre-shifted form's
    # mul_top_hi: 6 x (mad.lo + madc.hi) + 4 x mad.hi) against 152 x 64 x 2070 MHz
    want = macs / 0.100 * 16
    assert r["bound"] == "alu" and r["kernel"].startswith("block_fxc_kernel<2>")
    assert abs(r["achieved"] - want / 1e12) < 1e-9 * want
    assert abs(r["frac"] - want / (152 * 64 * 2070e6)) < 1e-12
    issued = macs / 0.100 * rec["inst_per_mac"]
    assert abs(r["issue"]["frac"] - issued / b.ISSUE_PEAK) < 1e-12
    assert r["traffic"] == rec["dram_bytes_per_launch"]
    assert abs(r["avg_launch_ms"] - 250.0 / 343) < 1e-12
    # QD: 49 IMAD per multiply-add (mul_top_hi<7>: 21 x 2 + 7)
    rq = b.roofline_of(_prof(macs, 100.0, 343), 4)
    assert abs(rq["frac"] - macs / 0.100 * 49 / (152 * 64 * 2070e6)) < 1e-12
    # tiles converted as staged: the per-tile kernel, whose counts are not committed
    r2 = b.roofline_of(_prof(macs, 100.0, 343, convert_launches=0), 2)
    assert r2["kernel"].startswith("block_fx_kernel<2>") and r2["traffic"] is None and "issue" not in r2


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
    # the algorithmic fraction needs no counts; the counter figures are withheld
    assert r["frac"] is not None and r["traffic"] is None and "issue" not in r


def test_roofline_of_int8_products():
    b = _bench()
    p = _prof(0.0, 0.0, 0, convert_launches=0, ozaki_launches=1)
    p["ozaki"].update(ops=2.0 * 4096 ** 3 * 32, busy_ms=30.0, sum_ms=30.0)
    r = b.roofline_of(p, 2)
    assert r["bound"] == "tensor"
    assert abs(r["frac"] - (2.0 * 4096 ** 3 * 32 / 0.030) / b.INT8_MMA_PEAK) < 1e-12


def test_oracle_check_of_sampled_results():
    """The CPU leg's sampled check: an exact product has zero error; a planted
    error of 2^-90 on one sampled entry shows in the elementwise ratio and
    the normwise estimate; an LU sample of an exact solution is in bound."""
    import numpy as np

    import oracle as O
    from paper_1510_08642_gb300 import inputs as I
    b = _bench()
    n = 64
    A = I.integer(n, n, 2, bits=10, seed=1)
    B = I.integer(n, n, 2, bits=10, seed=2)
    C = O.gemm_simple(A, B)  # integers: exact
    rows, cols = b.sample_rows(n, 6, seed=1), b.sample_rows(n, 6, seed=2)

    def chk(Cs):
        return {"name": "p", "kind": "gemm", "limbs": 2, "n": n, "A_rows": A[:, rows, :],
                "B_cols": B[:, :, cols], "C": Cs, "normA": float(np.linalg.norm(A[0])),
                "normB": float(np.linalg.norm(B[0]))}
    Cs = C[:, rows][:, :, cols].copy()
    out = b.cpu_oracle_check([chk(Cs)])["p"]
    assert out["max_abs_err"] == 0.0 and out["normwise_est"] == 0.0
    Cs[1, 0, 0] += 2.0 ** -90 * abs(Cs[0, 0, 0])
    out = b.cpu_oracle_check([chk(Cs)])["p"]
    assert out["max_abs_err"] > 0 and out["max_elementwise_over_u2"] > 2.0 ** 10
    X = np.zeros((2, n, 1))
    X[0] = 1.0
    Bv = O.gemm_simple(A, X)
    lu = {"name": "lu", "kind": "lu", "limbs": 2, "n": n, "A_rows": A[:, rows, :], "b_rows": Bv[:, rows, :],
          "x": X, "normA_inf": float(np.abs(A[0]).sum(axis=1).max())}
    r = b.cpu_oracle_check([lu])["lu"]
    assert r["residual_rel"] == 0.0 and r["within_bound"]


def test_pass_and_conversion_rates_from_the_one_stream_step():
    b = _bench()
    z = {"launches": 0, "sum_ms": 0.0, "busy_ms": 0.0, "ops": 0.0, "bytes": 0.0}
    prof = {"pass": dict(z, launches=300, sum_ms=40.0, busy_ms=9.0, bytes=8e9, ops=1e9),
            "convert": dict(z, launches=343, sum_ms=90.0, busy_ms=58.0, bytes=4e9, ops=3e8),
            "pass_isolated": dict(z, launches=300, sum_ms=10.0, busy_ms=10.0, bytes=8e9, ops=1e9),
            "convert_isolated": dict(z, launches=343, sum_ms=2.0, busy_ms=2.0, bytes=4e9, ops=3e8)}
    r = b.pass_and_conversion_rates(prof)
    # bytes over the summed durations of the one-stream step, not the overlapped seven-stream figures
    assert abs(r["passes"]["GB_per_s"] - 800.0) < 1e-9 and abs(r["conversions"]["GB_per_s"] - 2000.0) < 1e-9
    assert abs(r["conversions"]["elements_per_s"] - 1.5e11) < 1e-3 and r["passes"]["sums_per_s"] == 1e11
    assert abs(r["conversions"]["hbm_frac"] - 2000.0 / b.HBM_GBS) < 1e-12
    assert "one stream" in r["passes"]["measured"] and r["conversions"]["launches"] == 343
    # a Block product (nothing forks, no isolated step): its own profile; no passes
    block = {"pass": dict(z), "convert": dict(z, launches=2, sum_ms=0.5, busy_ms=0.5, bytes=1e9, ops=5e7)}
    r = b.pass_and_conversion_rates(block)
    assert set(r) == {"conversions"} and abs(r["conversions"]["GB_per_s"] - 2000.0) < 1e-9
    assert "forks nothing" in r["conversions"]["measured"]


def test_clock_samples_summarised():
    b = _bench()
    lines = ["0, 2070, 2070, 910.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
             "0, 1995, 2070, 1398.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
             "0, 2055, 2070, 1200.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
             "0, 2070, 20",  # a partial last line
             "[N/A], [N/A]\n"]
    rows = b.parse_clock_lines(lines)
    assert len(rows) == 3
    c = b.clock_summary(rows)
    assert c == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "samples": 3, "reasons": ["sw_power_cap"]}
    hot = b.parse_clock_lines(["0, 1500, 2070, 900, 0x48, Active, Active, Not Active, Not Active\n"])
    assert b.clock_summary(hot)["reasons"] == ["hw_slowdown", "hw_thermal_slowdown"]
    assert b.clock_summary([]) is None
