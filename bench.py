#!/usr/bin/env python
"""Benchmark: DD / QD GEMM 2mnl/s at n = 4096 on one GB300.

One step = one C := A B through the C ABI (dd_gemm) with the headline
workload: DD Winograd, n = 4096, operands U[-1, 1) with a random lower limb
(inputs.uniform, seeds fixed in workloads.py). Inputs are resident in HBM
before the timed region; three 4096^2 DD matrices are 768 MiB, well above
the 129 MB L2, so no L2 flush is needed between steps.

Printed: one JSON line (rank 0) with the metric, the end-to-end number
through host buffers, the roofline of the dominant kernel (the Block base
case on the integer pipe, issue bound; its per-launch figures come from one
profiled step after the timed steps), the CPU oracle timed on a bounded
sample, clocks sampled during the timed region, and extra measurements (DD
Block, QD Winograd and Block, INT8 products, n = 8192, LU solves, batched).

--impl reference times the CPU oracle (the plain Simple triple loop) on the
host cores instead, on a bounded sample of the same workload per step.

Multi-GPU: replicas only (one independent product per rank, no exchange).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1510_08642_gb300 import workloads as WL  # noqa: E402

METRIC = "DD/QD GEMM 2mnl/s at n=4096 & % FP64-op roofline; served-request p50/p99 latency"
UNIT = "G 2mnl/s"
SM_COUNT = 152
FP64_PER_CLK_PER_SM = 2          # measured: DFMA throughput probe (profiles/fp64_int8_peaks.md)
SM_MAX_MHZ = 2070.0               # profiling recipe / MEASURED_PEAKS.json
FP64_PEAK = SM_COUNT * FP64_PER_CLK_PER_SM * SM_MAX_MHZ * 1e6  # FP64 instructions per second
PINNED_MAC_OPS = {2: 27, 4: 218}  # DD / QD multiply then add of the Simple kernel
INT8_MMA_PEAK = 1.50e14           # mma.sync m16n8k32 s8 ops/s, measured by the same probe


def _measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


_PEAKS = _measured_peaks()
# copy bandwidth and cuBLAS bf16 GEMM rate measured on the GB300s;
# without the file, the profiling recipe's fallback figures
HBM_GBS = float(_PEAKS.get("hbm_gbs", 6800.0))
BF16_PEAK = float(_PEAKS.get("bf16_tflops", 1900.0)) * 1e12
PEAK_NOTE = "of measured (MEASURED_PEAKS.json)" if _PEAKS else "of fallback (6.8 TB/s, 1.9 PFLOP/s bf16)"
ISSUE_PER_CLK_PER_SM = 4 * 32     # 4 schedulers x one warp instruction (32 lanes) per clock
ISSUE_PEAK = SM_COUNT * ISSUE_PER_CLK_PER_SM * SM_MAX_MHZ * 1e6  # thread instructions per second
IMAD_PER_CLK_PER_SM = 64          # measured: IMAD throughput probe (profiles/fp64_int8_peaks.md)
IMAD_PEAK = SM_COUNT * IMAD_PER_CLK_PER_SM * SM_MAX_MHZ * 1e6   # 32-bit integer multiply-adds per second
# The Block multiply-add's irreducible integer multiplies, counted from the
# source (the pre-shifted form, fx_pre.cuh, fx::mul_top_hi): of the W-word
# operands the partial products a_i b_j with i + j >= W, a mad.lo and a
# madc.hi each, and the high halves (mad.hi) of the W with i + j = W - 1:
# DD (W = 4) 6 x 2 + 4 = 16 IMAD, QD (W = 7) 21 x 2 + 7 = 49 IMAD.
IMAD_FLOOR_PER_MAC = {2: 16, 4: 49}
IMAD_FLOOR_SOURCE = {2: "fx::mul_top_hi<4>: 6 partial products x (mad.lo + madc.hi) + 4 x mad.hi",
                     4: "fx::mul_top_hi<7>: 21 partial products x (mad.lo + madc.hi) + 7 x mad.hi"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default=WL.DD_WINOGRAD_4096.name)
    p.add_argument("--cutoff", type=int, default=None)
    p.add_argument("--extras", choices=["all", "none"], default="all")
    p.add_argument("--cpu-seconds", type=float, default=12.0,
                   help="CPU oracle sample length; 0 skips the CPU baseline")
    p.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg")
    p.add_argument("--lu-k", type=int, default=256, help="LU block column width K")
    p.add_argument("--sweep-n", type=int, default=1024, help="lu_alpha_sweep: matrix order")
    p.add_argument("--requests", type=int, default=500, help="serving: requests per rate point")
    p.add_argument("--serve-rates", type=float, nargs="+", default=[0.5, 0.9],
                   help="the bench's serving leg: arrival rates as fractions of the saturation rate")
    p.add_argument("--rates", type=float, nargs="+", default=[0.25, 0.5, 0.75, 0.9, 1.1],
                   help="serving: arrival rates as fractions of the saturation rate")
    p.add_argument("--record-counts", metavar="CSV", default=None,
                   help="write the ncu counters of CSV (a --csv --print-units base capture of "
                        "COUNT_METRICS) for --kernel into profiles/block_fx_counts.json and exit")
    p.add_argument("--kernel", default=None, help="--record-counts: kernel, e.g. 'block_fxc_kernel<2>'")
    p.add_argument("--leaf", type=int, default=256, help="--record-counts: leaf order (seven leaves per launch)")
    p.add_argument("--command", default="", help="--record-counts: the command that made CSV")
    return p.parse_args()


def workload_by_name(name):
    if name == "serving":
        return WL.Workload("serving", 2, 0, "winograd", 512, 0, 0)
    for v in vars(WL).values():
        if isinstance(v, WL.Workload) and v.name == name:
            return v
    raise SystemExit(f"unknown workload {name}")


# ------------------------------------------------------------- distributed --
def dist_init(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl"
        try:
            import torch
            if not torch.cuda.is_available():
                backend = "gloo"
        except Exception:
            backend = "gloo"
        dist.init_process_group(backend)
    return world, rank, local, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x, device=None):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks --
def parse_clock_lines(lines):
    """(SM MHz, max SM MHz, the four throttle flags) per nvidia-smi CSV line
    of the Clocks query; malformed lines (a partial last line) are skipped."""
    rows = []
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
        except ValueError:
            continue
    return rows


class Clocks:
    """nvidia-smi sampling every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            rows = parse_clock_lines(f)
        os.unlink(self.path)
        return clock_summary(rows)


def clock_summary(rows):
    """The bench line's clocks: median SM clock under load, the largest
    maximum clock seen, the sample count and every throttle reason that was
    active in any sample (None without samples)."""
    if not rows:
        return None
    sm = sorted(r[0] for r in rows)
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
    return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(r[1] for r in rows),
            "samples": len(rows), "reasons": reasons}


# --------------------------------------------------------------- CPU leg ----
def cpu_oracle_rate(w, seconds, seed_rows=8):
    """Oracle Simple product on host cores over a row sample; 2mnl/s."""
    import numpy as np

    import oracle as O
    from paper_1510_08642_gb300 import inputs as I
    n, limbs = w.n, w.limbs
    B = I.uniform(n, n, limbs, seed=w.seed_b)
    A_all = I.uniform(n, n, limbs, seed=w.seed_a)
    cores = O.threads()
    r = seed_rows
    t0 = time.perf_counter()
    O.gemm_simple(np.ascontiguousarray(A_all[:, :r]), B, nthreads=cores)
    t_probe = time.perf_counter() - t0
    rows = int(max(cores, min(n, r * seconds / max(t_probe, 1e-3))))
    rows = max(cores, (rows // cores) * cores)
    t0 = time.perf_counter()
    O.gemm_simple(np.ascontiguousarray(A_all[:, :rows]), B, nthreads=cores)
    t = time.perf_counter() - t0
    macs = rows * n * n
    return {"value": 2.0 * macs / t / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{'DD' if limbs == 2 else 'QD'} Simple (Eq. 1 triple loop, pinned op order) "
                      f"rows 0..{rows - 1} of the n={n} product ({rows}x{n}x{n} multiply-adds), "
                      f"{t:.1f} s on {cores} threads"}


def run_reference(args, w):
    world, rank, local, dist = dist_init(args.gpus)
    if rank != 0:
        return 0
    import numpy as np

    import oracle as O
    from paper_1510_08642_gb300 import inputs as I
    n, limbs = w.n, w.limbs
    B = I.uniform(n, n, limbs, seed=w.seed_b)
    A = I.uniform(n, n, limbs, seed=w.seed_a)
    cores = O.threads()
    # size one step to ~ (a few minutes / (K + W)) of work
    budget = max(2.0, min(20.0, 150.0 / (args.steps + args.warmup)))
    t0 = time.perf_counter()
    O.gemm_simple(np.ascontiguousarray(A[:, :cores]), B, nthreads=cores)
    t_probe = time.perf_counter() - t0
    rows = int(max(cores, min(n, cores * budget / max(t_probe, 1e-3))))
    rows = max(cores, (rows // cores) * cores)
    Ar = np.ascontiguousarray(A[:, :rows])
    for _ in range(args.warmup):
        O.gemm_simple(Ar, B, nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.gemm_simple(Ar, B, nthreads=cores)
    t = (time.perf_counter() - t0) / args.steps
    v = 2.0 * rows * n * n / t / 1e9
    sample = (f"{'DD' if limbs == 2 else 'QD'} Simple oracle, rows 0..{rows - 1} of the n={n} "
              f"product per step ({rows}x{n}x{n} multiply-adds)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w.name, "n": n, "limbs": limbs, "algo": "simple (CPU oracle)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ ncu counts --
# Counters captured per Block leaf-node launch (one pass each is not needed:
# the capture runs on a small workload, three launches).
COUNT_METRICS = ("dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum,smsp__inst_executed.sum,"
                 "sm__inst_executed_pipe_fma.sum,sm__inst_executed_pipe_alu.sum")
COUNT_SOURCES = ["paper_1510_08642_gb300/csrc/block_fx.cu", "paper_1510_08642_gb300/csrc/fx.cuh",
                 "paper_1510_08642_gb300/csrc/fx_round.cuh", "paper_1510_08642_gb300/csrc/fx_rescue.cuh",
                 "paper_1510_08642_gb300/csrc/fx_pre.cuh",
                 "paper_1510_08642_gb300/csrc/arith.cuh", "paper_1510_08642_gb300/csrc/kernels.cuh"]


def sources_hash(files):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()


def parse_ncu_csv(path, kernel):
    """Per-launch metric values of the launches of `kernel` in an ncu --csv
    log (one row per launch and metric), base units."""
    import csv
    scale = {"byte": 1.0, "kbyte": 1e3, "mbyte": 1e6, "gbyte": 1e9, "nsecond": 1.0, "ns": 1.0, "usecond": 1e3, "us": 1e3,
             "msecond": 1e6, "second": 1e9, "inst": 1.0, "kinst": 1e3, "minst": 1e6, "ginst": 1e9, "": 1.0}
    lines = open(path).read().splitlines()
    start = next(i for i, ln in enumerate(lines) if ln.startswith('"ID"'))
    launches = {}
    for row in csv.DictReader(lines[start:]):
        name = row["Kernel Name"].replace(" ", "")
        if kernel.replace(" ", "") not in name:
            continue
        v = float(row["Metric Value"].replace(",", "")) * scale[row["Metric Unit"].strip().lower()]
        launches.setdefault(int(row["ID"]), {})[row["Metric Name"]] = v
    return [launches[k] for k in sorted(launches)]


def record_counts(args):
    """Turn an ncu capture of Block leaf-node launches into the counts record
    the bench's roofline uses (per launch: seven leaf products of order
    --leaf), stamped with the hash of the kernel's current sources."""
    limbs = 2 if args.kernel.endswith("<2>") else 4
    runs = parse_ncu_csv(args.record_counts, args.kernel.split("<")[0] + "<" + str(limbs) + ">")
    if not runs:
        raise SystemExit(f"no launches of {args.kernel} in {args.record_counts}")
    macs = 7 * args.leaf ** 3
    mean = {k: sum(r[k] for r in runs) / len(runs) for k in runs[0]}
    rec = {
        "what": f"one launch of the seven {args.leaf}^3 {'DD' if limbs == 2 else 'QD'} Winograd leaf products "
                f"of a node, on converted operands, ncu",
        "command": args.command,
        "launches_read_write_ns_warpinst": [[r["dram__bytes_read.sum"], r["dram__bytes_write.sum"],
                                             r["gpu__time_duration.sum"], r["smsp__inst_executed.sum"]]
                                            for r in runs],
        "macs_per_launch": macs,
        "inst_per_mac": round(mean["smsp__inst_executed.sum"] * 32 / macs, 3),
        "fma_pipe_per_mac": round(mean.get("sm__inst_executed_pipe_fma.sum", 0.0) * 32 / macs, 3),
        "alu_pipe_per_mac": round(mean.get("sm__inst_executed_pipe_alu.sum", 0.0) * 32 / macs, 3),
        "dram_bytes_per_launch": round(mean["dram__bytes_read.sum"] + mean["dram__bytes_write.sum"]),
        "algorithmic_bytes_per_launch": 7 * 3 * args.leaf ** 2 * 8 * limbs,
        "dram_note": "DRAM bytes per launch (seven leaves): the 14 converted leaf operands read once; the "
                     "seven C leaves are still in L2 when the launch ends; algorithmic = A, B, C of the seven "
                     "products as DD / QD",
        "sources": COUNT_SOURCES,
        "sources_sha256": sources_hash(COUNT_SOURCES),
    }
    path = os.path.join(ROOT, "profiles", "block_fx_counts.json")
    try:
        allrec = json.load(open(path))
    except (OSError, ValueError):
        allrec = {}
    allrec[args.kernel] = rec
    with open(path, "w") as f:
        json.dump(allrec, f, indent=1)
        f.write("\n")
    print(json.dumps({args.kernel: {k: rec[k] for k in ("inst_per_mac", "fma_pipe_per_mac", "alu_pipe_per_mac",
                                                        "dram_bytes_per_launch")}}))
    return 0


# ----------------------------------------------------------------- GPU leg --
def profile_record(kernel: str):
    """The committed ncu counters of a Block leaf launch (profiles/block_fx_counts.json),
    or None when the kernel's sources changed since they were taken."""
    path = os.path.join(ROOT, "profiles", "block_fx_counts.json")
    try:
        rec = json.load(open(path))[kernel]
        if sources_hash(rec["sources"]) != rec["sources_sha256"]:
            return None
        return rec
    except (OSError, KeyError, ValueError):
        return None


def roofline_of(prof, limbs):
    """Dominant kernel: the tcgen05 residue products (BF16 operations against
    the measured bf16 GEMM rate), the INT8 GEMM (INT8 operations against the
    measured mma.sync peak) or the Block base case (its irreducible IMAD
    count per multiply-add against the IMAD pipe, plus the issue-slot use
    from the committed ncu counts)."""
    tc = prof.get("tensor")
    if tc and tc["launches"]:
        achieved = tc["ops"] / (tc["busy_ms"] * 1e-3)
        return {"bound": "tensor", "kernel": "crt_tc_kernel (tcgen05.mma kind::f16, BF16 residues, FP32 in "
                                             "tensor memory, TMA operands)",
                "achieved": achieved / 1e12, "peak": BF16_PEAK / 1e12, "unit": "T BF16-op/s",
                "frac": achieved / BF16_PEAK, "traffic": None,
                "peak_source": f"bf16_tflops {PEAK_NOTE}: cuBLAS bf16 GEMM, burst (the kernel is timed alone)",
                "algorithmic": "2 x N moduli x m l n (padded to 128 x 64 x 128) BF16 multiply-adds per product",
                "launches": int(tc["launches"]), "avg_launch_ms": tc["sum_ms"] / tc["launches"],
                "busy_ms": tc["busy_ms"]}
    oz = prof.get("ozaki")
    if oz and oz["launches"]:
        achieved = oz["ops"] / (oz["busy_ms"] * 1e-3)
        return {"bound": "tensor", "kernel": "oz_gemm_kernel (INT8 mma.sync m16n8k32)",
                "achieved": achieved / 1e12, "peak": INT8_MMA_PEAK / 1e12, "unit": "T INT8-op/s",
                "frac": achieved / INT8_MMA_PEAK, "traffic": None,
                "peak_source": "measured: mma.sync s8 throughput probe (tcgen05 has no INT8 kind on "
                               "sm_103a; MEASURED_PEAKS.json has no INT8 figure)",
                "launches": int(oz["launches"]), "avg_launch_ms": oz["sum_ms"] / oz["launches"],
                "busy_ms": oz["busy_ms"]}
    b = prof["block"]
    if not b["launches"]:
        return None
    macs_per_s = b["ops"] / (b["busy_ms"] * 1e-3)  # kind 1 counts multiply-adds
    avg_ms = b["sum_ms"] / b["launches"]
    # operands converted once per product (kind 5 launches) or per staged tile
    kernel = f"block_fxc_kernel<{limbs}>" if prof.get("convert", {}).get("launches") else f"block_fx_kernel<{limbs}>"
    rec = profile_record(kernel)
    # algorithmic: the multiply-adds' irreducible IMAD count against the IMAD
    # pipe (64 per clock per SM); independent of how many other instructions
    # the kernel issues
    floor = IMAD_FLOOR_PER_MAC[limbs]
    achieved = macs_per_s * floor
    out = {"bound": "alu", "kernel": f"{kernel} (multiply-add on the integer pipe, no FP64)",
           "achieved": achieved / 1e12, "peak": IMAD_PEAK / 1e12, "unit": "T IMAD/s",
           "frac": achieved / IMAD_PEAK,
           "peak_source": f"derived: {SM_COUNT} SMs x {IMAD_PER_CLK_PER_SM} IMAD per clock per SM (measured "
                          f"by the IMAD throughput probe) x {SM_MAX_MHZ:.0f} MHz",
           "algorithmic": f"{floor} IMAD per {'DD' if limbs == 2 else 'QD'} multiply-add "
                          f"({IMAD_FLOOR_SOURCE[limbs]}) x multiply-adds per busy second",
           "macs_per_s": macs_per_s, "launches": int(b["launches"]), "avg_launch_ms": avg_ms,
           "busy_ms": b["busy_ms"], "sum_launch_ms": b["sum_ms"]}
    if rec is None:
        out.update({"traffic": None, "note": "kernel sources changed since the committed ncu counts"})
        return out
    issued = macs_per_s * rec["inst_per_mac"]
    out.update({"traffic": rec.get("dram_bytes_per_launch"),
                "traffic_note": rec.get("dram_note"),
                "issue": {"inst_per_mac": rec["inst_per_mac"], "achieved": issued / 1e12,
                          "peak": ISSUE_PEAK / 1e12, "unit": "T thread-instr/s", "frac": issued / ISSUE_PEAK,
                          "note": "issue slots used (grows with extra instructions; not algorithmic)"},
                "fma_pipe_per_mac": rec.get("fma_pipe_per_mac"),
                "alu_pipe_per_mac": rec.get("alu_pipe_per_mac"),
                "counts_source": "profiles/block_fx_counts.json (ncu, same sources)"})
    return out


def time_gpu(P, torch, w, dA, dB, dC, cutoff, steps, warmup, stream, dist=None, device=None,
             profile=True):
    """`steps` timed steps (CUDA events on the stream, no per-launch events),
    then, with `profile`, steps under the library's launch profile (events
    around every launch, for the per-kernel figures): the first creates the
    profile's events, the second, reusing them, is the one reported."""
    from paper_1510_08642_gb300 import capi
    kw = dict(algo=w.algo, cutoff=cutoff, slices=w.slices)
    for _ in range(warmup):
        P.gemm(dA, dB, dC, **kw)
    torch.cuda.synchronize()
    barrier(dist)
    torch.cuda.synchronize()
    launches0 = capi.ddg_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        P.gemm(dA, dB, dC, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    launches = capi.ddg_kernel_launches() - launches0
    ms = e0.elapsed_time(e1) / steps
    ms = max_over_ranks(dist, ms, device)
    prof = None
    if profile:
        for _ in range(2):
            capi.ddg_profile_begin()
            P.gemm(dA, dB, dC, **kw)
            torch.cuda.synchronize()
            prof = capi.ddg_profile_end()
        prof["steps"] = 1
        if w.algo in ("winograd", "strassen"):
            # the quadrant passes timed alone: one more step with the seven
            # sub-products in order on one stream, so that no pass shares the
            # GPU with a leaf product of another stream
            capi.ddg_profile_begin()
            P.gemm(dA, dB, dC, streams=1, **kw)
            torch.cuda.synchronize()
            iso = capi.ddg_profile_end()
            prof["pass_isolated"] = iso["pass"]
            prof["convert_isolated"] = iso["convert"]
    return ms, prof, launches


def pass_and_conversion_rates(prof):
    """The fused quadrant passes' and the operand conversions' rates:
    algorithmic bytes (and sums / converted elements) over the sum of their
    launch durations, from the profiled step with the sub-products in order
    on one stream where there is one (none of their launches overlaps
    another kernel there), else from the profiled step itself (a Block
    product forks nothing)."""
    out = {}
    for kind, name, rate in (("pass", "passes", "sums_per_s"), ("convert", "conversions", "elements_per_s")):
        iso = prof.get(kind + "_isolated")
        k = iso if iso is not None else prof[kind]
        if not k["launches"] or k["sum_ms"] <= 0:
            continue
        sec = k["sum_ms"] * 1e-3
        out[name] = {"launches": int(k["launches"]), "sum_ms": k["sum_ms"],
                     "GB_per_s": k["bytes"] / sec / 1e9, "hbm_frac": k["bytes"] / sec / 1e9 / HBM_GBS,
                     rate: k["ops"] / sec,
                     "measured": "algorithmic bytes over the sum of the launch durations, in a profiled step "
                                 + ("with the sub-products on one stream (no launch overlaps another kernel)"
                                    if iso is not None else "of a product that forks nothing")}
    return out


def run_e2e(P, torch, w, args, dist, device, stream, hA, hB, hC, dA, dB, dC, cutoff, world):
    """Same metric through host buffers: every step copies A and B from pinned
    host memory, runs the product and reads C back, all inside the timed
    region. Two device buffer sets and two copy streams pipeline the steps:
    the inputs of step i + 1 are copied in while step i's product runs, and
    step i's C is read back while step i + 1 runs."""
    h2d = torch.cuda.Stream(device)
    d2h = torch.cuda.Stream(device)
    sets = [(dA, dB, dC, hC),
            (torch.empty_like(dA), torch.empty_like(dB), torch.empty_like(dC), torch.empty_like(hC).pin_memory())]
    barrier(dist)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    computed = [None, None]  # product of the last step that used the set
    read = [None, None]      # read-back of that step's C
    e0.record(stream)
    h2d.wait_event(e0)
    for i in range(args.steps):
        k = i % 2
        xA, xB, xC, yC = sets[k]
        with torch.cuda.stream(h2d):
            if computed[k] is not None:
                h2d.wait_event(computed[k])  # the product two steps back has read xA, xB
            xA.copy_(hA, non_blocking=True)
            xB.copy_(hB, non_blocking=True)
            ready = torch.cuda.Event()
            ready.record(h2d)
        stream.wait_event(ready)
        if read[k] is not None:
            stream.wait_event(read[k])  # xC of two steps back has been read
        P.gemm(xA, xB, xC, algo=w.algo, cutoff=cutoff)
        computed[k] = torch.cuda.Event()
        computed[k].record(stream)
        with torch.cuda.stream(d2h):
            d2h.wait_event(computed[k])
            yC.copy_(xC, non_blocking=True)
            read[k] = torch.cuda.Event()
            read[k].record(d2h)
    for k in range(2):
        if read[k] is not None:
            stream.wait_event(read[k])
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    ms_e2e = max_over_ranks(dist, e0.elapsed_time(e1) / args.steps, device)
    del sets
    return {"value": world * 2.0 * w.macs / (ms_e2e * 1e-3) / 1e9, "unit": UNIT,
            "h2d_bytes_per_step": int(hA.numel() * 8 + hB.numel() * 8),
            "d2h_bytes_per_step": int(hC.numel() * 8), "ms_per_step": ms_e2e,
            "pipelined": "two buffer sets: the copies of one step overlap the product of the next / previous"}


def time_lu(P, torch, w, device, stream, K):
    """Section 4 solve: dd_getrf / qd_getrf (Winograd trailing updates) +
    dd_getrs / qd_getrs, b = A 1."""
    from paper_1510_08642_gb300 import inputs as I
    n = w.n
    A0 = torch.from_numpy(I.uniform(n, n, w.limbs, seed=w.seed_a)).to(device)
    ones = torch.zeros((w.limbs, n, 1), dtype=torch.float64, device=device)
    ones[0] = 1.0
    b0 = P.gemm(A0, ones, algo="block")
    times = []
    for it in range(4):  # one warm-up, three timed (median reported)
        A = A0.clone()
        b = b0.clone()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ipiv = P.getrf(A, K=K, pivot=True, algo=w.algo, cutoff=w.cutoff)
        P.getrs(A, ipiv, b)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = sorted(times[1:])[len(times[1:]) // 2]
    err = float((b[0] - 1.0 + b[1:].sum(dim=0)).abs().max().item())
    rows = sample_rows(n, 24, seed=7)
    chk = {"name": w.name, "kind": "lu", "limbs": w.limbs, "n": n,
           "A_rows": A0[:, rows, :].cpu().numpy(), "b_rows": b0[:, rows, :].cpu().numpy(),
           "x": b.cpu().numpy(), "normA_inf": float(A0[0].abs().sum(dim=1).max().item())}
    return ({"value": (2.0 * n ** 3 / 3.0) / (ms * 1e-3) / 1e9, "unit": "G 2mnl/s (2n^3/3 per solve)",
             "ms": ms, "K": K, "cutoff": w.cutoff, "pivot": "partial", "steps": len(times) - 1, "warmup": 1,
             "max_abs_err_x_minus_1": err}, chk)


def time_batched(P, torch, device, stream, count=1000, reps=3, tune_buckets=8):
    """The batched workload: `count` products, m, l, n log-uniform in
    [32, 1024], 70% DD / 30% QD, one batch plan replayed as a CUDA graph.
    Operands are views into one resident 1024^2 pool per limb count (A and B
    may be shared between problems; every C is its own)."""
    import numpy as np

    from paper_1510_08642_gb300 import autotune, inputs as I
    dims = I.log_uniform_dims(count, 32, 1024, seed=4)
    kind = I.uniform01(5, count)
    off = I.splitmix64(6, 4 * count).reshape(count, 4)
    pools = {L: torch.from_numpy(I.uniform(1024, 1024, L, seed=200 + L)).to(device) for L in (2, 4)}
    # the autotuner's table, built here (outside the timed region) for the
    # shape buckets that carry the most work; the others use its model
    tuner = autotune.Tuner(os.path.join(tempfile.mkdtemp(), "tune.json"))
    kinds = [4 if kind[t] < 0.3 else 2 for t in range(count)]
    work_by_bucket = {}
    for t in range(count):
        m, l, n = (int(x) for x in dims[t])
        key = (kinds[t],) + tuple(1 << int(round(np.log2(x))) for x in (m, l, n))
        work_by_bucket[key] = work_by_bucket.get(key, 0.0) + 2.0 * m * l * n
    top = sorted(work_by_bucket, key=lambda k: -work_by_bucket[k])[:tune_buckets]
    t_tune = time.perf_counter()
    for key in top:
        tuner.tune(key[0], *(min(x, 1024) for x in key[1:]), copies=2, reps=2)
    t_tune = time.perf_counter() - t_tune
    tuner.save()
    probs, probs_host, keep, work = [], [], [], 0.0
    for t in range(count):
        m, l, n = (int(x) for x in dims[t])
        L = 4 if kind[t] < 0.3 else 2
        pool = pools[L]
        r0, c0 = int(off[t, 0] % (1025 - m)), int(off[t, 1] % (1025 - l))
        r1, c1 = int(off[t, 2] % (1025 - l)), int(off[t, 3] % (1025 - n))
        A = pool[:, r0:r0 + m, c0:c0 + l]
        B = pool[:, r1:r1 + l, c1:c1 + n]
        C = torch.empty((L, m, n), dtype=torch.float64, device=device)
        algo, cutoff = tuner.choose(L, m, l, n)
        probs.append(P.problem(A, B, C, algo, cutoff))
        probs_host.append((A, B))
        keep.append(C)
        work += 2.0 * m * l * n
    # plans, each replayed as a CUDA graph: the tuned recursion with the
    # operands of larger leaves converted once (default), the same with every
    # leaf in one persistent grouped launch (tiles converted as staged: the
    # same bits), and every problem as Block in that one launch (a single
    # kernel per run); the fastest is the bench's plan
    variants = {
        "tuned": (probs, False),
        "tuned_one_leaf_launch": (probs, True),
        "block_one_launch": ([P.problem(pr_A, pr_B, keep[t], "block", 512)
                              for t, (pr_A, pr_B) in enumerate(probs_host)], True),
    }
    timings = {}
    for name, (plist, one) in variants.items():
        b = P.Batch(plist, use_graph=True, one_launch=one)
        b.run(stream)  # warm-up (graph capture)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            b.run(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_v = e0.elapsed_time(e1) / reps
        timings[name] = {"ms": ms_v, "value": work / (ms_v * 1e-3) / 1e9,
                         "launches_per_run": b.stats["launches_per_run"]}
        b.close()
    best = min(timings, key=lambda k: timings[k]["ms"])
    plist, one = variants[best]
    batch = P.Batch(plist, use_graph=True, one_launch=one)
    batch.run(stream)
    torch.cuda.synchronize()
    # host copies for the CPU leg's oracle check of a few results (the four
    # largest problems of each limb count): their operands and 6 x 6 sampled
    # entries
    checks = []
    for L in (2, 4):
        idx = sorted((t for t in range(count) if kinds[t] == L), key=lambda t: -float(np.prod(dims[t])))[:4]
        for t in idx:
            hA = probs_host[t][0].cpu().numpy()
            hB = probs_host[t][1].cpu().numpy()
            checks.append(sample_for_check(f"batched problem {t}", hA, hB, keep[t], torch))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        batch.run(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    st = dict(batch.stats)
    batch.close()
    return ({"value": work / (ms * 1e-3) / 1e9, "unit": UNIT, "ms": ms, "problems": count,
            "plan": best, "plans": timings,
            "launches_per_run": st["launches_per_run"], "leaf_tiles": st["leaf_tiles"],
            "workspace_bytes": st["workspace_bytes"], "graph": True, "steps": reps, "warmup": 1,
            "tuning_table": os.path.exists(tuner.path),
            "tuned": {f"{'DD' if k[0] == 2 else 'QD'} {k[1]}x{k[2]}x{k[3]}": tuner.choose(*k) for k in top},
            "tuned_work_share": sum(work_by_bucket[k] for k in top) / sum(work_by_bucket.values()),
            "tuning_seconds": t_tune}, checks)


def sample_rows(n, count, seed):
    """`count` distinct sampled indices in [0, n), always with 0 and n - 1."""
    import numpy as np
    rng = np.random.default_rng(seed)
    idx = set(int(x) for x in rng.choice(n, size=min(n, count), replace=False))
    idx |= {0, n - 1}
    return np.array(sorted(idx), dtype=np.int64)


def sample_for_check(name, hA, hB, dC, torch):
    """Host copies of what the oracle needs to check 8 x 8 sampled entries of
    the product C = A B: those rows of A, columns of B and entries of C."""
    import numpy as np
    m, n = hA.shape[1], hB.shape[2]
    rows, cols = sample_rows(m, 6, seed=1), sample_rows(n, 6, seed=2)
    r_t = torch.as_tensor(rows, device=dC.device)
    c_t = torch.as_tensor(cols, device=dC.device)
    C = dC.index_select(1, r_t).index_select(2, c_t).cpu().numpy()
    return {"name": name, "kind": "gemm", "limbs": hA.shape[0], "m": m, "n": n,
            "A_rows": np.ascontiguousarray(hA[:, rows, :]), "B_cols": np.ascontiguousarray(hB[:, :, cols]),
            "C": C, "normA": float(np.linalg.norm(hA[0])), "normB": float(np.linalg.norm(hB[0]))}


def cpu_oracle_check(checks):
    """The oracle's exact error of each sampled result (CPU leg, outside any
    timed region): for products, the normwise error estimated from the
    sampled entries (RMS error x sqrt(m n) / (||A||_F ||B||_F)) and the
    largest elementwise error over sum_k |a_ik b_kj| in units of u^2
    (2^-106 DD, 2^-212 QD); for LU solves, the exact residual of sampled
    rows over ||A||_inf ||x||_inf and the bound n 2^-100 (QD: n 2^-200)."""
    import numpy as np

    import oracle as O
    out = {}
    for c in checks:
        if c["kind"] == "gemm":
            A, B, C = c["A_rows"], c["B_cols"], c["C"]
            err = O.gemm_error(A, B, C)
            mn = float(c.get("m", c["n"])) * c["n"]
            nw = float(np.sqrt(np.mean(err ** 2) * mn) / (c["normA"] * c["normB"]))
            u2 = 2.0 ** -106 if c["limbs"] == 2 else 2.0 ** -212
            scale = np.abs(A[0]) @ np.abs(B[0])
            ew = float(np.max(np.abs(err) / (scale * u2)))
            out[c["name"]] = {"sampled_entries": int(err.size), "normwise_est": nw,
                              "normwise_est_log2": float(np.log2(nw)) if nw > 0 else None,
                              "max_elementwise_over_u2": ew, "max_abs_err": float(np.abs(err).max())}
        else:
            A, b, x = c["A_rows"], c["b_rows"], c["x"]
            r = O.gemm_error(A, x, b)  # A x - b for the sampled rows, exact
            rel = float(np.abs(r).max() / (c["normA_inf"] * np.abs(x[0]).max()))
            bound = c["n"] * (2.0 ** -100 if c["limbs"] == 2 else 2.0 ** -200)
            out[c["name"]] = {"sampled_rows": int(A.shape[1]), "residual_rel": rel, "bound": bound,
                              "within_bound": rel <= bound}
    return out


def cutoff_sweep(P, torch, device, stream, orders=(1024, 2048, 4096), cutoffs=(64, 128, 256, 512, 1024)):
    """The Winograd cutoff sweep of the square workloads (Section 3's n_min):
    G 2mnl/s, DD and QD, 1 warm-up + 3 timed steps per point."""
    from paper_1510_08642_gb300 import inputs as I
    out = {}
    for limbs in (2, 4):
        key = "dd" if limbs == 2 else "qd"
        out[key] = {}
        for n in orders:
            XA = torch.from_numpy(I.uniform(n, n, limbs, seed=130 + n)).to(device)
            XB = torch.from_numpy(I.uniform(n, n, limbs, seed=131 + n)).to(device)
            XC = torch.empty((limbs, n, n), dtype=torch.float64, device=device)
            row = {}
            for cut in cutoffs:
                xw = WL.Workload(f"sweep_{key}_{n}_{cut}", limbs, n, "winograd", cut, 0, 0)
                ms, _, _ = time_gpu(P, torch, xw, XA, XB, XC, cut, 3, 1, stream, profile=False)
                row[str(cut)] = round(2.0 * n ** 3 / (ms * 1e-3) / 1e9, 1)
            out[key][str(n)] = row
            del XA, XB, XC
            torch.cuda.empty_cache()
    out["unit"] = UNIT
    return out


def time_serving(args):
    """The serving leg: saturation rate and p50 / p99 latency per request
    type at two arrival rates (fractions of saturation), args.requests
    requests per point (Poisson arrivals, 50% DD GEMM n log-uniform in
    [256, 2048], 50% DD LU solves n in {1024, 2048, 4096})."""
    from paper_1510_08642_gb300 import serving as S
    srv = S.Server(slots=4, hbm_budget=96 << 30, max_batch=32, gemm_cutoff=512, lu_K=256, lu_cutoff=512)
    t0 = time.perf_counter()
    res = S.sweep(rates=tuple(args.serve_rates), count=args.requests, seed=3, server=srv)
    srv.close()
    res["requests_per_point"] = args.requests
    res["wall_s"] = time.perf_counter() - t0
    return res


def run_ours(args, w):
    import numpy as np
    import torch

    world, rank, local, dist = dist_init(args.gpus)
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    import paper_1510_08642_gb300 as P
    from paper_1510_08642_gb300 import capi, inputs as I
    capi.load()
    cutoff = args.cutoff or w.cutoff
    n, limbs = w.n, w.limbs
    A = I.uniform(n, n, limbs, seed=w.seed_a)
    B = I.uniform(n, n, limbs, seed=w.seed_b)
    hA = torch.from_numpy(A).pin_memory()
    hB = torch.from_numpy(B).pin_memory()
    hC = torch.empty((limbs, n, n), dtype=torch.float64).pin_memory()
    dA = hA.to(device)
    dB = hB.to(device)
    dC = torch.empty((limbs, n, n), dtype=torch.float64, device=device)
    stream = torch.cuda.current_stream(device)

    clocks = Clocks(local)
    # -------- timed region: device-resident inputs
    for _ in range(args.warmup):
        P.gemm(dA, dB, dC, algo=w.algo, cutoff=cutoff, slices=w.slices)
    torch.cuda.synchronize()
    clocks.start()
    ms, prof, launches = time_gpu(P, torch, w, dA, dB, dC, cutoff, args.steps, 0, stream, dist, device)
    clk = clocks.stop()
    macs = w.macs
    value = world * 2.0 * macs / (ms * 1e-3) / 1e9

    # -------- end to end through host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(P, torch, w, args, dist, device, stream, hA, hB, hC, dA, dB, dC, cutoff, world)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n": n, "limbs": limbs, "algo": w.algo, "cutoff": cutoff,
                       "streams": 7, "distribution": "uniform: hi U[-1,1), lo hi*2^-53*U[-1/2,1/2)",
                       "l2": "no flush: A, B, C resident are 768 MiB (DD) > 129 MB L2",
                       "parallelism": f"replicas x{world}"},
            "clocks": clk, "e2e": e2e, "gpu_launches": int(launches)}
    line["roofline"] = roofline_of(prof, limbs)
    if line["roofline"]:
        line["roofline"]["measured"] = ("CUDA events around every launch on its own stream, in a profiled "
                                        "step after the timed steps (value is timed without them)")
    line["fp64_roofline_2mnl"] = {
        "value": 2.0 * FP64_PEAK / PINNED_MAC_OPS[limbs] / 1e9,
        "frac": value / world / (2.0 * FP64_PEAK / PINNED_MAC_OPS[limbs] / 1e9),
        "note": "2 x FP64 peak / FP64 instructions of the pinned multiply-add (DD 27, QD 218)"}
    line.update(pass_and_conversion_rates(prof))
    dC_keep = dC
    del dA, dB, hA, hB, hC
    torch.cuda.empty_cache()

    # -------- extras (single-GPU run only; 1 warm-up, 3 timed steps each)
    checks = []
    if args.extras == "all" and world == 1 and w.name == WL.DD_WINOGRAD_4096.name:
        extras = {}
        for xw in (WL.DD_BLOCK_4096, WL.QD_WINOGRAD_4096, WL.QD_BLOCK_4096, WL.DD_WINOGRAD_3000,
                   WL.QD_WINOGRAD_3000, WL.DD_OZAKI_4096_S16, WL.DD_OZAKI_4096_S13, WL.DD_WINOGRAD_8192,
                   WL.DD_OZAKI_8192_S16, WL.QD_OZAKI_4096_S32, WL.DD_OZAKI2_4096_N32, WL.DD_OZAKI2_8192_N32,
                   WL.DD_OZAKI2TC_4096_N32, WL.DD_OZAKI2TC_8192_N32):
            hXA = I.uniform(xw.n, xw.n, xw.limbs, seed=xw.seed_a)
            hXB = I.uniform(xw.n, xw.n, xw.limbs, seed=xw.seed_b)
            XA, XB = torch.from_numpy(hXA).to(device), torch.from_numpy(hXB).to(device)
            XC = torch.empty((xw.limbs, xw.n, xw.n), dtype=torch.float64, device=device)
            xms, xprof, _ = time_gpu(P, torch, xw, XA, XB, XC, xw.cutoff, 3, 1, stream)
            extras[xw.name] = {"value": 2.0 * xw.macs / (xms * 1e-3) / 1e9, "unit": UNIT, "ms": xms,
                               "roofline": roofline_of(xprof, xw.limbs), "steps": 3, "warmup": 1}
            checks.append(sample_for_check(xw.name, hXA, hXB, XC, torch))
            del XA, XB, XC, hXA, hXB
            torch.cuda.empty_cache()
        extras["cutoff_sweep"] = cutoff_sweep(P, torch, device, stream)
        for lw in (WL.DD_LU_4096, WL.DD_LU_4096_OZ2, WL.DD_LU_4096_OZ2TC, WL.QD_LU_2048):
            extras[lw.name], chk = time_lu(P, torch, lw, device, stream, K=256)
            checks.append(chk)
        extras["batched_1000_mixed"], bchecks = time_batched(P, torch, device, stream)
        checks += bchecks
        extras["serving"] = time_serving(args)
        line["extras"] = extras
    if checks:
        checks.insert(0, sample_for_check(w.name, A, B, dC_keep, torch))

    del dC_keep
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        # the CPU leg: the oracle timed on host cores (DD, and QD on the QD
        # workload), then the oracle's exact error of every sampled result
        line["cpu_baseline"] = cpu_oracle_rate(w, args.cpu_seconds)
        line["cpu_baseline"]["qd"] = cpu_oracle_rate(WL.QD_WINOGRAD_4096, args.cpu_seconds / 2)
        if checks:
            errs = cpu_oracle_check(checks)
            line["error_vs_oracle"] = errs[w.name]
            for name, e in errs.items():
                if name in line.get("extras", {}):
                    line["extras"][name]["error_vs_oracle"] = e
                elif name.startswith("batched problem") and "batched_1000_mixed" in line.get("extras", {}):
                    line["extras"]["batched_1000_mixed"].setdefault("error_vs_oracle", {})[name] = e
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_serving(args):
    """The serving workload: Poisson arrivals of DD GEMMs (n log-uniform in
    [256, 2048]) and DD LU solves (n in {1024, 2048, 4096}), 50 / 50, at
    fractions of the measured saturation rate; p50 / p99 latency per type."""
    import torch
    torch.cuda.set_device(0)
    from paper_1510_08642_gb300 import serving as S
    srv = S.Server(slots=4, hbm_budget=96 << 30, max_batch=32, gemm_cutoff=512, lu_K=256,
                   lu_cutoff=512)
    res = S.sweep(rates=tuple(args.rates), count=args.requests, seed=3, server=srv)
    srv.close()
    print(json.dumps({"workload": "serving_dd_gemm_lu_mix", "requests_per_point": args.requests, **res}),
          flush=True)
    return 0


def run_lu_only(args, w):
    """An LU workload as the timed step (for profiling the solve alone)."""
    import torch
    torch.cuda.set_device(0)
    device = torch.device("cuda", 0)
    import paper_1510_08642_gb300 as P
    from paper_1510_08642_gb300 import capi
    capi.load()
    stream = torch.cuda.current_stream(device)
    r, _ = time_lu(P, torch, w, device, stream, K=args.lu_k)
    print(json.dumps({"workload": w.name, **r}), flush=True)
    return 0


def run_lu_alpha_sweep(args):
    """Section 4 Fig. 5 setting: no pivoting, K = alpha n_min (alpha = 1..10,
    n_min = 32), random [-1, 1] matrix, x = [0, 1, ..., n-1], b = A x; time
    of dd_getrf + dd_getrs (and the QD pair) and the maximum relative error
    of x, with Winograd and Block trailing updates."""
    import torch
    torch.cuda.set_device(0)
    device = torch.device("cuda", 0)
    import paper_1510_08642_gb300 as P
    from paper_1510_08642_gb300 import capi, inputs as I
    capi.load()
    stream = torch.cuda.current_stream(device)
    n, nmin = args.sweep_n, 32
    rows = []
    for limbs in (2, 4):
        A0 = torch.from_numpy(I.uniform(n, n, limbs, seed=116)).to(device)
        X = torch.zeros((limbs, n, 1), dtype=torch.float64, device=device)
        X[0, :, 0] = torch.arange(n, dtype=torch.float64, device=device)
        b0 = P.gemm(A0, X, algo="block")
        for alpha in range(1, 11):
            for algo in ("winograd", "block"):
                K = alpha * nmin
                times = []
                for _ in range(2):  # one warm-up, one timed
                    A, b = A0.clone(), b0.clone()
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    ipiv = P.getrf(A, K=K, pivot=False, algo=algo, cutoff=nmin)
                    P.getrs(A, ipiv, b)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    times.append(e0.elapsed_time(e1))
                xi = X[0, 1:, 0]
                d = (b[0, 1:, 0] - xi) + b[1:, 1:, 0].sum(dim=0)
                rel = float((d.abs() / xi).max().item())
                rows.append({"limbs": limbs, "alpha": alpha, "K": K, "algo": algo, "ms": times[-1],
                             "max_rel_err": rel})
    print(json.dumps({"workload": "lu_alpha_sweep", "n": n, "n_min": nmin, "pivot": "none",
                      "matrix": "uniform [-1, 1], x = [0..n-1]", "points": rows}), flush=True)
    return 0


def run_batched_only(args):
    """The batched workload alone (tuning, one plan, timed replays)."""
    import torch
    torch.cuda.set_device(0)
    device = torch.device("cuda", 0)
    import paper_1510_08642_gb300 as P
    from paper_1510_08642_gb300 import capi
    capi.load()
    r, _ = time_batched(P, torch, device, torch.cuda.current_stream(device), reps=args.steps)
    print(json.dumps({"workload": "batched_1000_mixed", **r}), flush=True)
    return 0


def main():
    args = parse()
    if args.record_counts:
        return record_counts(args)
    if args.workload == "batched_1000_mixed":
        return run_batched_only(args)
    if args.workload == "lu_alpha_sweep":
        return run_lu_alpha_sweep(args)
    w = workload_by_name(args.workload)
    if args.impl == "reference":
        return run_reference(args, w)
    if w.name.startswith(("dd_lu", "qd_lu")):
        return run_lu_only(args, w)
    if w.name == "serving":
        return run_serving(args)
    return run_ours(args, w)


if __name__ == "__main__":
    sys.exit(main())
