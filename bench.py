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
HBM_GBS = 6790.7                  # MEASURED_PEAKS.json hbm_gbs (copy bandwidth)
ISSUE_PER_CLK_PER_SM = 4 * 32     # 4 schedulers x one warp instruction (32 lanes) per clock
ISSUE_PEAK = SM_COUNT * ISSUE_PER_CLK_PER_SM * SM_MAX_MHZ * 1e6  # thread instructions per second


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
    p.add_argument("--requests", type=int, default=120, help="serving: requests per rate point")
    p.add_argument("--rates", type=float, nargs="+", default=[0.25, 0.5, 0.75, 0.9, 1.1],
                   help="serving: arrival rates as fractions of the saturation rate")
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
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
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


# ----------------------------------------------------------------- GPU leg --
def profile_record(kernel: str):
    """The committed ncu counters of a Block leaf launch (profiles/block_fx_counts.json),
    or None when the kernel's sources changed since they were taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "block_fx_counts.json")
    try:
        rec = json.load(open(path))[kernel]
        h = hashlib.sha256()
        for f in rec["sources"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        if h.hexdigest() != rec["sources_sha256"]:
            return None
        return rec
    except (OSError, KeyError, ValueError):
        return None


def roofline_of(prof, limbs):
    """Dominant kernel: the Block base case (thread instructions issued per
    busy second, from its multiply-adds and the committed ncu count of
    instructions per multiply-add, against the SM issue rate) or, for the
    INT8 products, the INT8 GEMM (INT8 ops against the measured mma.sync
    peak)."""
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
    out = {"bound": "alu", "kernel": f"{kernel} (multiply-add on the integer pipe, no FP64)",
           "peak": ISSUE_PEAK / 1e12, "unit": "T instr/s",
           "peak_source": f"derived: {SM_COUNT} SMs x 4 schedulers x 32 lanes (one warp instruction "
                          f"per scheduler per clock) x {SM_MAX_MHZ:.0f} MHz",
           "macs_per_s": macs_per_s, "launches": int(b["launches"]), "avg_launch_ms": avg_ms,
           "busy_ms": b["busy_ms"], "sum_launch_ms": b["sum_ms"]}
    if rec is None:
        out.update({"achieved": None, "frac": None, "traffic": None,
                    "note": "kernel sources changed since the committed ncu counts"})
        return out
    achieved = macs_per_s * rec["inst_per_mac"]
    out.update({"achieved": achieved / 1e12, "frac": achieved / ISSUE_PEAK,
                "inst_per_mac": rec["inst_per_mac"],
                "traffic": rec.get("dram_bytes_per_launch"),
                "traffic_note": rec.get("dram_note"),
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
    return ms, prof, launches


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
    for it in range(2):  # one warm-up, one timed
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
    ms = times[-1]
    err = float((b[0] - 1.0 + b[1:].sum(dim=0)).abs().max().item())
    return {"value": (2.0 * n ** 3 / 3.0) / (ms * 1e-3) / 1e9, "unit": "G 2mnl/s (2n^3/3 per solve)",
            "ms": ms, "K": K, "cutoff": w.cutoff, "pivot": "partial", "steps": 1, "warmup": 1,
            "max_abs_err_x_minus_1": err}


def time_batched(P, torch, device, stream, count=1000, reps=3):
    """The batched workload: `count` products, m, l, n log-uniform in
    [32, 1024], 70% DD / 30% QD, one batch plan replayed as a CUDA graph.
    Operands are views into one resident 1024^2 pool per limb count (A and B
    may be shared between problems; every C is its own)."""
    from paper_1510_08642_gb300 import autotune, inputs as I
    dims = I.log_uniform_dims(count, 32, 1024, seed=4)
    kind = I.uniform01(5, count)
    off = I.splitmix64(6, 4 * count).reshape(count, 4)
    pools = {L: torch.from_numpy(I.uniform(1024, 1024, L, seed=200 + L)).to(device) for L in (2, 4)}
    tuner = autotune.Tuner()
    probs, keep, work = [], [], 0.0
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
        keep.append(C)
        work += 2.0 * m * l * n
    batch = P.Batch(probs, use_graph=True)
    batch.run(stream)
    torch.cuda.synchronize()
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
    return {"value": work / (ms * 1e-3) / 1e9, "unit": UNIT, "ms": ms, "problems": count,
            "launches_per_run": st["launches_per_run"], "leaf_tiles": st["leaf_tiles"],
            "workspace_bytes": st["workspace_bytes"], "graph": True, "steps": reps, "warmup": 1,
            "tuning_table": os.path.exists(tuner.path)}


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
    passes = prof["pass"]
    if passes["launches"]:
        line["passes"] = {"launches": int(passes["launches"]), "busy_ms": passes["busy_ms"] / prof["steps"],
                          "GB_per_s": passes["bytes"] / (passes["busy_ms"] * 1e-3) / 1e9,
                          "hbm_frac": passes["bytes"] / (passes["busy_ms"] * 1e-3) / 1e9 / HBM_GBS,
                          "sums_per_s": passes["ops"] / (passes["busy_ms"] * 1e-3)}
    conv = prof["convert"]
    if conv["launches"]:
        line["conversions"] = {"launches": int(conv["launches"]), "busy_ms": conv["busy_ms"] / prof["steps"],
                               "GB_per_s": conv["bytes"] / (conv["busy_ms"] * 1e-3) / 1e9,
                               "hbm_frac": conv["bytes"] / (conv["busy_ms"] * 1e-3) / 1e9 / HBM_GBS,
                               "elements_per_s": conv["ops"] / (conv["busy_ms"] * 1e-3)}
    del dA, dB, dC, hA, hB, hC
    torch.cuda.empty_cache()

    # -------- extras (rank 0 of a single-GPU run only; 1 warm-up, 1 timed)
    if args.extras == "all" and world == 1 and w.name == WL.DD_WINOGRAD_4096.name:
        extras = {}
        for xw in (WL.DD_BLOCK_4096, WL.QD_WINOGRAD_4096, WL.QD_BLOCK_4096, WL.DD_OZAKI_4096_S16,
                   WL.DD_OZAKI_4096_S13, WL.DD_WINOGRAD_8192, WL.DD_OZAKI_8192_S16,
                   WL.QD_OZAKI_4096_S32, WL.DD_OZAKI2_4096_N32, WL.DD_OZAKI2_8192_N32):
            XA = torch.from_numpy(I.uniform(xw.n, xw.n, xw.limbs, seed=xw.seed_a)).to(device)
            XB = torch.from_numpy(I.uniform(xw.n, xw.n, xw.limbs, seed=xw.seed_b)).to(device)
            XC = torch.empty((xw.limbs, xw.n, xw.n), dtype=torch.float64, device=device)
            xms, xprof, _ = time_gpu(P, torch, xw, XA, XB, XC, xw.cutoff, 1, 1, stream)
            extras[xw.name] = {"value": 2.0 * xw.macs / (xms * 1e-3) / 1e9, "unit": UNIT, "ms": xms,
                               "roofline": roofline_of(xprof, xw.limbs), "steps": 1, "warmup": 1}
            del XA, XB, XC
            torch.cuda.empty_cache()
        extras[WL.DD_LU_4096.name] = time_lu(P, torch, WL.DD_LU_4096, device, stream, K=256)
        extras[WL.DD_LU_4096_OZ2.name] = time_lu(P, torch, WL.DD_LU_4096_OZ2, device, stream, K=256)
        extras[WL.QD_LU_2048.name] = time_lu(P, torch, WL.QD_LU_2048, device, stream, K=256)
        extras["batched_1000_mixed"] = time_batched(P, torch, device, stream)
        line["extras"] = extras

    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        line["cpu_baseline"] = cpu_oracle_rate(w, args.cpu_seconds)
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
    r = time_lu(P, torch, w, device, stream, K=args.lu_k)
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


def main():
    args = parse()
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
