"""Continuous-batching request server for DD products and DD linear solves.

The paper's Section 4 application (A x = b by blocked LU whose trailing
update is the Winograd DD product) and the DD product itself, served to
requests that arrive over time:

* arrival: requests (GEMM of order n, or an LU solve of order n) arrive at
  given times (a Poisson process for the rate sweeps);
* admission: a request is admitted when its HBM footprint (operands,
  result and the library's temporaries) fits in the memory budget next to
  the requests in flight and a slot (CUDA stream) is free; its operands
  are then created on the device and stay there until it completes;
* batching: all GEMM requests admitted together form one batch plan
  (grouped persistent launches of the library); each LU solve takes a slot
  of its own (dd_getrf with Winograd trailing updates, then dd_getrs);
  slots are split between GEMM batches and LU solves so that short products
  do not wait behind long solves; a solve's launches are queued by a worker
  thread of its slot, so that the loop keeps admitting GEMMs meanwhile;
* continuous: requests that arrive while others run are admitted as slots
  and memory free up, so their work overlaps on the device;
* completion: a CUDA event per unit of work; latency = completion time on
  the device clock (relative to a reference event) minus arrival time;
* workspace: the library's temporaries come from its pool, reserved at
  start-up (ddg_workspace_reserve) so that no request maps memory;
* refusal and deadlines: a malformed request (unknown kind, order < 1 or
  above the server's limit) or one whose footprint can never fit the budget
  is refused at arrival; a request still queued past its admission deadline
  (seconds after arrival) is cancelled before anything of it is launched.
  Work already on the GPU always runs to completion (kernels are not
  interrupted), so a deadline bounds the wait for admission, not the run;
* failures: a unit of work whose library call or device allocation raises
  (a refused plan, a failed launch, device memory exhausted) ends its
  requests with status "error" and the reason; its slot is handed back once
  whatever it had queued has finished, and the loop serves the others.

Every arithmetic step runs in the CUDA library; this module only schedules.
Operands are generated on the device from a seed per request (uniform
[-1, 1) leading limbs, lower limbs 2^-53 U[-1/2, 1/2) below), so a request
gives the same result alone and in any mix.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import Batch, capi, getrf, getrs, problem


@dataclass
class Request:
    rid: int
    kind: str            # "gemm" or "lu"
    n: int
    arrival: float       # seconds after the start of the run
    seed: int
    deadline: float = math.inf  # latest admission, seconds after arrival
    admitted: float = math.nan
    done: float = math.nan
    result: object = None   # device tensor (C, or x for an LU solve)
    info: int = 0           # LU: 0 or 1 + column of a zero pivot
    status: str = "queued"  # queued, running, ok, refused, timeout, error
    error: str = ""         # why a request was refused, cancelled or failed
    operands: tuple = ()    # with keep_results: (A, B) of a GEMM, (A, b) of a solve

    @property
    def latency(self) -> float:
        return self.done - self.arrival

    @property
    def work(self) -> float:
        """2 m l n of the product, or 2 n^3 / 3 for the solve."""
        return 2.0 * self.n ** 3 if self.kind == "gemm" else 2.0 * self.n ** 3 / 3.0


def footprint(req: Request) -> int:
    """Device bytes a request holds while in flight (DD: 16 bytes/entry)."""
    n2 = req.n * req.n * 16
    if req.kind == "gemm":
        return 3 * n2 + 4 * n2          # A, B, C and Winograd temporaries (< 3.5 n^2 entries)
    return n2 + 2 * req.n * 16 + n2     # A (factored in place), b / x, temporaries of the updates


KINDS = ("gemm", "lu")


def check_request(req: Request, budget: int, max_n: int) -> str:
    """Why the server refuses `req` at arrival ("" if it can be served)."""
    if req.kind not in KINDS:
        return f"unknown request kind {req.kind!r}"
    if not isinstance(req.n, (int, np.integer)) or req.n < 1:
        return f"order must be a positive integer, got {req.n!r}"
    if req.n > max_n:
        return f"order {req.n} above the server's limit {max_n}"
    if footprint(req) > budget:
        return f"footprint {footprint(req)} B above the HBM budget {budget} B"
    return ""


def expired(req: Request, now: float) -> bool:
    """Whether a queued request has passed its admission deadline."""
    return now - req.arrival > req.deadline


def make_operands(req: Request, device):
    import torch
    g = torch.Generator(device=device).manual_seed(req.seed)

    def dd(rows, cols):
        T = torch.empty((2, rows, cols), dtype=torch.float64, device=device)
        T[0].uniform_(-1.0, 1.0, generator=g)
        T[1] = T[0] * (2.0 ** -53) * (torch.rand((rows, cols), generator=g, dtype=torch.float64,
                                                 device=device) - 0.5)
        return T

    if req.kind == "gemm":
        return dd(req.n, req.n), dd(req.n, req.n)
    A = dd(req.n, req.n)
    return (A,)


def poisson_requests(count: int, rate: float, seed: int, gemm_n=(256, 2048), lu_n=(1024, 2048, 4096)):
    """The serving workload: Poisson arrivals at `rate` per second, 50% DD
    GEMMs (n log-uniform in gemm_n), 50% DD LU solves (n uniform from lu_n)."""
    from . import inputs as I
    u = I.uniform01(seed, 4 * count).reshape(count, 4)
    gaps = -np.log1p(-u[:, 0]) / rate if rate > 0 else np.zeros(count)
    t = np.cumsum(gaps) - gaps[0]
    reqs = []
    for i in range(count):
        if u[i, 1] < 0.5:
            lo, hi = gemm_n
            n = int(round(math.exp(math.log(lo) + u[i, 2] * (math.log(hi) - math.log(lo)))))
            reqs.append(Request(i, "gemm", n, float(t[i]), seed * 100003 + i))
        else:
            n = int(lu_n[min(int(u[i, 2] * len(lu_n)), len(lu_n) - 1)])
            reqs.append(Request(i, "lu", n, float(t[i]), seed * 100003 + i))
    return reqs


@dataclass
class Unit:
    kind: str
    reqs: list
    slot: int
    event: object
    bytes: int
    keep: list = field(default_factory=list)
    future: object = None  # an LU solve still being queued by its worker thread
    info: object = None    # an LU solve's device info tensor
    error: str = ""        # set if queueing the unit's work raised


class Server:
    def __init__(self, device=None, slots: int = 4, hbm_budget: int = 64 << 30, max_batch: int = 32,
                 lu_slots: int | None = None,
                 gemm_algo: str = "winograd", gemm_cutoff: int = 256, lu_K: int = 256,
                 lu_algo: str = "winograd", lu_cutoff: int = 512, keep_results: bool = False,
                 workspace_reserve: int = 8 << 30, max_n: int = 16384):
        import torch
        self.torch = torch
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        capi.load()
        # slots [0, lu_slots) take LU solves, the others GEMM batches, so that
        # short products are not queued behind long solves; GEMM slots get the
        # higher stream priority, so their blocks are scheduled first while a
        # solve keeps the GPU busy
        self.lu_slots = max(1, slots // 2) if lu_slots is None else lu_slots
        self.streams = [torch.cuda.Stream(device=self.device, priority=0 if i < self.lu_slots else -1)
                        for i in range(slots)]
        self.budget = hbm_budget
        self.max_batch = max_batch
        self.gemm_algo, self.gemm_cutoff = gemm_algo, gemm_cutoff
        self.lu_K, self.lu_algo, self.lu_cutoff = lu_K, lu_algo, lu_cutoff
        self.keep_results = keep_results
        self.max_n = max_n
        # keep the library's temporaries mapped between requests (the solves
        # synchronise the host, which would otherwise hand the pool back)
        self.dev_index = self.device.index if self.device.index is not None else torch.cuda.current_device()
        self.workspace_reserve = workspace_reserve
        if workspace_reserve:
            capi.ddg_workspace_reserve(self.dev_index, workspace_reserve)
        # an LU solve queues thousands of launches; a worker thread per LU
        # slot queues them (the library's calls release the GIL) while this
        # loop keeps admitting and launching GEMM batches
        from concurrent.futures import ThreadPoolExecutor
        self.workers = ThreadPoolExecutor(max_workers=max(1, self.lu_slots))

    def close(self):
        """Stop the worker threads; return the reserved workspace to the device."""
        self.workers.shutdown(wait=True)
        if self.workspace_reserve:
            self.torch.cuda.synchronize(self.device)
            capi.ddg_workspace_release(self.dev_index)
            self.workspace_reserve = 0

    # -- dispatch -----------------------------------------------------------
    def _start_gemms(self, reqs, slot):
        torch = self.torch
        s = self.streams[slot]
        keep, probs, error = [], [], ""
        with torch.cuda.stream(s):
            try:
                for r in reqs:
                    A, B = make_operands(r, self.device)
                    C = torch.empty((2, r.n, r.n), dtype=torch.float64, device=self.device)
                    keep += [A, B, C]
                    algo = self.gemm_algo if r.n > self.gemm_cutoff else "block"
                    probs.append(problem(A, B, C, algo, self.gemm_cutoff))
                    r.result = C
                    if self.keep_results:
                        r.operands = (A, B)
                batch = Batch(probs, use_graph=False, stream=s)
                try:
                    batch.run(s)
                finally:
                    batch.close(s)
            except RuntimeError as e:  # the library's refusals, CUDA and allocation errors
                error = f"{type(e).__name__}: {e}"
            # recorded in every case: the slot is free again once whatever
            # was queued on it has run
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(s)
        return Unit("gemm", reqs, slot, ev, sum(footprint(r) for r in reqs), keep, error=error)

    def _start_lu(self, r, slot):
        fut = self.workers.submit(self._queue_lu, r, slot)
        return Unit("lu", [r], slot, None, footprint(r), [], future=fut)

    def _queue_lu(self, r, slot):
        """Worker thread: queue one solve on its slot's stream; returns the
        completion event, the tensors to keep until then, the device info
        tensor and the error text ("" if everything was queued)."""
        torch = self.torch
        torch.cuda.set_device(self.device)
        s = self.streams[slot]
        keep, info, error = [], None, ""
        with torch.cuda.stream(s):
            try:
                (A,) = make_operands(r, self.device)
                ones = torch.zeros((2, r.n, 1), dtype=torch.float64, device=self.device)
                keep += [A, ones]
                ones[0] = 1.0
                from . import gemm
                b = gemm(A, ones, algo="block", stream=s)
                keep.append(b)
                if self.keep_results:  # the system as posed, before A is factored in place
                    r.operands = (A.clone(), b.clone())
                info = torch.zeros(1, dtype=torch.int64, device=self.device)
                keep.append(info)
                ipiv = getrf(A, K=self.lu_K, pivot=True, algo=self.lu_algo, cutoff=self.lu_cutoff,
                             info=info, stream=s)
                keep.append(ipiv)
                getrs(A, ipiv, b, stream=s)
                r.result = b
            except RuntimeError as e:  # the library's refusals, CUDA and allocation errors
                error = f"{type(e).__name__}: {e}"
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(s)
        return ev, keep, info, error

    # -- device clock -------------------------------------------------------
    def _clock_start(self):
        """Drain the device and record the run's time origin on it."""
        torch = self.torch
        torch.cuda.synchronize(self.device)
        self._ref = torch.cuda.Event(enable_timing=True)
        self._ref.record(torch.cuda.current_stream(self.device))
        torch.cuda.synchronize(self.device)

    def _device_seconds(self, event) -> float:
        """Seconds from the run's time origin to a completed event."""
        return self._ref.elapsed_time(event) * 1e-3

    # -- loop ---------------------------------------------------------------
    def run(self, requests, poll_s: float = 2e-4):
        """Serve `requests` (arrival times relative to the start); returns stats.
        Refused, cancelled and failed requests end with status "refused" /
        "timeout" / "error" and their reason in `error`; the others with
        status "ok"."""
        torch = self.torch
        pending = sorted(requests, key=lambda r: r.arrival)
        for r in requests:
            r.status, r.error = "queued", ""
        queue, inflight = [], []
        free_lu = list(range(self.lu_slots))
        free_gemm = list(range(self.lu_slots, len(self.streams)))
        if not free_gemm:
            free_gemm = free_lu  # one shared pool
        used = 0
        self._clock_start()
        t0 = time.perf_counter()
        done = 0
        ip = 0
        while done < len(requests):
            now = time.perf_counter() - t0
            while ip < len(pending) and pending[ip].arrival <= now:
                r = pending[ip]
                ip += 1
                why = check_request(r, self.budget, self.max_n)
                if why:
                    r.status, r.error, r.done = "refused", why, now
                    done += 1
                else:
                    queue.append(r)
            for r in [r for r in queue if expired(r, now)]:
                queue.remove(r)
                r.status, r.done = "timeout", now
                r.error = f"not admitted within {r.deadline} s of arrival"
                done += 1
            # completions
            still = []
            for u in inflight:
                if u.future is not None:
                    if not u.future.done():
                        still.append(u)
                        continue
                    # raises only what the worker did not catch (a bug)
                    u.event, u.keep, u.info, u.error = u.future.result()
                    u.future = None
                if u.event.query():
                    t_dev = self._device_seconds(u.event)
                    for r in u.reqs:
                        r.done = t_dev
                        if u.error:
                            r.status, r.error, r.result = "error", u.error, None
                            continue
                        r.status = "ok"
                        if u.info is not None:
                            r.info = int(u.info.item())
                        if not self.keep_results:
                            r.result = None
                    used -= u.bytes
                    (free_lu if u.kind == "lu" else free_gemm).append(u.slot)
                    done += len(u.reqs)
                else:
                    still.append(u)
            inflight = still
            progressed = False
            # GEMMs: every queued GEMM that fits, in arrival order, one batch per free slot
            while free_gemm:
                take, b = [], 0
                for r in queue:
                    if r.kind != "gemm" or len(take) >= self.max_batch:
                        continue
                    if used + b + footprint(r) > self.budget and (inflight or take):
                        break
                    take.append(r)
                    b += footprint(r)
                if not take:
                    break
                for r in take:
                    queue.remove(r)
                    r.admitted = time.perf_counter() - t0
                    r.status = "running"
                u = self._start_gemms(take, free_gemm.pop(0))
                inflight.append(u)
                used += u.bytes
                progressed = True
            # LU solves: the oldest queued one that fits, one per free slot
            while free_lu:
                lu = next((r for r in queue if r.kind == "lu"), None)
                if lu is None or (used + footprint(lu) > self.budget and inflight):
                    break
                queue.remove(lu)
                lu.admitted = time.perf_counter() - t0
                lu.status = "running"
                u = self._start_lu(lu, free_lu.pop(0))
                inflight.append(u)
                used += u.bytes
                progressed = True
            if not progressed:
                nxt = pending[ip].arrival - (time.perf_counter() - t0) if ip < len(pending) else poll_s
                time.sleep(max(0.0, min(poll_s, nxt)))
        torch.cuda.synchronize(self.device)
        return stats(requests)


def stats(requests) -> dict:
    """p50 / p99 latency and throughput of the served requests per kind, and
    the counts of refused, cancelled and failed ones."""
    out = {}
    for kind in ("gemm", "lu", "all"):
        rs = [r for r in requests
              if (kind == "all" or r.kind == kind) and r.status not in ("refused", "timeout", "error")]
        if not rs:
            continue
        lat = np.array([r.latency for r in rs]) * 1e3
        span = max(r.done for r in rs) - min(r.arrival for r in rs)
        out[kind] = {"count": len(rs), "p50_ms": float(np.percentile(lat, 50)),
                     "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
                     "throughput_rps": len(rs) / span if span > 0 else float("inf"),
                     "work_G2mnl_per_s": sum(r.work for r in rs) / span / 1e9 if span > 0 else float("inf")}
    out["refused"] = sum(r.status == "refused" for r in requests)
    out["timeout"] = sum(r.status == "timeout" for r in requests)
    out["error"] = sum(r.status == "error" for r in requests)
    return out


def saturation_rate(server: Server, count: int = 40, seed: int = 1) -> float:
    """Requests per second when every request is already queued at t = 0."""
    reqs = poisson_requests(count, 0.0, seed)
    st = server.run(reqs)
    return st["all"]["throughput_rps"]


def sweep(rates=(0.25, 0.5, 0.75, 0.9, 1.1), count: int = 60, seed: int = 2, server: Server | None = None):
    """p50 / p99 latency and throughput at fractions of the saturation rate
    (measured after one warm-up run: the first run of a process pays for
    module loading and the growth of the stream-ordered memory pools)."""
    server = server or Server()
    saturation_rate(server)  # warm-up
    mu = saturation_rate(server)
    rows = []
    for i, f in enumerate(rates):
        reqs = poisson_requests(count, f * mu, seed + i)
        st = server.run(reqs)
        rows.append({"rate_fraction": f, "rate_rps": f * mu, **{k: v for k, v in st.items()}})
    return {"saturation_rps": mu, "points": rows}


if __name__ == "__main__":
    import json
    import sys
    count = int(sys.argv[1]) if len(sys.argv) > 1 else 60
    print(json.dumps(sweep(count=count)))
