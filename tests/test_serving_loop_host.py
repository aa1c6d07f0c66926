"""The serving loop's scheduling on the CPU, with the device replaced.

`Server.run` and the methods that queue work run as written; the CUDA
streams, events and the library calls (operand generation, batch plans,
dd_getrf / dd_getrs) are fakes that keep a simulated timeline per stream:
work queued on a stream ends a fixed time after the stream's previous work,
and an event recorded on the stream completes then. The tests check what the
loop promises: every request served, slots used by one unit at a time and by
the right kind, the HBM budget never exceeded by the work in flight, batches
no larger than max_batch, deadlines, and that a library call that fails ends
its requests as errors while the others are served (faults injected on the
host: nothing runs on a GPU).
"""
import contextlib
import itertools
import threading
import time

import pytest
import torch

import paper_1510_08642_gb300 as P
from paper_1510_08642_gb300 import capi
from paper_1510_08642_gb300 import serving as S

GEMM_S = 1.5e-3  # simulated device time of one product in a batch
LU_S = 4e-3      # ... of one solve


class Stream:
    """A stream of the simulated device: work runs in order."""
    ids = itertools.count()

    def __init__(self, device=None, priority=0):
        self.idx = next(Stream.ids)
        self.free_at = 0.0
        self.lock = threading.Lock()

    def enqueue(self, seconds):
        with self.lock:
            now = time.perf_counter()
            start = max(self.free_at, now)
            self.free_at = start + seconds
            return now, start, self.free_at


class Event:
    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream):
        with stream.lock:
            self.t = max(stream.free_at, time.perf_counter())

    def query(self):
        return time.perf_counter() >= self.t

    def elapsed_time(self, other):
        return (other.t - self.t) * 1e3


class Device:
    """The fake library: records every unit of work it is given."""

    def __init__(self, fail_gemm=(), fail_lu=(), bug_lu=()):
        self.fail_gemm, self.fail_lu, self.bug_lu = set(fail_gemm), set(fail_lu), set(bug_lu)
        self.units = []  # (kind, stream idx, queued at, busy from, busy until, orders)
        self.seeds = []
        self.lock = threading.Lock()

    def log(self, kind, stream, seconds, orders):
        queued, start, end = stream.enqueue(seconds)
        with self.lock:
            self.units.append((kind, stream.idx, queued, start, end, tuple(orders)))

    def make_operands(self, req, device):
        with self.lock:
            self.seeds.append(req.seed)
        A = torch.zeros((2, req.n, req.n), dtype=torch.float64)
        return (A, A.clone()) if req.kind == "gemm" else (A,)

    def problem(self, A, B, C, algo, cutoff):
        return C.shape[1]

    def Batch(self, probs, use_graph=False, stream=None):
        dev = self
        if dev.fail_gemm & set(probs):
            raise capi.DDGError(capi.DDG_EINVAL, "batch plan refused (injected)")

        class Plan:
            def run(self, s):
                dev.log("gemm", s, GEMM_S * len(probs), probs)

            def close(self, s):
                pass
        return Plan()

    def gemm(self, A, ones, algo="block", stream=None):
        return torch.zeros((2, A.shape[1], 1), dtype=torch.float64)

    def getrf(self, A, K, pivot, algo, cutoff, info, stream):
        n = A.shape[1]
        if n in self.bug_lu:
            raise TypeError("a bug in the caller (injected)")
        if n in self.fail_lu:
            raise capi.DDGError(capi.DDG_ENOMEM, "workspace exhausted (injected)")
        self.log("lu", stream, LU_S, [n])
        return torch.zeros(n, dtype=torch.int64)

    def getrs(self, LU, ipiv, b, stream=None):
        return b


@pytest.fixture
def device(monkeypatch):
    dev = Device()
    default = Stream()
    monkeypatch.setattr(torch.cuda, "Stream", Stream)
    monkeypatch.setattr(torch.cuda, "Event", Event)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "current_stream", lambda device=None: default)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 0)
    monkeypatch.setattr(torch.cuda, "set_device", lambda device: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda device=None: None)
    monkeypatch.setattr(capi, "load", lambda path=None: None)
    for name in ("make_operands", "problem", "Batch", "getrf", "getrs"):
        monkeypatch.setattr(S, name, getattr(dev, name))
    monkeypatch.setattr(P, "gemm", dev.gemm)
    return dev


def server(**kw):
    kw.setdefault("workspace_reserve", 0)
    return S.Server(device=torch.device("cpu"), **kw)


def mix(count, rate, seed, gemm_n=(24, 96), lu_n=(40, 64, 80)):
    return S.poisson_requests(count, rate, seed, gemm_n=gemm_n, lu_n=lu_n)


def wait_done(reqs):
    """Every request ended, and none before it arrived."""
    for r in reqs:
        assert r.status in ("ok", "refused", "timeout", "error"), (r.rid, r.status)
        assert r.done >= r.arrival - 1e-3, (r.rid, r.done, r.arrival)


def test_every_request_served_slots_exclusive_and_by_kind(device):
    srv = server(slots=4, lu_slots=2, max_batch=5)
    reqs = mix(60, 2000.0, seed=3)
    st = srv.run(reqs)
    wait_done(reqs)
    assert all(r.status == "ok" for r in reqs)
    assert st["all"]["count"] == 60 and st["refused"] == st["timeout"] == st["error"] == 0
    assert st["gemm"]["count"] + st["lu"]["count"] == 60
    served = sorted(n for u in device.units for n in u[5])
    assert served == sorted(r.n for r in reqs)
    lu_ids = {s.idx for s in srv.streams[:2]}
    for kind, idx, queued, start, end, orders in device.units:
        # solves on the LU slots, batches of at most max_batch on the others
        assert (idx in lu_ids) == (kind == "lu"), (kind, idx)
        assert len(orders) <= (5 if kind == "gemm" else 1)
        # a slot takes new work only after its previous unit has completed
        assert start <= queued + 1e-9, (kind, idx, queued, start)
    # requests that arrive together are batched, max_batch at a time
    device.units.clear()
    together = mix(24, 0.0, seed=9)
    srv.run(together)
    srv.close()
    sizes = [len(u[5]) for u in device.units if u[0] == "gemm"]
    assert max(sizes) == 5 and sum(sizes) == sum(r.kind == "gemm" for r in together)


def test_work_in_flight_stays_within_the_budget(device):
    reqs = mix(40, 0.0, seed=4)
    biggest = max(S.footprint(r) for r in reqs)
    srv = server(slots=6, lu_slots=3, hbm_budget=int(1.5 * biggest))
    st = srv.run(reqs)
    srv.close()
    wait_done(reqs)
    assert st["all"]["count"] == 40
    fp = {("gemm", r.n): S.footprint(r) for r in reqs if r.kind == "gemm"}
    fp.update({("lu", r.n): S.footprint(r) for r in reqs if r.kind == "lu"})
    units = [(u[2], u[4], sum(fp[(u[0], n)] for n in u[5])) for u in device.units]
    most = 0
    for t, _, own in units:
        # the units whose device work overlaps time t (the server holds
        # their bytes at least that long) fit the budget, unless one is alone
        busy = [b for (q, e, b) in units if q <= t < e]
        assert sum(busy) <= srv.budget or len(busy) == 1, (t, busy)
        most = max(most, len(busy))
    assert most > 1  # the budget let small units overlap


def test_failures_end_as_errors_and_the_rest_is_served(device):
    reqs = mix(50, 3000.0, seed=5)
    lu_fail = next(r.n for r in reqs if r.kind == "lu")
    gemm_fail = next(r.n for r in reqs if r.kind == "gemm")
    device.fail_lu.add(lu_fail)
    device.fail_gemm.add(gemm_fail)
    srv = server(slots=4, lu_slots=2, max_batch=4)
    st = srv.run(reqs)
    srv.close()
    wait_done(reqs)
    bad = [r for r in reqs if r.status == "error"]
    assert bad and st["error"] == len(bad)
    assert st["all"]["count"] == 50 - len(bad)
    for r in bad:
        assert r.result is None
        if r.kind == "lu":
            assert r.n == lu_fail and "ENOMEM" in r.error and "injected" in r.error
        else:
            assert "EINVAL" in r.error and "injected" in r.error
    # every failed solve was of the failing order, and every solve of it failed
    assert {r.rid for r in reqs if r.kind == "lu" and r.n == lu_fail} == {r.rid for r in bad if r.kind == "lu"}
    # every product of the failing order failed (with the rest of its batch)
    assert all(r.status == "error" for r in reqs if r.kind == "gemm" and r.n == gemm_fail)
    assert any(r.kind == "gemm" and r.status == "ok" for r in reqs)
    # slots came back after a failure: work admitted after the first one was served
    assert any(r.status == "ok" and r.admitted > min(b.admitted for b in bad) for r in reqs)


def test_a_bug_in_queued_work_is_not_swallowed(device):
    reqs = mix(10, 0.0, seed=6)
    device.bug_lu.add(next(r.n for r in reqs if r.kind == "lu"))
    srv = server(slots=2, lu_slots=1)
    with pytest.raises(TypeError, match="injected"):
        srv.run(reqs)
    srv.close()


def test_deadline_cancels_before_launch(device):
    # one request at a time (budget), each solve 4 ms: requests behind the
    # first few wait longer than their 5 ms deadline and are cancelled
    reqs = [S.Request(i, "lu", 64, 0.0, 1000 + i, deadline=5e-3) for i in range(12)]
    srv = server(slots=2, lu_slots=1, hbm_budget=S.footprint(reqs[0]))
    st = srv.run(reqs)
    srv.close()
    wait_done(reqs)
    late = [r for r in reqs if r.status == "timeout"]
    assert late and st["timeout"] == len(late)
    assert st.get("all", {"count": 0})["count"] == 12 - len(late)
    launched = set(device.seeds)
    assert all(r.seed not in launched for r in late)
    assert all(r.seed in launched for r in reqs if r.status == "ok")
    assert all("not admitted within" in r.error for r in late)


def test_refusals_never_reach_the_device(device):
    reqs = mix(8, 0.0, seed=7)
    reqs += [S.Request(100, "qr", 64, 0.0, 1), S.Request(101, "lu", 0, 0.0, 2),
             S.Request(102, "gemm", 10 ** 6, 0.0, 3)]
    srv = server(slots=2, lu_slots=1)
    st = srv.run(reqs)
    srv.close()
    wait_done(reqs)
    assert st["refused"] == 3 and st["all"]["count"] == 8
    assert not {1, 2, 3} & set(device.seeds)
