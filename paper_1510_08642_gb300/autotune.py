"""Autotuner for the recursion cutoff of DD / QD products (the tuning of block
size and recursion depth that Kouya 2015, Section 5, leaves as future work).

For a shape bucket (limb count and the binary order of m, l, n) it times the
candidate configurations -- Block, and Winograd / Strassen with cutoffs that
split at least once -- on a small batch of that shape through the batched
grouped launch, and keeps the fastest. The table is stored as JSON keyed by
GPU name, so a later process reuses it; shapes without an entry fall back to
a model: Winograd when the smallest dimension exceeds 512 (cutoff 256, or
1/32 of the dimension above 8192), Block otherwise.

Timing only: choices never change results beyond the algorithms' bounds.
"""
from __future__ import annotations

import json
import math
import os
import time

from . import capi

CUTOFFS = (128, 256, 512)


def bucket(limbs: int, m: int, l: int, n: int) -> str:
    b = lambda x: int(round(math.log2(max(x, 1))))  # noqa: E731
    return f"{limbs}:{b(m)}:{b(l)}:{b(n)}"


def default_choice(limbs: int, m: int, l: int, n: int):
    """Winograd once the smallest dimension exceeds 512, with leaves of 256
    (the best of the n = 4096 and n = 8192 cutoff sweeps) or, above 8192, of
    1/32 of the dimension (at most five levels: deeper recursions queue
    thousands of launches on each of the seven streams); Block otherwise."""
    mn = min(m, l, n)
    if mn > 512:
        return "winograd", max(256, (1 << (mn - 1).bit_length()) // 32)
    return "block", 512


class Tuner:
    def __init__(self, path: str | None = None):
        from . import build
        self.path = path or os.environ.get("DDG_TUNE_TABLE") or os.path.join(build.OUT_DIR, "tune.json")
        self.gpu = self._gpu_name()
        self.table = {}
        if os.path.exists(self.path):
            try:
                self.table = json.load(open(self.path)).get(self.gpu, {})
            except (OSError, ValueError):
                self.table = {}

    @staticmethod
    def _gpu_name() -> str:
        try:
            import torch
            return torch.cuda.get_device_name(0) if torch.cuda.is_available() else "cpu"
        except Exception:
            return "unknown"

    def choose(self, limbs: int, m: int, l: int, n: int):
        e = self.table.get(bucket(limbs, m, l, n))
        if e:
            return e["algo"], e["cutoff"]
        return default_choice(limbs, m, l, n)

    def candidates(self, m: int, l: int, n: int):
        out = [("block", 512)]
        for c in CUTOFFS:
            if min(m, l, n) > c:
                out.append(("winograd", c))
                out.append(("strassen", c))
        return out

    def tune(self, limbs: int, m: int, l: int, n: int, copies: int = 4, reps: int = 3):
        """Time every candidate on `copies` products of this shape; store the best."""
        import torch

        from . import Batch, problem
        dev = torch.device("cuda")
        g = torch.Generator(device=dev).manual_seed(1234)
        A = torch.rand((limbs, m, l), generator=g, device=dev, dtype=torch.float64) * 2 - 1
        B = torch.rand((limbs, l, n), generator=g, device=dev, dtype=torch.float64) * 2 - 1
        for T in (A, B):
            for q in range(1, limbs):
                T[q] = T[q - 1] * (2.0 ** -54) * torch.rand_like(T[q])
        Cs = [torch.empty((limbs, m, n), device=dev, dtype=torch.float64) for _ in range(copies)]
        best = None
        results = {}
        for algo, cutoff in self.candidates(m, l, n):
            b = Batch([problem(A, B, C, algo, cutoff) for C in Cs], use_graph=True)
            b.run()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                b.run()
            torch.cuda.synchronize()
            dt = (time.perf_counter() - t0) / reps
            b.close()
            results[f"{algo}:{cutoff}"] = dt
            if best is None or dt < best[0]:
                best = (dt, algo, cutoff)
        self.table[bucket(limbs, m, l, n)] = {"algo": best[1], "cutoff": best[2], "seconds": best[0],
                                             "timings": results}
        return best[1], best[2]

    def save(self):
        data = {}
        if os.path.exists(self.path):
            try:
                data = json.load(open(self.path))
            except (OSError, ValueError):
                data = {}
        data[self.gpu] = self.table
        os.makedirs(os.path.dirname(self.path) or ".", exist_ok=True)
        tmp = self.path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def ensure_capi():
    capi.load()
