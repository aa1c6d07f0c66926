"""Autotuner for DD / QD products (the tuning of block size and recursion
depth that Kouya 2015, Section 5, leaves as future work).

Batched products (tune / choose): for a shape bucket (limb count and the
binary order of m, l, n) it times the candidate configurations -- Block,
and Winograd / Strassen with cutoffs that split at least once -- on a small
batch of that shape through the batched grouped launch, and keeps the
fastest.

Single products (tune_product / choose_product): the same candidates, each
also with the Block base case converting its operands once or tile by tile
(accum "fx" / "fx_tile"), and, when the caller accepts normwise accuracy,
the CRT product on the tensor cores with the fewest moduli N whose scaling
precision P meets the requested bits (the slice count of the precision
path: moduli_for). The Block kernel's register tile (16 x 32 outputs for
DD, 8 x 32 for QD) is compiled per limb count, not a run-time choice.

The table is stored as JSON keyed by GPU name, so a later process reuses
it; shapes without an entry fall back to a model: Winograd when the
smallest dimension exceeds 512 (cutoff 256, or 1/32 of the dimension above
8192), Block otherwise.

Choices never change results beyond the chosen algorithm's bound.
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


def moduli_for(l: int, bits: int = 104) -> int:
    """The fewest CRT moduli N whose scaling precision P (ddg_ozaki2_precision)
    is at least bits + ceil(log2 l): the per-entry error l 2^-P of the row /
    column scale is then within 2^-bits of it; 0 if no N <= 40 reaches it."""
    need = bits + max(0, (int(l) - 1).bit_length())
    for N in range(2, 41):
        if capi.ddg_ozaki2_precision(N, l) >= need:
            return N
    return 0


def default_choice(limbs: int, m: int, l: int, n: int):
    """Winograd once the smallest dimension exceeds 512, with leaves of 256
    (the best of the n = 4096 and n = 8192 cutoff sweeps) or, above 8192, of
    1/32 of the dimension (at most five levels: deeper recursions queue
    thousands of launches on each of the seven streams); Block otherwise."""
    mn = min(m, l, n)
    if mn > 512:
        return "winograd", max(256, (1 << (mn - 1).bit_length()) // 32)
    return "block", 512


def _read_table(path: str) -> dict:
    """The stored tables by GPU name ({} if the file is absent or unreadable)."""
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return {}
    return data if isinstance(data, dict) else {}


class Tuner:
    def __init__(self, path: str | None = None):
        from . import build
        self.path = path or os.environ.get("DDG_TUNE_TABLE") or os.path.join(build.OUT_DIR, "tune.json")
        self.gpu = self._gpu_name()
        self.table = _read_table(self.path).get(self.gpu, {})

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

    def product_candidates(self, limbs: int, m: int, l: int, n: int, allow_normwise: bool = False,
                           bits: int = 104):
        out = [dict(algo="block", cutoff=512, accum="fx", slices=0),
               dict(algo="block", cutoff=512, accum="fx_tile", slices=0)]
        for c in CUTOFFS:
            if min(m, l, n) > c:
                for algo in ("winograd", "strassen"):
                    out.append(dict(algo=algo, cutoff=c, accum="fx", slices=0))
        if allow_normwise and limbs == 2 and l <= 65536 and m <= 65535:
            N = moduli_for(l, bits)
            if N:
                out.append(dict(algo="ozaki2_tc", cutoff=512, accum="fx", slices=N))
        return out

    def tune_product(self, limbs: int, m: int, l: int, n: int, allow_normwise: bool = False, bits: int = 104,
                     reps: int = 3):
        """Time every single-product candidate (dd_gemm / qd_gemm); store the
        fastest under the bucket (and accuracy class) of this shape."""
        import torch

        from . import gemm
        dev = torch.device("cuda")
        g = torch.Generator(device=dev).manual_seed(4321)
        A = torch.rand((limbs, m, l), generator=g, device=dev, dtype=torch.float64) * 2 - 1
        B = torch.rand((limbs, l, n), generator=g, device=dev, dtype=torch.float64) * 2 - 1
        for T in (A, B):
            for q in range(1, limbs):
                T[q] = T[q - 1] * (2.0 ** -54) * torch.rand_like(T[q])
        C = torch.empty((limbs, m, n), device=dev, dtype=torch.float64)
        s = torch.cuda.current_stream()
        best, results = None, {}
        for cand in self.product_candidates(limbs, m, l, n, allow_normwise, bits):
            kw = dict(cand)
            gemm(A, B, C, **kw)  # warm-up (workspace, module load)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(reps):
                gemm(A, B, C, **kw)
            e1.record(s)
            torch.cuda.synchronize()
            dt = e0.elapsed_time(e1) * 1e-3 / reps
            key = f"{cand['algo']}:{cand['cutoff']}:{cand['accum']}:{cand['slices']}"
            results[key] = dt
            if best is None or dt < best[0]:
                best = (dt, cand)
        entry = dict(best[1], seconds=best[0], timings=results)
        self.table[self._pkey(limbs, m, l, n, allow_normwise, bits)] = entry
        return dict(best[1])

    @staticmethod
    def _pkey(limbs, m, l, n, allow_normwise, bits):
        return f"p:{bucket(limbs, m, l, n)}:{'normwise' if allow_normwise else 'elementwise'}:{bits}"

    def choose_product(self, limbs: int, m: int, l: int, n: int, allow_normwise: bool = False, bits: int = 104):
        """Options for one product (algo, cutoff, accum, slices): the tuned
        entry of this bucket, else the model (elementwise-class algorithms)."""
        e = self.table.get(self._pkey(limbs, m, l, n, allow_normwise, bits))
        if e:
            return {k: e[k] for k in ("algo", "cutoff", "accum", "slices")}
        algo, cutoff = default_choice(limbs, m, l, n)
        return dict(algo=algo, cutoff=cutoff, accum="fx", slices=0)

    def save(self):
        data = _read_table(self.path)
        data[self.gpu] = self.table
        os.makedirs(os.path.dirname(self.path) or ".", exist_ok=True)
        tmp = self.path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def ensure_capi():
    capi.load()
